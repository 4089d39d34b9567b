"""Failure paths on the GPU, made on the host (RIFT_FAULT): a failed upload, a non-finite sample
and a bounded device wait that runs out.  None of them faults, traps or hangs the GPU; after
each one the handle (or a new one) keeps working and gives the same results as before."""
from __future__ import annotations

import pytest

import workload as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    return W.make_point(W.cfg_small(), 5)


KW = dict(seed=61, n_per_round=20000, max_evals=20000)


def test_injected_upload_fault(lib, cuda, pt, monkeypatch):
    monkeypatch.setenv("RIFT_FAULT", "h2d")
    with pytest.raises(lib.RiftError) as e:
        lib.rift_ile_create(pt)
    assert e.value.status == 4
    monkeypatch.delenv("RIFT_FAULT")
    h = lib.rift_ile_create(pt)
    assert lib.rift_ile_marginalize(h, **KW)["n_evals"] == 20000
    lib.rift_ile_destroy(h)


def test_injected_nan_sample(lib, cuda, pt, monkeypatch):
    h = lib.rift_ile_create(pt)
    ref = lib.rift_ile_marginalize(h, **KW)
    monkeypatch.setenv("RIFT_FAULT", "nan_sample")
    with pytest.raises(lib.RiftError) as e:
        lib.rift_ile_marginalize(h, **KW)
    assert e.value.status == 6
    monkeypatch.delenv("RIFT_FAULT")
    again = lib.rift_ile_marginalize(h, **KW)      # status word cleared; same result as before
    assert again["lnL_marg"] == ref["lnL_marg"]
    lib.rift_ile_destroy(h)


def test_bounded_wait_runs_out(lib, cuda, pt, monkeypatch):
    """The window copies are announced on the mbarrier but not issued: every CTA's bounded wait
    (about 1 s) expires, the kernel reports RIFT_ETIMEOUT and returns, and the context stays usable."""
    h = lib.rift_ile_create(pt)
    ref = lib.rift_ile_marginalize(h, **KW)
    monkeypatch.setenv("RIFT_FAULT", "stage_timeout")
    with pytest.raises(lib.RiftError) as e:
        lib.rift_ile_marginalize(h, **KW)
    assert e.value.status == 5
    monkeypatch.delenv("RIFT_FAULT")
    again = lib.rift_ile_marginalize(h, **KW)
    assert again["lnL_marg"] == ref["lnL_marg"]
    lib.rift_ile_destroy(h)
