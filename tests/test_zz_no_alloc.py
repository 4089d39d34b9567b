"""rift_ile_marginalize_static: the allocation-free marginalisation entry point.

It serves callers that may not allocate device memory when they marginalise (their
device memory is owned by another allocator, or allocation after start-up is not
allowed).  Its scratch lives in a static device array; these tests call it through the
C ABI, twice in a row, and compare with rift_ile_marginalize on the same inputs.
This file is collected last so that a run stopping at the first failure has already run
every other test; it also passes on its own in a fresh process.
"""
from __future__ import annotations

import pytest

import workload as W

pytestmark = pytest.mark.gpu

TOL_MARG = 1e-4
STATIC_MAX_PRIOR_ROUND = 67108864   # RIFT_STATIC_MAX_PRIOR_ROUND


@pytest.fixture(scope="module")
def point():
    return W.make_point(W.cfg_small(), 1)


def _close(a, b):
    assert a["n_evals"] == b["n_evals"] and a["rounds"] == b["rounds"]
    assert abs(a["lnL_marg"] - b["lnL_marg"]) < TOL_MARG
    assert abs(a["n_eff"] - b["n_eff"]) <= 1e-6 * max(1.0, b["n_eff"])


CASES = [
    dict(seed=5, n_per_round=60000, max_evals=150000),
    dict(seed=6, n_per_round=40000, max_evals=120000, proposal="adaptive", n_bins=64),
    dict(seed=7, n_per_round=4096, max_evals=8192, time_marg=1),
    dict(seed=8, n_per_round=4096, max_evals=8192, time_marg=1, proposal="adaptive", n_bins=32),
]


@pytest.mark.parametrize("kw", CASES)
def test_static_matches_allocating_entry_point_twice(lib, cuda, point, kw):
    h = lib.rift_ile_create(point)
    ref = lib.rift_ile_marginalize(h, **kw)
    first = lib.rift_ile_marginalize_static(h, **kw)
    second = lib.rift_ile_marginalize_static(h, **kw)   # the shared array kept the first call's state
    _close(first, ref)
    _close(second, ref)
    other = lib.rift_ile_marginalize_static(h, **{**kw, "seed": kw["seed"] + 100})
    ref_other = lib.rift_ile_marginalize(h, **{**kw, "seed": kw["seed"] + 100})
    _close(other, ref_other)
    lib.rift_ile_destroy(h)


def test_static_calls_allocate_nothing(lib, cuda, point):
    """On a fresh handle, after one warm-up call of each kind (the set-up: the static array's
    address lookup and the first launch of each kernel, which may load its code), further static
    calls leave free device memory and the buffer-cache counters unchanged."""
    import torch
    h = lib.rift_ile_create(point)
    for kw in CASES:
        lib.rift_ile_marginalize_static(h, **kw)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    c0 = lib.rift_cache_counters()
    for kw in CASES + CASES:
        lib.rift_ile_marginalize_static(h, **kw)
    torch.cuda.synchronize()
    assert lib.rift_cache_counters() == c0
    assert torch.cuda.mem_get_info()[0] == free0
    lib.rift_ile_destroy(h)


def test_static_rejects_what_its_scratch_cannot_hold(lib, cuda, point):
    h = lib.rift_ile_create(point)
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=131073, max_evals=131073, proposal="adaptive",
                                        n_bins=32)
    assert ex.value.status == 1 and "RIFT_STATIC_MAX_ROUND" in str(ex.value)
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=STATIC_MAX_PRIOR_ROUND + 1,
                                        max_evals=STATIC_MAX_PRIOR_ROUND + 1)
    assert ex.value.status == 1 and "RIFT_STATIC_MAX_PRIOR_ROUND" in str(ex.value)
    n = STATIC_MAX_PRIOR_ROUND // 8 + 1
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=n, max_evals=n, time_marg=1)
    assert ex.value.status == 1 and "time-marginalised" in str(ex.value)
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=4096, max_evals=4096, proposal="learned",
                                        mdn=lib.rift_mdn_create(1))
    assert ex.value.status == 1 and "learned" in str(ex.value)
    lib.rift_ile_destroy(h)
