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


@pytest.fixture(scope="module")
def point():
    return W.make_point(W.cfg_small(), 1)


def _close(a, b):
    assert a["n_evals"] == b["n_evals"] and a["rounds"] == b["rounds"]
    assert abs(a["lnL_marg"] - b["lnL_marg"]) < TOL_MARG
    assert abs(a["n_eff"] - b["n_eff"]) <= 1e-6 * max(1.0, b["n_eff"])


@pytest.mark.parametrize("kw", [
    dict(seed=5, n_per_round=60000, max_evals=150000),
    dict(seed=6, n_per_round=40000, max_evals=120000, proposal="adaptive", n_bins=64),
])
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


def test_static_rejects_rounds_beyond_its_scratch(lib, cuda, point):
    h = lib.rift_ile_create(point)
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=131073, max_evals=131073, proposal="adaptive",
                                        n_bins=32)
    assert ex.value.status == 1 and "RIFT_STATIC_MAX_ROUND" in str(ex.value)
    with pytest.raises(lib.RiftError) as ex:
        lib.rift_ile_marginalize_static(h, seed=1, n_per_round=67108865, max_evals=67108865)
    assert ex.value.status == 1 and "RIFT_STATIC_MAX_PRIOR_ROUND" in str(ex.value)
