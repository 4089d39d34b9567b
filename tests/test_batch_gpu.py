"""Batched marginalisation (many intrinsic points, uneven mode counts and Q lengths, one
persistent launch per round replayed as a CUDA graph) against the oracle and against
single-point runs of the same points."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import mc

pytestmark = pytest.mark.gpu

TOL_MARG = 1e-4


@pytest.fixture(scope="module")
def batch_points():
    specs = W.batch_specs(6, seed=3, snr_range=(8.0, 15.0), fs=4096.0, t_range=(200, 600), m_range=(5, 21))
    for s in specs:
        s.seg_len = 2.0
    return [W.make_point(s, 100 + i) for i, s in enumerate(specs)]


def test_batch_specs_are_ragged(batch_points):
    Ms = {p["Q"].shape[1] for p in batch_points}
    Ts = {p["Q"].shape[2] for p in batch_points}
    assert len(Ms) > 2 and len(Ts) > 2
    for p in batch_points:
        lm = [tuple(x) for x in p["lm"].tolist()]
        assert (2, 2) in lm and (2, -2) in lm


@pytest.mark.parametrize("S", [(1, 1, 1), (4, 2, 4)])
def test_batch_plain_matches_oracle(lib, cuda, batch_points, S):
    h = lib.rift_ile_batch_create(batch_points)
    res = lib.rift_ile_batch_marginalize(h, seed=9, n_per_round=20000, max_evals=50000, strata=S)
    assert len(res) == len(batch_points)
    for p, (pt, r) in enumerate(zip(batch_points, res)):
        ref = mc.marginalize(pt, 9, p, mc.Prior(pt["t_lo"], pt["t_hi"]), 20000, 50000, 1e300, strata=S)
        assert r["n_evals"] == 50000 and r["rounds"] == 3
        assert abs(r["lnL_marg"] - ref["lnL_marg"]) < TOL_MARG, (p, r["lnL_marg"], ref["lnL_marg"])


def test_batch_equals_single_point_runs_with_stopping(lib, cuda, batch_points):
    """Adaptive proposals and the n_eff stopping rule per point: every point of the batch gives
    exactly what a single-point run of that point (same Philox point word) gives, although the
    points stop at different rounds."""
    kw = dict(seed=12, n_per_round=16384, max_evals=16384 * 12, n_eff_target=1.6, proposal="adaptive",
              n_bins=32, strata=(2, 2, 2))
    hb = lib.rift_ile_batch_create(batch_points)
    res = lib.rift_ile_batch_marginalize(hb, **kw)
    rounds = set()
    for p, pt in enumerate(batch_points):
        h1 = lib.rift_ile_create(pt)
        one = lib.rift_ile_marginalize(h1, point_id=p, **kw)
        assert res[p]["rounds"] == one["rounds"] and res[p]["n_evals"] == one["n_evals"], (p, res[p], one)
        assert abs(res[p]["lnL_marg"] - one["lnL_marg"]) < 1e-9
        assert abs(res[p]["n_eff"] - one["n_eff"]) < 1e-6 * max(1.0, one["n_eff"])
        rounds.add(one["rounds"])
    assert len(rounds) > 1, "test should exercise points stopping at different rounds"


def test_batch_fixed_tables_matches_oracle(lib, cuda, batch_points):
    nb = 16
    c = np.concatenate([[0.0], np.cumsum(np.linspace(1.0, 3.0, nb))])
    tab1 = (c / c[-1]).astype(np.float32)
    tab1[-1] = 1.0
    tab = np.stack([tab1, tab1[::-1].copy() * 0 + tab1, tab1])
    h = lib.rift_ile_batch_create(batch_points[:3])
    res = lib.rift_ile_batch_marginalize(h, seed=14, n_per_round=20000, max_evals=40000, proposal="adaptive",
                                         n_bins=nb, tables=tab, adapt_rounds=0, strata=(2, 2, 2))
    for p, pt in enumerate(batch_points[:3]):
        ref = mc.marginalize(pt, 14, p, mc.Prior(pt["t_lo"], pt["t_hi"]), 20000, 40000, 1e300, adaptive=True,
                             n_bins=nb, tables=tab, adapt_rounds=0, strata=(2, 2, 2))
        assert abs(res[p]["lnL_marg"] - ref["lnL_marg"]) < TOL_MARG


def test_batch_graph_is_reused_and_recaptured(lib, cuda, batch_points):
    """The handle keeps the instantiated graph of its last batched run: a second call with the same
    options replays it (same results, bit for bit), other options capture a new one (the results of
    those options), and going back gives the first results again."""
    h = lib.rift_ile_batch_create(batch_points)
    kw = dict(seed=12, n_per_round=20000, max_evals=60000, proposal="adaptive", n_bins=32)
    a = lib.rift_ile_batch_marginalize(h, **kw)
    b = lib.rift_ile_batch_marginalize(h, **kw)
    assert a == b
    c = lib.rift_ile_batch_marginalize(h, **dict(kw, seed=13))
    fresh = lib.rift_ile_batch_create(batch_points)
    assert c == lib.rift_ile_batch_marginalize(fresh, **dict(kw, seed=13))
    assert a == lib.rift_ile_batch_marginalize(h, **kw)
    lib.rift_ile_destroy(fresh)
    lib.rift_ile_destroy(h)
