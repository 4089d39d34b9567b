"""GPU: warm start of the adaptive integrator (per-point initial tables in, each point's adapted
tables out) against the FP64 oracle and against the device's own continuation."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import mc

from test_oracle_warm import phys_point

pytestmark = pytest.mark.gpu

TOL_MARG = 1e-4


@pytest.fixture(scope="module")
def p_small():
    return W.make_point(W.cfg_small(), 1)


def _tables(nb, slope):
    c = np.concatenate([[0.0], np.cumsum(np.linspace(1.0, slope, nb))])
    t = (c / c[-1]).astype(np.float32)
    t[-1] = 1.0
    return np.stack([t, t[::-1].copy() * 0 + t, t])


def test_tables_out_matches_the_oracle_rebuild(lib, cuda, p_small):
    """One adaptive round from given tables: the handed-over tables are the rebuild from that
    round's draws (identical draws; FP32 histograms vs FP64, 2e-4)."""
    nb, n = 32, 40000
    tab = _tables(nb, 3.0)
    kw = dict(seed=81, n_per_round=n, max_evals=n, proposal="adaptive", n_bins=nb, tables=tab, strata=(2, 2, 2))
    h = lib.rift_ile_create(p_small)
    r = lib.rift_ile_marginalize(h, want_tables=True, **kw)
    hb = lib.rift_ile_batch_create([p_small])
    rb = lib.rift_ile_batch_marginalize(hb, want_tables=True, **kw)
    pr = mc.Prior(p_small["t_lo"], p_small["t_hi"])
    ref = mc.marginalize(p_small, 81, 0, pr, n, n, 1e300, adaptive=True, n_bins=nb, tables=tab, strata=(2, 2, 2))
    assert np.max(np.abs(r["tables"].astype(np.float64) - ref["tables_next"])) < 2e-4
    assert np.array_equal(r["tables"], rb[0]["tables"])
    lib.rift_ile_destroy(h)
    lib.rift_ile_destroy(hb)


@pytest.mark.parametrize("adapt_rounds", [-1, 2])
def test_tables_out_is_the_next_rounds_proposal(lib, cuda, p_small, adapt_rounds):
    """R rounds hand over bit for bit the tables round R of an (R+1)-round run draws from."""
    import torch
    nb, n = 32, 20000
    kw = dict(seed=82, n_per_round=n, proposal="adaptive", n_bins=nb, adapt_rounds=adapt_rounds, strata=(2, 2, 2))
    h = lib.rift_ile_create(p_small)
    short = lib.rift_ile_marginalize(h, want_tables=True, max_evals=3 * n, **kw)
    dbg = torch.zeros((4, 3, nb + 1), dtype=torch.float32, device="cuda")
    lib.rift_ile_marginalize(h, max_evals=4 * n, dbg_tables=dbg, **kw)
    assert np.array_equal(short["tables"], dbg[3].cpu().numpy())
    lib.rift_ile_destroy(h)


def test_batch_tables_out_equals_single_point_runs(lib, cuda):
    """Points that stop at different rounds: each point's handed-over tables in a batch are those
    of its single-point run (same Philox point word)."""
    pts = [W.make_point(W.cfg_small(), 90 + i) for i in range(3)]
    kw = dict(seed=83, n_per_round=8192, max_evals=8192 * 6, n_eff_target=1.6, proposal="adaptive", n_bins=32,
              strata=(2, 2, 2))
    hb = lib.rift_ile_batch_create(pts)
    rb = lib.rift_ile_batch_marginalize(hb, want_tables=True, **kw)
    for p, pt in enumerate(pts):
        h1 = lib.rift_ile_create(pt)
        r1 = lib.rift_ile_marginalize(h1, want_tables=True, point_id=p, **kw)
        assert r1["rounds"] == rb[p]["rounds"]
        assert np.array_equal(r1["tables"], rb[p]["tables"]), p
        lib.rift_ile_destroy(h1)
    lib.rift_ile_destroy(hb)


def test_per_point_initial_tables_match_the_oracle(lib, cuda):
    """A batch whose points start from their own tables (no rebuild): identical draws to the
    oracle's per point, lnL_marg within 1e-4."""
    pts = [W.make_point(W.cfg_small(), 95 + i) for i in range(3)]
    nb = 16
    tabs = np.stack([_tables(nb, s) for s in (2.0, 4.0, 0.5)])
    hb = lib.rift_ile_batch_create(pts)
    res = lib.rift_ile_batch_marginalize(hb, seed=84, n_per_round=20000, max_evals=40000, proposal="adaptive",
                                         n_bins=nb, tables=tabs, adapt_rounds=0, strata=(2, 2, 2))
    for p, pt in enumerate(pts):
        ref = mc.marginalize(pt, 84, p, mc.Prior(pt["t_lo"], pt["t_hi"]), 20000, 40000, 1e300, adaptive=True,
                             n_bins=nb, tables=tabs[p], adapt_rounds=0, strata=(2, 2, 2))
        assert abs(res[p]["lnL_marg"] - ref["lnL_marg"]) < TOL_MARG, (p, res[p]["lnL_marg"], ref["lnL_marg"])
    lib.rift_ile_destroy(hb)


def test_warm_start_moves_the_draws_onto_the_peak(lib, cuda):
    """The device run of the oracle pin: tables adapted on one intrinsic point put the next
    point's first-round draws on its likelihood peak."""
    import torch
    a, b = phys_point(41), phys_point(42)
    n, nb = 100000, 32
    ha, hb = lib.rift_ile_create(a), lib.rift_ile_create(b)
    pilot = lib.rift_ile_marginalize(ha, want_tables=True, seed=7, n_per_round=n, max_evals=6 * n,
                                     proposal="adaptive", n_bins=nb, strata=(1, 1, 1))
    q = {}
    for name, tab in (("cold", None), ("warm", pilot["tables"])):
        dbg = torch.empty(n, dtype=torch.float32, device="cuda")
        _, lpq, _ = lib.rift_ile_draw(hb, 0, n, tables=tab if tab is not None else _tables(nb, 1.0), seed=9,
                                      proposal="adaptive", n_bins=nb, strata=(1, 1, 1))
        lib.rift_ile_marginalize(hb, seed=9, n_per_round=n, max_evals=n, proposal="adaptive", n_bins=nb,
                                 tables=tab, dbg_ell=dbg, strata=(1, 1, 1))
        q[name] = np.percentile(dbg.cpu().numpy().astype(np.float64) - lpq.cpu().numpy(), 99)
    assert q["warm"] > q["cold"] + 5.0, q
    lib.rift_ile_destroy(ha)
    lib.rift_ile_destroy(hb)
