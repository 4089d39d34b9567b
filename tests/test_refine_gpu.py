"""GPU: refinement of heavy samples (rift_mc_opts.refine) against the FP64 oracle.

Estimates that rest on a few samples (n_eff ~ 1) carry those samples' FP32 error; with refine the
heaviest samples of each round are evaluated again in FP64 and the estimate uses those values."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import mc

from test_parity_gpu import _peaked_tables

pytestmark = pytest.mark.gpu


def test_benchmark_round_refined_matches_oracle(lib, cuda):
    """The benchmark's own round (full-size point, 1e7 prior samples, seed 1234, strata chosen by
    the library): n_eff ~ 1, so the estimate is the heaviest sample's log weight.  With refine,
    lnL_marg agrees with the oracle evaluating all 1e7 samples within 5e-5 (half the 1e-4 bar), and
    n_eff within 1e-6 relative."""
    from oracle_pool import OraclePool
    pool = OraclePool("cfg_full", 2)   # spawned before any device work of this test
    try:
        n = 10_000_000
        h = lib.rift_ile_create(W.make_point(W.cfg_full(), 2))
        plain = lib.rift_ile_marginalize(h, seed=1234, n_per_round=n, max_evals=n)
        ref_run = lib.rift_ile_marginalize(h, seed=1234, n_per_round=n, max_evals=n, refine=1)
        lib.rift_ile_destroy(h)
        assert ref_run["n_refined"] >= 1 and plain["n_refined"] == 0
        assert tuple(ref_run["strata"]) == tuple(plain["strata"])
        want = pool.accum(1234, tuple(ref_run["strata"]), n).result()
    finally:
        pool.close()
    err = abs(ref_run["lnL_marg"] - want[0])
    assert err < 5e-5, (ref_run["lnL_marg"], plain["lnL_marg"], want[0])
    assert err <= abs(plain["lnL_marg"] - want[0]) + 1e-6
    assert abs(ref_run["n_eff"] - want[1]) <= 1e-6 * want[1], (ref_run["n_eff"], want[1])


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_refined_prior_round_matches_oracle(lib, cuda, seed):
    """Full-size point, 2e5 prior samples, stratified: refined lnL_marg within 5e-5 of the oracle."""
    pt = W.make_point(W.cfg_full(), 2)
    n = 200_000
    S = (16, 8, 16)
    h = lib.rift_ile_create(pt)
    got = lib.rift_ile_marginalize(h, seed=seed, n_per_round=n, max_evals=n, strata=S, refine=1)
    lib.rift_ile_destroy(h)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    th, _, lq = mc.draw(seed, 0, 0, np.arange(n, dtype=np.uint64), pr, None, S, n)
    want = mc.Accum.of(mc.lnL_samples(pt, th) + lq).result()
    assert got["n_refined"] >= 1
    assert abs(got["lnL_marg"] - want[0]) < 5e-5, (got["lnL_marg"], want[0], got["n_eff"])


def test_refined_adaptive_rounds_match_oracle(lib, cuda):
    """Fixed adapted tables (the inverse CDF and ln p - ln q redone in FP64), two rounds, small point."""
    p_small = W.make_point(W.cfg_small(), 1)
    nb = 64
    tab = _peaked_tables(p_small, nb)
    S = (4, 4, 4)
    h = lib.rift_ile_create(p_small)
    got = lib.rift_ile_marginalize(h, seed=25, n_per_round=50000, max_evals=100000, proposal="adaptive", n_bins=nb,
                                   tables=tab, adapt_rounds=0, strata=S, refine=1)
    lib.rift_ile_destroy(h)
    ref = mc.marginalize(p_small, 25, 0, mc.Prior(p_small["t_lo"], p_small["t_hi"]), 50000, 100000, 1e300,
                         adaptive=True, n_bins=nb, tables=tab, adapt_rounds=0, strata=S)
    assert got["n_refined"] >= 1
    assert abs(got["lnL_marg"] - ref["lnL_marg"]) < 5e-5, (got["lnL_marg"], ref["lnL_marg"])


def test_refined_batch_equals_single_point_runs(lib, cuda):
    """The batched graph runner refines each point's rounds exactly as a single-point run does."""
    specs = W.batch_specs(3, seed=12, t_range=(800, 1200))
    pts = [W.make_point(sp, 40 + i) for i, sp in enumerate(specs)]
    kw = dict(seed=83, n_per_round=40000, max_evals=120000, n_eff_target=1e300, proposal="adaptive", n_bins=32,
              refine=1)
    hb = lib.rift_ile_batch_create(pts)
    batch = lib.rift_ile_batch_marginalize(hb, **kw)
    lib.rift_ile_destroy(hb)
    for i, p in enumerate(pts):
        h = lib.rift_ile_create(p)
        one = lib.rift_ile_marginalize(h, point_id=i, **kw)
        lib.rift_ile_destroy(h)
        assert batch[i]["n_refined"] == one["n_refined"] >= 1
        assert batch[i]["lnL_marg"] == one["lnL_marg"], (i, batch[i]["lnL_marg"], one["lnL_marg"])


def test_refine_refused_where_unsupported(lib, cuda):
    """refine does not combine with save/resume, nor with the allocation-free entry point."""
    h = lib.rift_ile_create(W.make_point(W.cfg_small(), 1))
    kw = dict(seed=1, n_per_round=10000, max_evals=10000, refine=1)
    with pytest.raises(lib.RiftError):
        lib.rift_ile_marginalize(h, save=True, **kw)
    with pytest.raises(lib.RiftError):
        lib.rift_ile_marginalize_static(h, **kw)
    lib.rift_ile_destroy(h)
