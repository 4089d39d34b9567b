"""Pins of the warm start of the adaptive integrator (Sec. II.C and III.B: the integrator adapted on
one intrinsic point is reused for the next): the carried-over tables are exactly the proposal a
further round would use, and they move the next point's draws onto its likelihood peak."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L
from oracle import mc


@pytest.fixture(scope="module")
def small():
    return W.make_point(W.cfg_small(), 1)


@pytest.mark.parametrize("adapt_rounds,time_marg", [(-1, False), (1, False), (-1, True)])
def test_tables_next_is_the_proposal_of_the_following_round(small, adapt_rounds, time_marg):
    """A run of R rounds hands over exactly the tables round R of a longer run draws from."""
    pr = mc.Prior(small["t_lo"], small["t_hi"])
    n = 1500 if time_marg else 4000
    kw = dict(adaptive=True, n_bins=16, keep=True, adapt_rounds=adapt_rounds, time_marg=time_marg)
    short = mc.marginalize(small, 5, 0, pr, n, 2 * n, 1e300, **kw)
    long_ = mc.marginalize(small, 5, 0, pr, n, 3 * n, 1e300, **kw)
    assert np.array_equal(short["tables_next"], long_["history"][2]["tables"])
    if adapt_rounds == 1:
        assert np.array_equal(short["tables_next"], short["history"][1]["tables"])
    else:
        assert not np.array_equal(short["tables_next"], short["history"][1]["tables"])
    if time_marg:
        assert np.array_equal(short["tables_next"][2], mc.uniform_time_table(16))


def phys_point(seed, snr=10.0):
    """Physical injection (H1, L1, V1; l = 2 modes) with the template of seed `seed`: points of
    different seeds are different intrinsic points seeing the same source."""
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.L2_MODES), fs=4096.0, snr=snr, t_half=0.02,
                       seg_len=4.0)
    tens = np.stack([W.detector(d)[0] for d in spec.dets])
    pos = np.stack([W.detector(d)[1] for d in spec.dets])
    coef, tk = L.injection((tens, pos), spec.modes, ra=2.0, dec=0.5, t=0.003, psi=0.3, phi=1.0, incl=0.6,
                           dist=300.0, d_ref=spec.d_ref, t_ref_gps=spec.t_ref_gps)
    return W.make_point(spec, seed, injection=(coef, tk))


def test_warm_start_moves_the_draws_onto_the_peak():
    """Tables adapted on one intrinsic point put a clearly larger share of the next point's first
    round on its likelihood peak than the prior does (same seed, same number of draws)."""
    a, b = phys_point(41), phys_point(42)
    pr = mc.Prior(a["t_lo"], a["t_hi"])
    n = 30000
    pilot = mc.marginalize(a, 7, 0, pr, n, 6 * n, 1e300, adaptive=True, n_bins=32)
    q = {}
    for name, tab in (("cold", None), ("warm", pilot["tables_next"])):
        r = mc.marginalize(b, 9, 0, pr, n, n, 1e300, adaptive=True, n_bins=32, tables=tab, keep=True)
        h = r["history"][0]
        _, _, lpq = mc.draw(9, 0, 0, np.arange(n, dtype=np.uint64), pr, h["tables"], (1, 1, 1), n)
        q[name] = np.percentile(h["ell"] - lpq, 99)
    assert q["warm"] > q["cold"] + 5.0, q
