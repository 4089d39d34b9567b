"""Pins of the posterior-sample oracle: systematic resampling against its closed form and its
defining count property, the time draw against the closed-form conditional of a single tone, and
the weighted export against the run's estimate and the brute-force likelihood."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workload as W
from oracle import geometry as G
from oracle import likelihood as L
from oracle import mc
from oracle import posterior as PO
from oracle.swsh import ylm_m2


def test_equal_weights_resample_to_evenly_spaced_rows():
    """Equal weights: slot h takes row floor((h + 1/2) N / H)."""
    for N, H in ((1000, 100), (997, 64), (5, 12)):
        idx, _ = PO.systematic_resample(np.full(N, -3.25), H)
        want = np.floor((np.arange(H) + 0.5) * N / H).astype(np.int64)
        assert np.array_equal(idx, want), (N, H)


def test_resample_counts_are_within_one_of_the_expected_share():
    """Each row is taken floor or ceil of H w_i / sum w times; rows of zero weight never."""
    r = np.random.default_rng(4)
    ell = r.normal(0, 3, 2000)
    ell[r.integers(0, 2000, 50)] = -np.inf
    H = 777
    idx, _ = PO.systematic_resample(ell, H)
    w = np.where(np.isfinite(ell), np.exp(ell - ell[np.isfinite(ell)].max()), 0.0)
    share = H * w / w.sum()
    cnt = np.bincount(idx, minlength=ell.size)
    assert cnt.sum() == H
    assert np.all(cnt >= np.floor(share) - 1e-9) and np.all(cnt <= np.ceil(share) + 1e-9)
    assert np.all(cnt[~np.isfinite(ell)] == 0)
    assert np.all(np.diff(idx) >= 0)


def _single_tone_point(m_cycles=2, A=3.0 + 4.0j, u=5.0):
    """One detector at the geocentre, mode (2,2), Q[n] = A exp(2 pi i m n / J) on a grid aligned with
    the quadrature times, U = u, V = 0: lnL(t_j) = a cos(2 pi m j / J + arg) - b."""
    fs, J, n0 = 256.0, 64, 8
    t_lo = -J / (2 * fs)
    tens = W.detector("H1")[0]
    T = J + 2 * n0
    tau0 = t_lo + 0.5 / fs - n0 / fs
    n = np.arange(T)
    Q = (A * np.exp(2j * np.pi * m_cycles * (n - n0) / J)).reshape(1, 1, T)
    return dict(det_tensor=tens[None], det_pos=np.zeros((1, 3)), lm=np.array([[2, 2]], dtype=np.int32), Q=Q,
                q_t0_gps=np.array([1e9 + tau0]), fs=fs, U=np.full((1, 1, 1), u, dtype=np.complex128),
                V=np.zeros((1, 1, 1), dtype=np.complex128), t_ref_gps=1e9, d_ref_mpc=100.0, t_lo=t_lo,
                t_hi=-t_lo), J


def test_time_draw_inverts_the_closed_form_conditional():
    pt, J = _single_tone_point()
    ra, dec, psi, phi, incl, dist = 1.1, 0.3, 0.7, 2.0, 0.9, 40.0
    gmst = G.gmst_from_gps(pt["t_ref_gps"])
    F = G.complex_antenna(pt["det_tensor"][0], np.array([ra]), np.array([dec]), np.array([psi]), gmst)[0]
    Y = ylm_m2([(2, 2)], np.array([incl]), np.array([phi]))[0, 0]
    x = pt["d_ref_mpc"] / dist
    z = x * F * np.conj(Y) * (3.0 + 4.0j)                               # Q at the first grid time is A
    j = np.arange(J)
    lin = np.abs(z) * np.cos(2 * np.pi * 2 * j / J + np.angle(z))     # Re(z e^{2 pi i m j / J})
    p = np.exp(lin - lin.max())
    cdf = np.cumsum(p) / p.sum()
    assert p.max() / p.min() > 10.0                                   # a conditional far from flat
    for u in (0.013, 0.2, 0.45, 0.77, 0.9999):   # 0.5 sits on a boundary: two whole periods
        jj, t, l, c = PO.time_draw(pt, ra, dec, psi, phi, incl, dist, u)
        assert jj == int(np.searchsorted(cdf, u, side="right")), u
        assert abs(t - (pt["t_lo"] + (jj + 0.5) / pt["fs"])) < 1e-15
        b = 0.25 * x * x * abs(F) ** 2 * abs(Y) ** 2 * 5.0
        assert abs(l - (lin[jj] - b)) < 1e-9 * max(1.0, abs(l))
        assert np.allclose(c, cdf, rtol=0, atol=1e-12)


@pytest.fixture(scope="module")
def small():
    return W.make_point(W.cfg_small(), 6)


def test_single_round_export_reproduces_the_estimate(small):
    pr = mc.Prior(small["t_lo"], small["t_hi"])
    n = 3000
    for kw in (dict(strata=(4, 2, 2)), dict(adaptive=True, n_bins=16, max_rounds=1)):
        S = PO.last_round(small, 31, 0, pr, n, n, 1e300, **kw)
        assert S["lnL"].size == n
        assert abs(PO.weighted_mean_log(S["lnL"], S["lnpq"]) - S["result"]["lnL_marg"]) < 1e-10
    # the prior proposal without strata weighs every draw by the likelihood alone
    S = PO.last_round(small, 32, 0, pr, 500, 500, 1e300)
    assert np.all(S["lnpq"] == 0.0)


def test_exported_rows_are_self_consistent_with_the_bruteforce_likelihood():
    """Each exported row's lnL is the frequency-domain likelihood at that row's parameters (a
    swapped or mistransformed column fails by far more than the interpolation error)."""
    spec = W.PointSpec(dets=("H1", "L1"), modes=list(W.L2_MODES), fs=4096.0, snr=10.0, t_half=0.01, seg_len=2.0)
    pt = W.make_point(spec, 12)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    S = PO.last_round(pt, 33, 0, pr, 400, 400, 1e300)
    rows = np.argsort(S["lnL"])[-4:]
    for i in rows:
        bf = L.lnL_bruteforce(pt, S["ra"][i], S["dec"][i], S["t"][i], S["psi"][i], S["phi"][i], S["incl"][i],
                              S["dist"][i])
        assert abs(S["lnL"][i] - bf) < 2e-3 * max(1.0, abs(bf)), (i, S["lnL"][i], bf)


def test_flat_likelihood_posterior_is_the_prior():
    """Q = U = V = 0: every weight is equal, so the resampled rows are evenly spaced prior draws and
    each column follows its prior (cos incl and sin dec uniform, D^3 uniform)."""
    pt = W.make_point(W.cfg_small(), 7)
    pt = dict(pt, Q=np.zeros_like(pt["Q"]), U=np.zeros_like(pt["U"]), V=np.zeros_like(pt["V"]))
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    H = 2000
    out = PO.posterior(pt, 34, 0, pr, 4000, 4000, 1e300, H)
    assert np.all(out["lnL"] == 0.0)
    assert np.array_equal(out["idx"], np.floor((np.arange(H) + 0.5) * 4000 / H).astype(np.int64))
    from scipy.stats import kstest
    for v, lo, hi in ((np.cos(out["incl"]), -1, 1), (np.sin(out["dec"]), -1, 1), (out["psi"], 0, math.pi),
                      (out["dist"] ** 3, 1.0, 1e9), (out["t"], pt["t_lo"], pt["t_hi"])):
        assert kstest((v - lo) / (hi - lo), "uniform").pvalue > 1e-3
