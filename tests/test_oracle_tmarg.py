"""Pins of the time-marginalised likelihood oracle, Eq. (lnL:tmarg), against closed forms,
the brute-force definition and an invariance of the time grid."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workload as W
from oracle import geometry as G
from oracle import likelihood as L
from oracle import tmarg as TM
from oracle.swsh import ylm_m2


def _single_tone_point(m_cycles, A=3.0 + 4.0j, u=50.0):
    """One detector at the geocentre (no time of flight), one mode (2,2), Q on a grid aligned with
    the quadrature times: Q[n] = A exp(2 pi i m n / J), U = u, V = 0."""
    fs, J, n0 = 256.0, 64, 8
    t_lo = -J / (2 * fs)
    tens = W.detector("H1")[0]
    T = J + 2 * n0
    tau0 = t_lo + 0.5 / fs - n0 / fs                 # (t_j - tau0) fs = n0 + j exactly
    n = np.arange(T)
    Q = (A * np.exp(2j * np.pi * m_cycles * (n - n0) / J)).reshape(1, 1, T)
    return dict(det_tensor=tens[None], det_pos=np.zeros((1, 3)), lm=np.array([[2, 2]], dtype=np.int32), Q=Q,
                q_t0_gps=np.array([1e9 + tau0]), fs=fs, U=np.full((1, 1, 1), u, dtype=np.complex128),
                V=np.zeros((1, 1, 1), dtype=np.complex128), t_ref_gps=1e9, d_ref_mpc=100.0, t_lo=t_lo,
                t_hi=-t_lo), J


@pytest.mark.parametrize("m_cycles", [3, 5])
def test_single_tone_equals_bessel_closed_form(m_cycles):
    """lnL(t_j) = a cos(2 pi m j / J + phi0) - b, whose midpoint-rule mean over whole periods is
    I0(a) exp(-b) (aliases I_{J/g}(a) are below 1e-30 here)."""
    from scipy.special import ive
    pt, J = _single_tone_point(m_cycles)
    assert TM.time_grid(pt).size == J
    ra, dec, psi, phi, incl, dist = 1.1, 0.3, 0.7, 2.0, 0.9, 80.0
    gmst = G.gmst_from_gps(pt["t_ref_gps"])
    F = G.complex_antenna(pt["det_tensor"][0], np.array([ra]), np.array([dec]), np.array([psi]), gmst)[0]
    Y = ylm_m2([(2, 2)], np.array([incl]), np.array([phi]))[0, 0]
    x = pt["d_ref_mpc"] / dist
    a = x * abs(F * np.conj(Y) * pt["Q"][0, 0, 0])
    b = 0.25 * x * x * abs(F) ** 2 * abs(Y) ** 2 * 50.0
    want = math.log(ive(0, a)) + a - b
    got = TM.lnL_tmarg(pt, ra, dec, psi, phi, incl, dist)[0]
    assert abs(got - want) < 1e-9 * max(1.0, abs(want)), (got, want, a, b)


def test_constant_in_time_is_the_plain_likelihood():
    pt, J = _single_tone_point(0)
    th = dict(ra=0.4, dec=-0.2, psi=1.3, phi=0.5, incl=2.1, dist=150.0)
    one = L.lnL_factorised(pt, t=0.0, **th)[0]
    assert abs(TM.lnL_tmarg(pt, **th)[0] - one) < 1e-12 * max(1.0, abs(one))


def test_matches_bruteforce_definition_on_the_grid():
    """With the exact Q(t) (direct frequency sum) the quadrature equals the mean of exp(lnL) of the
    brute-force frequency-domain likelihood at the same grid times."""
    spec = W.PointSpec(dets=("H1", "L1"), modes=list(W.L2_MODES), fs=4096.0, snr=8.0, t_half=0.004, seg_len=2.0)
    pt = W.make_point(spec, 3)
    tj = TM.time_grid(pt)
    th = dict(ra=2.2, dec=0.4, psi=0.9, phi=1.7, incl=0.8, dist=300.0)
    bf = np.array([L.lnL_bruteforce(pt, th["ra"], th["dec"], t, th["psi"], th["phi"], th["incl"], th["dist"])
                   for t in tj])
    want = bf.max() + math.log(np.mean(np.exp(bf - bf.max())))
    got = TM.lnL_tmarg(pt, exact=True, **{k: np.array([v]) for k, v in th.items()})[0]
    assert abs(got - want) < 1e-9 * max(1.0, abs(want))


def test_whole_sample_shift_of_data_and_window_leaves_it_unchanged():
    """Moving the Q series and the time window together by whole samples changes nothing; a grid
    that is off by half a sample (a plausible mistake) would change the result."""
    pt = W.make_point(W.cfg_small(), 4)
    fs = float(pt["fs"])
    th = dict(ra=np.array([0.3, 4.0]), dec=np.array([0.2, -0.9]), psi=np.array([0.1, 2.0]),
              phi=np.array([1.0, 5.0]), incl=np.array([0.5, 2.5]), dist=np.array([200.0, 90.0]))
    base = TM.lnL_tmarg(pt, **th)
    sh = dict(pt)
    d = 7
    sh["t_lo"] = pt["t_lo"] + d / fs
    sh["t_hi"] = pt["t_hi"] + d / fs
    sh["q_t0_gps"] = np.asarray(pt["q_t0_gps"]) + d / fs
    assert np.allclose(TM.lnL_tmarg(sh, **th), base, rtol=0, atol=1e-9)
    half = dict(sh)
    half["q_t0_gps"] = np.asarray(pt["q_t0_gps"]) + (d + 0.5) / fs
    assert np.max(np.abs(TM.lnL_tmarg(half, **th) - base)) > 1e-3
