"""Pins of the Q/U/V oracle (Eq. QUV) against an FFT evaluation, the brute-force likelihood and the
algebraic properties of U and V."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L
from oracle import quv as QUV


@pytest.fixture(scope="module")
def small():
    return W.make_point(W.cfg_small(), 6)


def test_direct_sum_q_equals_the_fft_evaluation(small):
    """The generator forms Q with an inverse FFT over the whole grid; the oracle sums the band
    directly at each grid time: two algorithms, one definition."""
    Q, _, _ = QUV.quv(small)
    scale = np.abs(small["Q"]).max()
    assert np.abs(Q - small["Q"]).max() < 1e-10 * scale


def test_u_hermitian_psd_and_v_symmetric(small):
    _, U, V = QUV.quv(small)
    for k in range(U.shape[0]):
        assert np.allclose(U[k], U[k].conj().T, rtol=0, atol=1e-12 * np.abs(U[k]).max())
        assert np.linalg.eigvalsh(0.5 * (U[k] + U[k].conj().T)).min() > -1e-10 * np.abs(U[k]).max()
        assert np.allclose(V[k], V[k].T, rtol=0, atol=1e-12 * np.abs(V[k]).max())


def test_factorised_with_oracle_quv_equals_bruteforce_on_the_grid():
    """One detector at the geocentre and sample times on the Q grid (no interpolation error): the
    factorised likelihood built from the oracle's Q, U, V equals the brute-force frequency-domain
    likelihood, which checks Q, the U term and the mirror convention of V together."""
    spec = W.PointSpec(dets=("H1",), modes=list(W.L2_MODES) + [(3, 3), (3, -3)], fs=4096.0, snr=12.0,
                       t_half=0.02, seg_len=2.0)
    pt = W.make_point(spec, 9)
    pt["det_pos"] = np.zeros_like(pt["det_pos"])
    Q, U, V = QUV.quv(pt)
    fac = dict(pt, Q=Q, U=U, V=V)
    fs = float(pt["fs"])
    tau0 = pt["q_t0_gps"][0] - pt["t_ref_gps"]
    r = np.random.default_rng(2)
    for _ in range(5):
        j = int(r.integers(10, pt["n_t"] - 10))
        th = dict(ra=r.uniform(0, 6.28), dec=r.uniform(-1.2, 1.2), t=tau0 + j / fs, psi=r.uniform(0, 3.1),
                  phi=r.uniform(0, 6.28), incl=r.uniform(0.1, 3.0), dist=r.uniform(50, 500))
        bf = L.lnL_bruteforce(pt, **th)
        f = L.lnL_factorised(fac, **{k: np.array([v]) for k, v in th.items()})[0]
        assert abs(f - bf) < 1e-9 * max(1.0, abs(bf)), (f, bf)
