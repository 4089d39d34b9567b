"""GPU: detector-frame coefficients and arrival times of physical sources (rift_source_frame)
against the oracle's injection (Sec. II.A: detector response, time of flight, -2Y_lm), and a
physical injection built from them peaking where the oracle's does."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L

pytestmark = pytest.mark.gpu


def _sources(n, seed):
    r = np.random.default_rng(seed)
    return np.stack([r.uniform(0, 2 * np.pi, n), np.arcsin(r.uniform(-1, 1, n)), r.uniform(-0.05, 0.05, n),
                     r.uniform(0, np.pi, n), r.uniform(0, 2 * np.pi, n), np.arccos(r.uniform(-1, 1, n)),
                     r.uniform(20.0, 1000.0, n)], axis=1)


def test_source_frame_matches_oracle(lib, cuda):
    """The device's F_k, delay_k and -2Y_lm through c_{k,lm} = x conj(F_k) Y_lm and t_k = t + delay_k,
    for 400 random sources, three detectors and all 21 modes in a shuffled order, against the oracle
    at the same (float32-rounded) angles: coefficients within 1e-6 of the largest of the source,
    arrival times within 1e-8 s."""
    dets = ("H1", "L1", "V1")
    tens = np.stack([W.detector(d)[0] for d in dets])
    pos = np.stack([W.detector(d)[1] for d in dets])
    modes = [W.ALL_MODES[i] for i in np.random.default_rng(4).permutation(21)]
    src = _sources(400, 5)
    coef, tk = lib.rift_source_frame(tens, pos, modes, W.T_REF_GPS, 100.0, src)
    assert coef.shape == (400, 3, 21) and tk.shape == (400, 3)
    s32 = src.copy()
    s32[:, [0, 1, 3, 4, 5, 6]] = s32[:, [0, 1, 3, 4, 5, 6]].astype(np.float32)
    for i in range(400):
        ra, dec, t, psi, phi, incl, D = s32[i]
        want, tw = L.injection((tens, pos), modes, ra, dec, t, psi, phi, incl, D, d_ref=100.0,
                               t_ref_gps=W.T_REF_GPS)
        assert np.abs(coef[i] - want).max() <= 1e-6 * np.abs(want).max(), i
        assert np.abs(tk[i] - tw).max() <= 1e-8, i


def test_source_frame_rejects_bad_input(lib, cuda):
    tens = np.stack([W.detector("H1")[0]])
    pos = np.stack([W.detector("H1")[1]])
    src = _sources(3, 6)
    with pytest.raises(lib.RiftError):
        lib.rift_source_frame(tens, pos, [(2, 2), (2, 2)], W.T_REF_GPS, 100.0, src)
    bad = src.copy()
    bad[1, 6] = -1.0
    with pytest.raises(lib.RiftError):
        lib.rift_source_frame(tens, pos, [(2, 2)], W.T_REF_GPS, 100.0, bad)


def test_device_injection_peaks_at_the_source(lib, cuda):
    """A zero-noise point injected with the device's coefficients: its likelihood at the source, by
    the oracle's exact (direct-sum) Q, is rho^2 / 2 (the optimal SNR of the injection), the
    maximum of Eq. (lnL) by Cauchy-Schwarz; and the device's likelihood at the source matches the
    oracle's with the interpolated Q."""
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.L2_MODES), fs=4096.0, snr=12.0, noise=False)
    tens = np.stack([W.detector(d)[0] for d in spec.dets])
    pos = np.stack([W.detector(d)[1] for d in spec.dets])
    src = np.array([[1.3, -0.4, 0.004, 0.9, 2.2, 1.1, 400.0]])
    coef, tk = lib.rift_source_frame(tens, pos, spec.modes, spec.t_ref_gps, spec.d_ref, src)
    pt = W.make_point(spec, 12, injection=(coef[0], tk[0]))
    peak = L.lnL_factorised(pt, *[np.array([v]) for v in src[0]], exact=True)[0]
    assert abs(peak - 0.5 * spec.snr ** 2) < 1e-6 * spec.snr ** 2, peak
    s32 = src[0].astype(np.float32)
    h = lib.rift_ile_create(pt)
    got = lib.rift_ile_lnL_host(h, *[np.array([v], dtype=np.float32) for v in s32])[0]
    lib.rift_ile_destroy(h)
    want = L.lnL_factorised(pt, *[np.array([float(v)]) for v in s32])[0]
    assert abs(got - want) < 1e-3, (got, want)
