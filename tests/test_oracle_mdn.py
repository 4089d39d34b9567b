"""Pins of the learned-proposal oracle (oracle/mdn.py): gradients against central finite
differences, normalisation of the proposal density on its box, agreement of the sampler with
the density, the defensive bound, Adam's first step, bfloat16 rounding, GELU values."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workload as W
from oracle import mc
from oracle import mdn
from oracle import philox as P


def _weights(seed, scale=0.3):
    r = np.random.default_rng(seed)
    return {k: r.normal(0.0, scale / math.sqrt(max(1, s[-1])), s) for k, s in mdn.SHAPES.items()}


def _samples(seed, H, a, b):
    r = np.random.default_rng(seed)
    x = r.uniform(0.02, 0.98, (H, 5))
    return a + (b - a) * x, r.uniform(0.1, 1.0, H)


def test_gelu_and_bf16_reference_values():
    assert mdn.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mdn.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15      # x Phi(x) at 1
    assert abs(mdn.gelu(np.array([-2.0]))[0] - (-2.0 * 0.022750131948179195)) < 1e-15
    v = mdn.bf16_round(np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, -3.140625, 1e-30]))
    assert v[0] == 1.0 and v[1] == 1.0 and v[2] == 1.0 + 2.0 ** -7 and v[3] == -3.140625
    x = np.random.default_rng(0).normal(size=1000).astype(np.float32)
    y = mdn.bf16_round(x)
    assert np.all(np.abs(y - x) <= np.abs(x) * 2.0 ** -8)


def test_head_gradient_matches_finite_differences():
    a, b = mdn.bounds(-0.05, 0.05, 1.0, 1000.0)
    th5, w = _samples(1, 40, a, b)
    head = np.random.default_rng(2).normal(0, 0.5, mdn.N_OUT)
    head[mdn.N_COMP + mdn.N_COMP * mdn.N_DIM:] = np.random.default_rng(3).uniform(-1.5, 0.5, 40)
    _, g = mdn.nll_head_grad(head, th5, w, a, b)
    for i in range(mdn.N_OUT):
        e = np.zeros(mdn.N_OUT)
        e[i] = 1e-6
        fd = (mdn.nll_head_grad(head + e, th5, w, a, b)[0] - mdn.nll_head_grad(head - e, th5, w, a, b)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 * max(1.0, abs(fd)), i


def test_weight_gradient_matches_finite_differences():
    Wt = _weights(4)
    a, b = mdn.bounds(-0.05, 0.05, 1.0, 1000.0)
    S = np.random.default_rng(5).normal(0, 1, (3, mdn.N_IN))
    samples = [_samples(10 + i, 20, a, b) for i in range(3)]
    loss, g = mdn.loss_and_grad(Wt, S, samples, [a] * 3, [b] * 3)
    flat = mdn.flatten(Wt)
    gf = mdn.flatten(g)
    r = np.random.default_rng(6)
    for i in r.choice(flat.size, 40, replace=False):
        e = np.zeros_like(flat)
        e[i] = 1e-6
        lp = mdn.loss_and_grad(mdn.unflatten(flat + e), S, samples, [a] * 3, [b] * 3)[0]
        lm = mdn.loss_and_grad(mdn.unflatten(flat - e), S, samples, [a] * 3, [b] * 3)[0]
        fd = (lp - lm) / 2e-6
        assert abs(fd - gf[i]) <= 2e-5 * max(1.0, abs(fd)), i


def test_proposal_density_is_normalised_on_its_box():
    """E_prior[q_MDN / p5] = 1 for any head."""
    pr = mc.Prior(-0.05, 0.05, 1.0, 1000.0)
    a, b = mdn.bounds(pr.t_lo, pr.t_hi, pr.d_lo, pr.d_hi)
    head = np.random.default_rng(7).normal(0, 0.6, mdn.N_OUT)[None]
    u = P.uniforms(8, 0, 0, np.arange(400000, dtype=np.uint64), 8)
    th = mc.prior_transform(u, pr)
    th5 = np.stack([th["ra"], th["sindec"], th["t"], th["cosi"], np.log(th["dist"])], axis=-1)
    lp = mdn.ln_prior5(th5, pr.d_lo, pr.d_hi, pr.t_lo, pr.t_hi)
    ratio = np.exp(mdn.ln_q_mdn(th5, head, a, b) - lp)
    assert abs(ratio.mean() - 1.0) < 5 * ratio.std() / math.sqrt(ratio.size) + 1e-3


def test_sampler_agrees_with_density_and_defensive_bound():
    """E_q[p5 / q] = 1 over the sampler's own draws (density and sampler agree), and p5/q <= 10."""
    pr = mc.Prior(-0.05, 0.05, 1.0, 1000.0)
    head = np.random.default_rng(9).normal(0, 0.6, mdn.N_OUT)[None]
    u = P.uniforms(10, 0, 0, np.arange(300000, dtype=np.uint64), 10)
    th, lpq = mdn.sample(u, head, pr)
    r = np.exp(lpq)
    assert abs(r.mean() - 1.0) < 5 * r.std() / math.sqrt(r.size) + 1e-3
    assert np.max(lpq) <= math.log(1.0 / mdn.DEFENSIVE) + 1e-12
    assert th["t"].min() > pr.t_lo and th["t"].max() < pr.t_hi


def test_adam_first_step():
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    new, m, v = mdn.adam(th, g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(new, th - 0.01 * g / (np.abs(g) + 1e-8))


def test_summary_features_shape_and_physics():
    pt = W.make_point(W.cfg_small(), 5)
    s = mdn.summary(pt)
    assert s.shape == (64,) and np.all(np.isfinite(s))
    # the (2,2) mean time of each detector lies inside its Q window
    T = pt["Q"].shape[2]
    for k in range(2):
        tau0 = pt["q_t0_gps"][k] - pt["t_ref_gps"]
        assert tau0 <= s[10 * k] <= tau0 + (T - 1) / pt["fs"]
    # a pure time shift of the data by an integer number of samples shifts the mean times
    pt2 = dict(pt)
    pt2["q_t0_gps"] = pt["q_t0_gps"] + 3.0 / pt["fs"]
    s2 = mdn.summary(pt2)
    assert abs((s2[0] - s[0]) - 3.0 / pt["fs"]) < 1e-12
    assert np.allclose(s2[1:5], s[1:5])


def test_summary_closed_form_gaussian_envelope():
    """Every summary feature on Q whose features are known in closed form: in each detector the
    (2, 2) and (2, -2) modes are Gaussian envelopes A exp(-(tau - t0)^2 / (2 s^2)) of constant
    phase theta, sampled far inside the window.  With w = |Q|^8 the weight is a Gaussian of
    variance s^2 / 8, whose sampled moments equal the continuous ones to exponential accuracy
    (Poisson summation, s >> 1/fs): mean time t0, spread s / sqrt(8), log of the mean |Q|^8 over
    8 = ln A + ln(sqrt(2 pi) (s / sqrt(8)) fs / T) / 8, phase of sum w Q = theta; then
    ln sqrt(U_aa) per detector and mode, and the differences of the (2, 2) mean times."""
    fs, T, K = 4096.0, 1201, 3
    t_ref = 1187008882.4
    q_t0 = t_ref + np.array([-0.15, -0.148, -0.1505])
    lm = [(2, -2), (2, 1), (2, 2)]
    params = {  # (k, mode): (A, t0 relative to t_ref, s, theta)
        (0, (2, 2)): (3.0, -0.0031, 12 / fs, 0.7), (0, (2, -2)): (0.5, -0.0027, 9 / fs, -2.1),
        (1, (2, 2)): (2.0, 0.0043, 15 / fs, 2.9), (1, (2, -2)): (7.0, 0.0049, 10 / fs, 0.2),
        (2, (2, 2)): (1.5, 0.0002, 11 / fs, -1.3), (2, (2, -2)): (4.0, -0.0003, 13 / fs, 1.1),
    }
    Q = np.zeros((K, len(lm), T), dtype=np.complex128)
    for k in range(K):
        tau = (q_t0[k] - t_ref) + np.arange(T) / fs
        Q[k, lm.index((2, 1))] = 0.3 * np.exp(1j * 40.0 * tau)      # a mode the summary ignores
        for mode in ((2, 2), (2, -2)):
            A, t0, sg, th = params[(k, mode)]
            Q[k, lm.index(mode)] = A * np.exp(-(tau - t0) ** 2 / (2 * sg * sg)) * np.exp(1j * th)
    U = np.zeros((K, 3, 3), dtype=np.complex128)
    for k in range(K):
        U[k] = np.diag([5.0 + k, 1.0, 20.0 * (k + 1)])
    pt = dict(Q=Q, U=U, lm=np.array(lm, dtype=np.int32), fs=fs, q_t0_gps=q_t0, t_ref_gps=t_ref)
    s = mdn.summary(pt)
    want = []
    for k in range(K):
        for mode in ((2, 2), (2, -2)):
            A, t0, sg, th = params[(k, mode)]
            sw = sg / math.sqrt(8.0)
            want += [t0, sw, math.log(A) + math.log(math.sqrt(2 * math.pi) * sw * fs / T) / 8.0,
                     math.cos(th), math.sin(th)]
    for k in range(K):
        want += [0.5 * math.log(20.0 * (k + 1)), 0.5 * math.log(5.0 + k)]
    t22 = [params[(k, (2, 2))][1] for k in range(K)]
    want += [t22[0] - t22[1], t22[0] - t22[2], t22[1] - t22[2]]
    want += [0.0] * (64 - len(want))
    assert np.allclose(s, np.array(want), rtol=0, atol=1e-12), np.max(np.abs(s - np.array(want)))


def _far_head():
    """A proposal head far from any posterior: every component at the corner of the box with
    narrow widths, so that only the defensive prior component covers the likelihood."""
    head = np.zeros(mdn.N_OUT)
    head[mdn.N_COMP:mdn.N_COMP + 40] = 4.0
    head[mdn.N_COMP + 40:] = -3.0
    return head


def _weak_point():
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.L2_MODES), fs=4096.0, snr=4.0, t_half=0.02,
                       seg_len=4.0)
    return W.make_point(spec, 41)


def test_learned_fallback_switches_on_a_degenerate_round_and_stays_unbiased():
    """The fallback of the learned proposal: with a head far from the posterior the learned rounds'
    own n_eff (sum w / max w over a round) is small; a threshold below every learned round's keeps
    the point learned, one just above round 0's hands it to the adaptive sampler from round 1 on.
    The pooled estimate with the switch agrees with plain prior sampling within the Monte Carlo
    errors (each round enters with its own q)."""
    pt = _weak_point()
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    head = _far_head()
    n = 20000
    learned = mc.marginalize_learned(pt, 3, 0, pr, head, n, 3 * n, 1e300)
    rn = learned["round_neff"]
    assert len(rn) == 3 and learned["fallback_round"] == -1
    assert 1.0 < min(rn) and max(rn) < 0.2 * n
    keep = mc.marginalize_learned(pt, 3, 0, pr, head, n, 3 * n, 1e300, fallback_neff=0.99 * min(rn))
    assert keep["fallback_round"] == -1 and keep["lnL_marg"] == learned["lnL_marg"]
    fb = mc.marginalize_learned(pt, 3, 0, pr, head, n, 8 * n, 1e300, fallback_neff=1.01 * rn[0], n_bins=32)
    assert fb["fallback_round"] == 1 and fb["rounds"] == 8 and fb["acc"].n == 8 * n
    assert fb["round_neff"][0] == rn[0]
    plain = mc.marginalize(pt, 5, 0, pr, 100000, 400000, 1e300)
    s = math.hypot(plain["sigma"], fb["sigma"])
    assert abs(plain["lnL_marg"] - fb["lnL_marg"]) < 5 * s + 0.005, (plain["lnL_marg"], fb["lnL_marg"], s)
