"""Learned proposal: mixture-density network over the located extrinsic coordinates (FP64 oracle).

The paper anticipates moving the Monte Carlo machinery onto the GPU (Sec. V); the learned
proposal is an importance-sampling proposal q(theta | s) for one intrinsic point, conditioned
on a summary s of its Q time series, that keeps the estimator of Eq. (lnLmarg) unbiased.

Readings (none of this is in the paper):
* learned coordinates theta5 = (ra, sin dec, t, cos incl, ln D) on boxes [a, b]; psi, phi from
  the prior.  x = (theta - a)/(b - a), z = logit(x); an 8-component diagonal Gaussian mixture
  in z; ln q(theta) = ln q_z(z) - sum_d [ln(b_d - a_d) + ln x_d + ln(1 - x_d)] (exact change
  of variables, normalised on the box).
* defensive mixture q = 0.9 q_MDN + 0.1 p5 (p5: the prior of theta5), so p/q <= 10 on theta5.
* network: s (64) -> 256 -> 256 (GELU, erf form) -> 88 = 8 logits + 8x5 means + 8x5 log
  sigmas (clamped to [-8, 4]); weights rounded to bfloat16 (round to nearest even), activations
  and accumulation in float32 on the device, float64 here.
* loss: weighted negative log likelihood of harvested posterior samples of each point (box
  fractions clipped to [1e-6, 1 - 1e-6] so samples rounded onto the box edge stay finite),
  -sum_i sum_j wbar_ij ln q_MDN(theta_ij | s_i) / n_points, minimised with Adam
  (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
* sampling from uniforms u[0..9] of the sample's Philox stream: (u0,u1), (u2,u3), (u4,u5) ->
  Box-Muller normals n0..n5 (n0..n4 used), u6 picks the component (first j with
  u6 < cumsum(pi)_j in float32), u7 < 0.9 chooses the network (else the prior transforms of
  u0..u4), u8 -> psi, u9 -> phi.
* summary: for each detector and each of the (2,2), (2,-2) modes present, with w = |Q|^8 over
  the window: weighted mean time and spread (s), log of the mean |Q|^8 / 8, the phase of
  sum w Q as (cos, sin); per detector log sqrt(U_22,22), log sqrt(U_2-2,2-2); pairwise
  differences of the (2,2) mean times; zero padding to 64.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H, N_COMP, N_DIM = 64, 256, 8, 5
N_OUT = N_COMP * (1 + 2 * N_DIM)
DEFENSIVE = 0.1
LS_MIN, LS_MAX = -8.0, 4.0
SHAPES = {"W1": (N_H, N_IN), "b1": (N_H,), "W2": (N_H, N_H), "b2": (N_H,), "W3": (N_OUT, N_H), "b3": (N_OUT,)}
ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")


def bf16_round(x):
    """Round float32 values to bfloat16 (round to nearest, ties to even), returned as float64."""
    a = np.asarray(x, dtype=np.float32).copy()
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def flatten(W):
    return np.concatenate([np.asarray(W[k], dtype=np.float64).ravel() for k in ORDER])


def unflatten(v):
    out, o = {}, 0
    for k in ORDER:
        n = int(np.prod(SHAPES[k]))
        out[k] = np.asarray(v[o:o + n], dtype=np.float64).reshape(SHAPES[k])
        o += n
    return out


N_PARAM = sum(int(np.prod(s)) for s in SHAPES.values())


# ---------------------------------------------------------------- network
def gelu(x):
    return 0.5 * x * (1.0 + _erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + _erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def _erf(x):
    from scipy.special import erf
    return erf(x)


def forward(W, s, keep=False):
    """s: (N, 64) -> head (N, 88); keep=True also returns the pre-activations."""
    s = np.atleast_2d(np.asarray(s, dtype=np.float64))
    a1 = s @ W["W1"].T + W["b1"]
    h1 = gelu(a1)
    a2 = h1 @ W["W2"].T + W["b2"]
    h2 = gelu(a2)
    out = h2 @ W["W3"].T + W["b3"]
    if keep:
        return out, (s, a1, h1, a2, h2)
    return out


def split_head(out):
    """head (N, 88) -> logits (N, 8), mu (N, 8, 5), log sigma (N, 8, 5) (clamped)."""
    out = np.atleast_2d(out)
    alpha = out[:, :N_COMP]
    mu = out[:, N_COMP:N_COMP + N_COMP * N_DIM].reshape(-1, N_COMP, N_DIM)
    ls = np.clip(out[:, N_COMP + N_COMP * N_DIM:].reshape(-1, N_COMP, N_DIM), LS_MIN, LS_MAX)
    return alpha, mu, ls


# ---------------------------------------------------------------- densities
def bounds(t_lo, t_hi, d_lo, d_hi):
    a = np.array([0.0, -1.0, t_lo, -1.0, math.log(d_lo)])
    b = np.array([2.0 * math.pi, 1.0, t_hi, 1.0, math.log(d_hi)])
    return a, b


def ln_prior5(th5, d_lo, d_hi, t_lo, t_hi):
    """ln p of (ra, sin dec, t, cos incl, ln D) under the prior (p(D) ~ D^2)."""
    lnD = th5[..., 4]
    return (-math.log(2 * math.pi) - math.log(2.0) - math.log(t_hi - t_lo) - math.log(2.0)
            + math.log(3.0) + 3.0 * lnD - math.log(d_hi ** 3 - d_lo ** 3))


def ln_qz(z, alpha, mu, ls):
    """Mixture log density in z-space; z (N, 5), per-row parameters."""
    lp = alpha - np.log(np.sum(np.exp(alpha - alpha.max(axis=-1, keepdims=True)), axis=-1, keepdims=True)) \
        - alpha.max(axis=-1, keepdims=True)
    d = (z[:, None, :] - mu) * np.exp(-ls)
    comp = lp + np.sum(-0.5 * d * d - ls - 0.5 * math.log(2 * math.pi), axis=-1)
    m = comp.max(axis=-1, keepdims=True)
    return (m + np.log(np.sum(np.exp(comp - m), axis=-1, keepdims=True)))[:, 0]


def ln_q_mdn(th5, head, a, b, dims=None):
    """ln q_MDN(theta5) including the logit Jacobian; head (N, 88) or (1, 88).  dims: the
    coordinates kept (the mixture is diagonal, so dropping one integrates it out exactly)."""
    dims = list(range(N_DIM)) if dims is None else list(dims)
    x = ((th5 - a) / (b - a))[:, dims]
    z = np.log(x) - np.log1p(-x)
    alpha, mu, ls = split_head(head)
    return ln_qz(z, alpha, mu[..., dims], ls[..., dims]) - np.sum(np.log((b - a)[dims]) + np.log(x) + np.log1p(-x),
                                                                   axis=-1)


def ln_q_defensive(th5, head, a, b, lnp5):
    lq = ln_q_mdn(th5, head, a, b)
    return np.logaddexp(math.log(1.0 - DEFENSIVE) + lq, math.log(DEFENSIVE) + lnp5)


# ---------------------------------------------------------------- sampling
def sample(u, head, prior, time_marg=False):
    """Uniforms (10, N) -> theta dict (ra, sindec, t, psi, phi, cosi, dist), ln p5 - ln q.

    time_marg: the event time is integrated by quadrature (Eq. lnL:tmarg), so the weight is that
    of the other four coordinates: ln p4 - ln q4, q4 = 0.9 q_MDN (t dropped) + 0.1 p4."""
    alpha, mu, ls = split_head(head)
    alpha, mu, ls = alpha[0], mu[0], ls[0]
    n = []
    for i in range(3):
        r = np.sqrt(-2.0 * np.log(u[2 * i]))
        n.append(r * np.cos(2.0 * math.pi * u[2 * i + 1]))
        n.append(r * np.sin(2.0 * math.pi * u[2 * i + 1]))
    n = np.stack(n[:N_DIM], axis=-1)
    # component: first j with u6 < cumsum(pi)_j, the cumulative sum taken in float32
    e = np.exp(alpha - alpha.max())
    pi32 = (e / e.sum()).astype(np.float32)
    cw = np.cumsum(pi32, dtype=np.float32).astype(np.float64)
    j = np.minimum(np.searchsorted(cw, u[6], side="right"), N_COMP - 1)
    z = mu[j] + np.exp(ls[j]) * n
    x = 1.0 / (1.0 + np.exp(-z))
    a, b = bounds(prior.t_lo, prior.t_hi, prior.d_lo, prior.d_hi)
    th5 = a + (b - a) * x
    use_prior = u[7] >= 1.0 - DEFENSIVE
    # prior branch: the usual transforms of u0..u4
    pr = np.stack([2.0 * math.pi * u[0], 2.0 * u[1] - 1.0, prior.t_lo + (prior.t_hi - prior.t_lo) * u[2],
                   2.0 * u[3] - 1.0,
                   np.log(np.cbrt(prior.d_lo ** 3 + u[4] * (prior.d_hi ** 3 - prior.d_lo ** 3)))], axis=-1)
    th5 = np.where(use_prior[:, None], pr, th5)
    lnp5 = ln_prior5(th5, prior.d_lo, prior.d_hi, prior.t_lo, prior.t_hi)
    th = dict(ra=th5[:, 0], sindec=th5[:, 1], t=th5[:, 2], cosi=th5[:, 3], dist=np.exp(th5[:, 4]),
              psi=math.pi * u[8], phi=2.0 * math.pi * u[9])
    if time_marg:
        lnp4 = lnp5 + math.log(prior.t_hi - prior.t_lo)
        lq4 = np.logaddexp(math.log(1.0 - DEFENSIVE) + ln_q_mdn(th5, np.atleast_2d(head), a, b, dims=(0, 1, 3, 4)),
                           math.log(DEFENSIVE) + lnp4)
        return th, lnp4 - lq4
    lq = ln_q_defensive(th5, np.atleast_2d(head), a, b, lnp5)
    return th, lnp5 - lq


# ---------------------------------------------------------------- training
def nll_head_grad(head, th5, w, a, b):
    """Weighted NLL of one point's samples and its gradient w.r.t. the head (88,).

    loss = -sum_j w_j ln q_MDN(theta_j); the Jacobian term does not depend on the head."""
    head = np.asarray(head, dtype=np.float64)
    alpha = head[:N_COMP]
    mu = head[N_COMP:N_COMP + N_COMP * N_DIM].reshape(N_COMP, N_DIM)
    ls_raw = head[N_COMP + N_COMP * N_DIM:].reshape(N_COMP, N_DIM)
    ls = np.clip(ls_raw, LS_MIN, LS_MAX)
    # samples on the edge of the box (float rounding) are kept just inside it
    x = np.clip((th5 - a) / (b - a), 1e-6, 1.0 - 1e-6)
    z = np.log(x) - np.log1p(-x)
    lpi = alpha - alpha.max()
    lpi = lpi - np.log(np.sum(np.exp(lpi)))
    d = (z[:, None, :] - mu[None]) * np.exp(-ls)[None]
    comp = lpi[None] + np.sum(-0.5 * d * d - ls[None] - 0.5 * math.log(2 * math.pi), axis=-1)   # (H, 8)
    m = comp.max(axis=1, keepdims=True)
    lq = m[:, 0] + np.log(np.sum(np.exp(comp - m), axis=1))
    jac = np.sum(np.log(b - a) + np.log(x) + np.log1p(-x), axis=-1)
    loss = -np.sum(w * (lq - jac))
    r = np.exp(comp - lq[:, None])               # responsibilities (H, 8)
    wr = w[:, None] * r
    pi = np.exp(lpi)
    g_alpha = -(np.sum(wr, axis=0) - np.sum(w) * pi)
    g_mu = -np.sum(wr[:, :, None] * d * np.exp(-ls)[None], axis=0)
    g_ls = -np.sum(wr[:, :, None] * (d * d - 1.0), axis=0)
    g_ls = np.where((ls_raw > LS_MIN) & (ls_raw < LS_MAX), g_ls, 0.0)
    return loss, np.concatenate([g_alpha, g_mu.ravel(), g_ls.ravel()])


def backward(W, cache, g_out):
    """Gradients of sum(g_out * head) w.r.t. the weights; cache from forward(keep=True)."""
    s, a1, h1, a2, h2 = cache
    g = {"W3": g_out.T @ h2, "b3": g_out.sum(axis=0)}
    gh2 = g_out @ W["W3"]
    ga2 = gh2 * gelu_grad(a2)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(axis=0)
    gh1 = ga2 @ W["W2"]
    ga1 = gh1 * gelu_grad(a1)
    g["W1"] = ga1.T @ s
    g["b1"] = ga1.sum(axis=0)
    return g


def loss_and_grad(W, S, samples, a_list, b_list):
    """Mean over points of the weighted NLL and its weight gradient.

    S: (P, 64); samples: list of (theta5 (H, 5), w (H,)) per point; a/b: per-point boxes."""
    out, cache = forward(W, S, keep=True)
    P = S.shape[0]
    g_out = np.zeros_like(out)
    tot = 0.0
    for i, (th5, w) in enumerate(samples):
        l, g = nll_head_grad(out[i], th5, w, a_list[i], b_list[i])
        tot += l
        g_out[i] = g
    g = backward(W, cache, g_out / P)
    return tot / P, g


def adam(theta, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) of flat parameter vectors; returns theta, m, v."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


# ---------------------------------------------------------------- summary of a point
SUMMARY_MODES = ((2, 2), (2, -2))
SUMMARY_POWER = 8


def summary(pt):
    """64 features of one point from its Q time series and U (see module doc)."""
    Q = np.asarray(pt["Q"])
    U = np.asarray(pt["U"])
    lm = [tuple(x) for x in np.asarray(pt["lm"]).tolist()]
    K, M, T = Q.shape
    fs = float(pt["fs"])
    feats = []
    tmean22 = []
    for k in range(K):
        tau = (pt["q_t0_gps"][k] - pt["t_ref_gps"]) + np.arange(T) / fs
        for mode in SUMMARY_MODES:
            if mode in lm:
                q = Q[k, lm.index(mode)]
                a2 = (q.real ** 2 + q.imag ** 2)
                w = (a2 / a2.max()) ** (SUMMARY_POWER // 2)
                sw = w.sum()
                tm = float(np.sum(w * tau) / sw)
                sd = float(math.sqrt(max(np.sum(w * (tau - tm) ** 2) / sw, 0.0)))
                lmean = float(math.log(a2.max()) * (SUMMARY_POWER // 2) + math.log(sw / T)) / SUMMARY_POWER
                c = np.sum(w * q)
                ph = math.atan2(c.imag, c.real)
                feats += [tm, sd, lmean, math.cos(ph), math.sin(ph)]
                if mode == (2, 2):
                    tmean22.append(tm)
            else:
                feats += [0.0] * 5
                if mode == (2, 2):
                    tmean22.append(0.0)
    for k in range(K):
        for mode in SUMMARY_MODES:
            feats.append(0.5 * math.log(U[k, lm.index(mode), lm.index(mode)].real) if mode in lm else 0.0)
    for i in range(K):
        for j in range(i + 1, K):
            feats.append(tmean22[i] - tmean22[j])
    feats = feats[:N_IN]
    return np.array(feats + [0.0] * (N_IN - len(feats)))
