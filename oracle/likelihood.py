"""Extrinsic log-likelihood, FP64 oracle.

Two independent evaluations of the same quantity:

* lnL_bruteforce -- the definition, Eq. (lnL) with Eq. (overlap):
  lnL = sum_k <h_k|d_k> - 1/2 <h_k|h_k>, <a|b> = 2 int df conj(a) b / S_k over the band.
  Eq. (lnL) prints "- <d|d>"; the likelihood ratio against pure noise, which
  Eq. (def:lnL:Decomposed) expands, has "+ 1/2 <d|d> - 1/2 <d|d>", i.e. no data term.
* lnL_factorised -- Eq. (def:lnL:Decomposed) in terms of Q, U, V of Eq. (QUV).

Reading of Eq. (def:lnL:Decomposed) (fixed by the brute-force identity): with
F = F_+ - i F_x and h = h_+ - i h_x the detector output is h_k = Re(conj(F_k) h),
which gives

  lnL = x Re sum_k sum_lm F_k conj(Y_lm) Q_{k,lm}(t_k)
        - x^2/4 sum_k [ |F_k|^2 sum conj(Y_lm) Y_l'm' U_{k,lm,l'm'}
                        + Re( conj(F_k)^2 sum Y_lm Y_l'm' V_{k,lm,l'm'} ) ],   x = D_ref / D.

The printed form, (F_k Y)^* Q and F_k^2 V, is the same function with F_k replaced by
its conjugate (psi -> -psi).

Q_{k,lm}(t) between grid samples: cubic Lagrange interpolation on the uniform grid
(Sec. II.A: Q is kept as a uniformly sampled, truncated time series).  Taps
i-1..i+2 with i = floor(s), s = (t - tau0_k) fs, mu = s - i.
"""
from __future__ import annotations

import numpy as np

from .geometry import complex_antenna, delay, gmst_from_gps
from .swsh import ylm_m2


def lagrange_weights(mu, interp: int):
    """Tap offsets and weights for fractional position mu in [0, 1)."""
    mu = np.asarray(mu, dtype=np.float64)
    if interp == 3:
        w = np.stack([-mu * (mu - 1.0) * (mu - 2.0) / 6.0,
                      (mu + 1.0) * (mu - 1.0) * (mu - 2.0) / 2.0,
                      -(mu + 1.0) * mu * (mu - 2.0) / 2.0,
                      (mu + 1.0) * mu * (mu - 1.0) / 6.0], axis=-1)
        return np.array([-1, 0, 1, 2]), w
    if interp == 1:
        return np.array([0, 1]), np.stack([1.0 - mu, mu], axis=-1)
    if interp == 0:
        return np.array([0]), np.ones(mu.shape + (1,))
    raise ValueError("interp must be 0, 1 or 3")


def q_interp(Qk, s, interp: int = 3):
    """Qk: (M, T) complex grid of one detector; s: (N,) fractional sample index.
    Returns (N, M).  Raises if a tap falls outside the grid."""
    s = np.asarray(s, dtype=np.float64)
    if interp == 0:
        i = np.floor(s + 0.5).astype(np.int64)
        mu = np.zeros_like(s)
    else:
        i = np.floor(s).astype(np.int64)
        mu = s - i
    offs, w = lagrange_weights(mu, interp)
    taps = i[:, None] + offs[None, :]
    if taps.min() < 0 or taps.max() >= Qk.shape[1]:
        raise ValueError("Q window does not cover the requested times")
    g = Qk[:, taps]                      # (M, N, P)
    return np.einsum("mnp,np->nm", g, w)


def q_exact(pt, k, t):
    """Q_{k,lm}(t) of Eq. (QUV) by a direct frequency sum at arbitrary t (relative to t_ref)."""
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    f = pt["freqs"]
    X = np.conj(pt["hlm"]) * pt["data"][k][None, :] * pt["weight"][k][None, :]   # (M, Nf)
    ph = np.exp(2j * np.pi * np.outer(t, f))                                       # (N, Nf)
    return 2.0 * pt["df"] * ph @ X.T                                              # (N, M)


def _geometry(pt):
    return gmst_from_gps(pt["t_ref_gps"]), np.asarray(pt["det_tensor"]), np.asarray(pt["det_pos"])


def lnL_factorised(pt, ra, dec, t, psi, phi, incl, dist, interp: int = 3, exact: bool = False,
                   chunk: int = 8192):
    """Eq. (def:lnL:Decomposed) for sample arrays; returns (N,) float64."""
    ra, dec, t, psi, phi, incl, dist = (np.atleast_1d(np.asarray(a, dtype=np.float64))
                                        for a in (ra, dec, t, psi, phi, incl, dist))
    n = ra.shape[0]
    out = np.empty(n)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        out[a:b] = _lnL_block(pt, ra[a:b], dec[a:b], t[a:b], psi[a:b], phi[a:b], incl[a:b],
                              dist[a:b], interp, exact)
    return out


def _lnL_block(pt, ra, dec, t, psi, phi, incl, dist, interp, exact):
    gmst, tens, pos = _geometry(pt)
    modes = [tuple(x) for x in np.asarray(pt["lm"]).tolist()]
    Q, U, V = pt["Q"], pt["U"], pt["V"]
    fs = float(pt["fs"])
    x = pt["d_ref_mpc"] / dist
    Y = ylm_m2(modes, incl, phi)                          # (N, M)
    lin = np.zeros_like(ra)
    quad = np.zeros_like(ra)
    for k in range(tens.shape[0]):
        F = complex_antenna(tens[k], ra, dec, psi, gmst)  # (N,)
        tk = t + delay(pos[k], ra, dec, gmst)
        if exact:
            Qk = q_exact(pt, k, tk)
        else:
            tau0 = pt["q_t0_gps"][k] - pt["t_ref_gps"]
            Qk = q_interp(Q[k], (tk - tau0) * fs, interp)
        lin += np.real(F * np.sum(np.conj(Y) * Qk, axis=-1))
        A = np.real(np.einsum("na,ab,nb->n", np.conj(Y), U[k], Y))
        B = np.einsum("na,ab,nb->n", Y, V[k], Y)
        quad += np.abs(F) ** 2 * A + np.real(np.conj(F) ** 2 * B)
    return x * lin - 0.25 * x * x * quad


def detector_strain(pt, ra, dec, t, psi, phi, incl, dist):
    """h_k(f) of one sample: Re(conj(F_k) h) shifted to t_k, with h = x sum Y_lm h_lm."""
    gmst, tens, pos = _geometry(pt)
    modes = [tuple(v) for v in np.asarray(pt["lm"]).tolist()]
    Y = ylm_m2(modes, incl, phi)[0]
    x = pt["d_ref_mpc"] / dist
    f, hlm, mirror = pt["freqs"], pt["hlm"], pt["mirror"]
    H = x * (Y @ hlm)                        # h(f)
    Hbar = np.conj(H[mirror])                # transform of conj(h(t))
    out = []
    for k in range(tens.shape[0]):
        F = complex_antenna(tens[k], ra, dec, psi, gmst)
        tk = t + delay(pos[k], ra, dec, gmst)
        out.append(0.5 * (np.conj(F) * H + F * Hbar) * np.exp(-2j * np.pi * f * tk))
    return np.array(out)


def inner(a, b, weight, df):
    """Eq. (overlap): 2 df sum_f conj(a) b / S over the band (weight = band / S)."""
    return 2.0 * df * np.sum(np.conj(a) * b * weight)


def lnL_bruteforce(pt, ra, dec, t, psi, phi, incl, dist):
    """Eq. (lnL) for one sample: sum_k <h_k|d_k> - 1/2 <h_k|h_k>."""
    hk = detector_strain(pt, ra, dec, t, psi, phi, incl, dist)
    tot = 0.0
    for k in range(hk.shape[0]):
        w = pt["weight"][k]
        tot += np.real(inner(hk[k], pt["data"][k], w, pt["df"])) - 0.5 * np.real(inner(hk[k], hk[k], w, pt["df"]))
    return float(tot)


def injection(pt_geometry, modes, ra, dec, t, psi, phi, incl, dist, d_ref, t_ref_gps):
    """Detector-frame coefficients of a physical source: c_{k,lm} = x conj(F_k) Y_lm and
    arrival offsets t_k = t + delay_k, so that d_k = Re sum c_{k,lm} h_lm(t - t_k)."""
    tens, pos = pt_geometry
    gmst = gmst_from_gps(t_ref_gps)
    Y = ylm_m2(modes, incl, phi)[0]
    x = d_ref / dist
    K = tens.shape[0]
    coef = np.empty((K, len(modes)), dtype=np.complex128)
    tk = np.empty(K)
    for k in range(K):
        F = complex_antenna(tens[k], ra, dec, psi, gmst)
        coef[k] = x * np.conj(F) * Y
        tk[k] = t + delay(pos[k], ra, dec, gmst)
    return coef, tk
