"""Extrinsic posterior samples from the Monte Carlo draws, FP64 oracle (test infrastructure: only
tests, the smoke check and the benchmark's CPU leg use this package).

The importance-sampled integral of Eq. (lnLmarg) draws theta_i ~ q and weighs each draw by
w_i = L_i p_i / q_i; normalised, the weighted draws are samples of the extrinsic posterior
p(theta | d, lambda), proportional to L p, at the intrinsic point (Sec. VI: the same integration
yields the extrinsic distributions).

Readings (the paper gives no procedure):
* the weighted export is the last round of a run, every draw with its lnL and ln p - ln q
  (stratification factor included), so that w_i = exp(lnL_i + ln p_i - ln q_i);
* equal-weight samples by systematic resampling: with w_i = exp(l_i - max l), l the log weight,
  cumulative sums C_i = w_0 + ... + w_i and H slots, slot h takes the first i with
  C_i > (h + 1/2) C_{N-1} / H;
* a time-marginalised draw (Eq. lnL:tmarg) carries no event time, so each resampled draw gets one
  from its conditional on the quadrature grid, P(t_j | rest) = exp lnL(t_j) / sum_k exp lnL(t_k),
  by inversion: the first j whose cumulative probability exceeds u, with u the uniform of Philox
  block 3 of counter (slot h, round 0, point) (blocks 0-2 are the sampler's).
"""
from __future__ import annotations

import math

import numpy as np

from . import mc
from .likelihood import lnL_factorised
from .philox import uniforms
from .tmarg import time_grid

POSTERIOR_BLOCK = 3


def last_round(pt, seed, point, prior: mc.Prior, n_per_round, max_evals, n_eff_target, strata=(1, 1, 1),
               time_marg=False, interp=3, **kw):
    """Run Eq. (lnLmarg) and return the draws of its last round: dict with the columns ra, dec, t
    (NaN when time_marg), psi, phi, incl, dist, lnL, lnpq, the log weight ell = lnL + lnpq, and the
    run's result under "result"."""
    res = mc.marginalize(pt, seed, point, prior, n_per_round, max_evals, n_eff_target, strata=strata,
                         time_marg=time_marg, interp=interp, keep=True, **kw)
    last = res["history"][-1]
    rnd = res["rounds"] - 1
    n = last["ell"].size
    idx = np.arange(n, dtype=np.uint64)
    tables = last["tables"] if kw.get("adaptive") else None
    th, _, lpq = mc.draw(seed, point, rnd, idx, prior, tables, strata, n)
    ell = np.asarray(last["ell"], dtype=np.float64)
    return dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=np.full(n, np.nan) if time_marg else th["t"],
                psi=th["psi"], phi=th["phi"], incl=np.arccos(th["cosi"]), dist=th["dist"], lnL=ell - lpq,
                lnpq=lpq, ell=ell, result=res)


def systematic_resample(ell, H):
    """Slot h -> the first i with C_i > (h + 1/2) C_{N-1} / H, C the cumulative sums of
    exp(ell - max ell) (non-finite log weights weigh nothing)."""
    ell = np.asarray(ell, dtype=np.float64)
    w = np.where(np.isfinite(ell), np.exp(ell - np.max(ell[np.isfinite(ell)])), 0.0)
    C = np.cumsum(w)
    target = (np.arange(H) + 0.5) * C[-1] / H
    return np.searchsorted(C, target, side="right"), C


def time_draw(pt, ra, dec, psi, phi, incl, dist, u, interp=3):
    """Event time of one draw from its conditional on the quadrature grid of Eq. (lnL:tmarg).
    Returns (j, t_j, lnL(t_j), cumulative probabilities over the grid)."""
    tj = time_grid(pt)
    J = tj.size
    rep = lambda v: np.full(J, float(v))
    ll = lnL_factorised(pt, rep(ra), rep(dec), tj, rep(psi), rep(phi), rep(incl), rep(dist), interp=interp)
    p = np.exp(ll - ll.max())
    cdf = np.cumsum(p) / p.sum()
    j = int(np.searchsorted(cdf, u, side="right"))
    j = min(j, J - 1)
    return j, tj[j], ll[j], cdf


def posterior_uniforms(seed, point, H):
    """The uniform of each slot's time draw."""
    return uniforms(seed, point, 0, np.arange(H, dtype=np.uint64), 4 * POSTERIOR_BLOCK + 1)[4 * POSTERIOR_BLOCK]


def posterior(pt, seed, point, prior: mc.Prior, n_per_round, max_evals, n_eff_target, H, strata=(1, 1, 1),
              time_marg=False, interp=3, **kw):
    """H equal-weight extrinsic posterior samples: dict of the columns ra, dec, t, psi, phi, incl,
    dist, lnL, the resampled row of the last round ("idx") and the weighted draws ("draws")."""
    S = last_round(pt, seed, point, prior, n_per_round, max_evals, n_eff_target, strata=strata,
                   time_marg=time_marg, interp=interp, **kw)
    idx, _ = systematic_resample(S["ell"], H)
    out = {k: S[k][idx].copy() for k in ("ra", "dec", "t", "psi", "phi", "incl", "dist", "lnL")}
    if time_marg:
        u = posterior_uniforms(seed, point, H)
        for h in range(H):
            _, t, l, _ = time_draw(pt, out["ra"][h], out["dec"][h], out["psi"][h], out["phi"][h], out["incl"][h],
                                   out["dist"][h], u[h], interp)
            out["t"][h] = t
            out["lnL"][h] = l
    out["idx"] = idx
    out["draws"] = S
    return out


def weighted_mean_log(lnL, lnpq):
    """ln of the mean importance weight of a set of draws, in FP64 with the maximum factored out."""
    l = np.asarray(lnL, dtype=np.float64) + np.asarray(lnpq, dtype=np.float64)
    m = float(np.max(l))
    return m + math.log(np.mean(np.exp(l - m)))
