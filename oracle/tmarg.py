"""Time-marginalised likelihood, FP64 oracle (test infrastructure: only tests, the smoke check
and the benchmark's CPU leg use this package).

Eq. (lnL:tmarg): for each Monte Carlo draw of the extrinsic parameters other than the event time,
L_margT = int L dt / T over the coincidence window T (Sec. II.C: the event time is integrated
numerically for every draw, the other coordinates by Monte Carlo).

Reading of the quadrature (the paper does not print it): the midpoint rule on the sampling
interval of the Q time series, t_j = t_lo + (j + 1/2) / fs for j = 0 .. J-1 with
J = floor((t_hi - t_lo) fs), so that

    ln L_margT = ln( (1/J) sum_j exp(lnL(theta, t_j)) ),

evaluated with a running maximum (log-sum-exp).  lnL(theta, t) is Eq. (def:lnL:Decomposed)
(`likelihood.lnL_factorised`); the time grid and the per-time likelihoods are all FP64.
"""
from __future__ import annotations

import math

import numpy as np

from .likelihood import lnL_factorised


def time_grid(pt):
    """(t_j) of the quadrature: midpoints of J intervals of 1/fs from t_lo."""
    fs = float(pt["fs"])
    J = max(1, int(math.floor((pt["t_hi"] - pt["t_lo"]) * fs + 1e-9)))
    return pt["t_lo"] + (np.arange(J, dtype=np.float64) + 0.5) / fs


def lnL_tmarg(pt, ra, dec, psi, phi, incl, dist, interp: int = 3, exact: bool = False, chunk: int = 64):
    """ln L_margT for arrays of draws (N,); returns (N,) float64."""
    ra, dec, psi, phi, incl, dist = (np.atleast_1d(np.asarray(a, dtype=np.float64))
                                     for a in (ra, dec, psi, phi, incl, dist))
    tj = time_grid(pt)
    J = tj.size
    n = ra.size
    out = np.empty(n)
    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        m = b - a
        rep = lambda v: np.repeat(v[a:b], J)
        ll = lnL_factorised(pt, rep(ra), rep(dec), np.tile(tj, m), rep(psi), rep(phi), rep(incl), rep(dist),
                            interp=interp, exact=exact).reshape(m, J)
        mx = ll.max(axis=1)
        out[a:b] = mx + np.log(np.exp(ll - mx[:, None]).sum(axis=1)) - math.log(J)
    return out
