"""Monte Carlo marginalisation of the extrinsic likelihood, FP64 oracle.

Eq. (lnLmarg): L_marg = int L(lambda, theta) p(theta) d theta, estimated by
importance sampling with weights w = L p / q; Sec. II.C: relative error ~
1/sqrt(n_eff), stop at a fixed n_eff threshold; Sec. II.A and Sec. III.B: the
sampling prior is adapted from the most recent chunk of samples in the sky
coordinates (and optionally distance).

Readings (the paper refers to Pankow et al. 2015 for the adaptive details):
* prior: ra ~ U[0, 2pi), sin dec ~ U[-1, 1], t ~ U[t_lo, t_hi], psi ~ U[0, pi),
  phi ~ U[0, 2pi), cos incl ~ U[-1, 1], p(D) ~ D^2 on [D_lo, D_hi] (Sec. III.A).
* uniforms: Philox4x32-10 streams (oracle.philox), dims 0..6 in the order above.
* adaptive proposal: independent piecewise-constant densities on n_bins equal
  bins of (ra, sin dec, t), given by float32 CDF tables cdf[0..n_bins]; after a
  round the table of each dimension is rebuilt from that round's samples alone:
  h_b = sum over samples in bin b of exp(beta (l_i - max l)), with l the log
  importance weight, p_b = (1 - eps) h_b / sum h + eps / n_bins, cdf = cumsum p
  rounded to float32 (cdf[n_bins] = 1).
* stratification (optional, same estimator family): the round's n samples are split into
  C = S_ra S_sd S_t cells of the unit cube of the (ra, sin dec, t) uniforms (S powers of two),
  contiguous blocks of samples per cell, cells [0, rem) holding one sample more than the rest
  (n = base C + rem); sample i of cell c = c_ra + S_ra (c_sd + S_sd c_t) uses
  u_d' = (c_d + u_d) / S_d, and its log weight gains ln(n / (C n_c)), which makes the pooled
  mean the stratified estimator sum_c (1/C) mean_c(w).  Rounds with n < C are not stratified.
* estimator: every sample of every round enters with its own round's q:
  lnL_marg = log( sum_i w_i / N_total ); n_eff = sum w / max w; the Kish size
  (sum w)^2 / sum w^2 and the standard error of lnL_marg are also reported.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .tmarg import lnL_tmarg
from .likelihood import lnL_factorised
from .philox import uniforms

N_UNIFORMS = 8
ADAPT_DIMS = 3   # ra, sin dec, t


@dataclass
class Prior:
    t_lo: float
    t_hi: float
    d_lo: float = 1.0
    d_hi: float = 1000.0

    def ranges(self):
        """(lo, hi) of the adapted coordinates ra, sin dec, t."""
        return [(0.0, 2.0 * math.pi), (-1.0, 1.0), (self.t_lo, self.t_hi)]


def prior_transform(u, prior: Prior):
    """Uniforms (>=7, N) -> sample dict (ra, sindec, t, psi, phi, cosi, dist)."""
    return dict(
        ra=2.0 * math.pi * u[0],
        sindec=2.0 * u[1] - 1.0,
        t=prior.t_lo + (prior.t_hi - prior.t_lo) * u[2],
        psi=math.pi * u[3],
        phi=2.0 * math.pi * u[4],
        cosi=2.0 * u[5] - 1.0,
        dist=np.cbrt(prior.d_lo ** 3 + u[6] * (prior.d_hi ** 3 - prior.d_lo ** 3)),
    )


def uniform_tables(n_bins: int):
    """CDF tables of the prior itself (used as the first adaptive round)."""
    c = (np.arange(n_bins + 1, dtype=np.float64) / n_bins).astype(np.float32)
    return np.stack([c] * ADAPT_DIMS)


def inverse_cdf(cdf32, u):
    """Piecewise-constant inverse CDF on [0, 1): returns (x in [0,1), bin, bin probability).

    The bin is the largest b with cdf[b] <= u (comparison of exact float32 values)."""
    cdf = cdf32.astype(np.float64)
    nb = cdf.shape[0] - 1
    b = np.searchsorted(cdf, u, side="right") - 1
    b = np.clip(b, 0, nb - 1)
    pb = cdf[b + 1] - cdf[b]
    x = (b + (u - cdf[b]) / pb) / nb
    return x, b, pb


def effective_strata(n, strata):
    """Strata used for a round of n samples: none if the round has fewer samples than cells."""
    s = tuple(int(x) for x in strata)
    for x in s:
        if x < 1 or (x & (x - 1)):
            raise ValueError("strata must be powers of two")
    return s if n >= s[0] * s[1] * s[2] else (1, 1, 1)


def cell_of(i, n, C):
    """Cell of sample i of a round of n samples over C cells, and that cell's sample count."""
    i = np.asarray(i, dtype=np.int64)
    base, rem = divmod(int(n), int(C))
    big = rem * (base + 1)
    c = np.where(i < big, i // (base + 1), rem + (i - big) // max(base, 1))
    n_c = np.where(c < rem, base + 1, base)
    return c, n_c


def stratify(u, idx, n, strata):
    """Stratified uniforms of the (ra, sin dec, t) dimensions and the log-weight correction."""
    S = effective_strata(n, strata)
    C = S[0] * S[1] * S[2]
    if C == 1:
        return u, np.zeros(u.shape[1])
    c, n_c = cell_of(idx, n, C)
    cc = [c % S[0], (c // S[0]) % S[1], c // (S[0] * S[1])]
    u = u.copy()
    for d in range(3):
        u[d] = (cc[d] + u[d]) / S[d]
    return u, np.log(n / (C * n_c))


def draw(seed, point, rnd, idx, prior: Prior, tables=None, strata=(1, 1, 1), n_round=None):
    """Samples of one round.  Returns (theta dict, bins (3, N) or None, ln p - ln q).

    strata / n_round: stratification of the round (n_round = samples in the round; idx may
    be a subset of range(n_round))."""
    u = uniforms(seed, point, rnd, idx, N_UNIFORMS)
    n_round = len(idx) if n_round is None else n_round
    u, corr = stratify(u, idx, n_round, strata)
    th = prior_transform(u, prior)
    if tables is None:
        return th, None, corr
    nb = tables.shape[1] - 1
    bins = np.empty((ADAPT_DIMS, u.shape[1]), dtype=np.int64)
    lpq = corr.copy()
    for d, (key, (lo, hi)) in enumerate(zip(("ra", "sindec", "t"), prior.ranges())):
        x, b, pb = inverse_cdf(tables[d], u[d])
        th[key] = lo + (hi - lo) * x
        bins[d] = b
        lpq -= np.log(nb * pb)        # ln p_d - ln q_d with p_d = 1/(hi-lo), q_d = pb nb/(hi-lo)
    return th, bins, lpq


def lnL_samples(pt, th, interp=3):
    return lnL_factorised(pt, th["ra"], np.arcsin(th["sindec"]), th["t"], th["psi"], th["phi"],
                          np.arccos(th["cosi"]), th["dist"], interp=interp)


@dataclass
class Accum:
    """Mergeable log-sum-exp state over log weights l: (max, sum e^{l-max}, sum e^{2(l-max)}, n)."""
    m: float = -math.inf
    s1: float = 0.0
    s2: float = 0.0
    n: int = 0

    @staticmethod
    def of(ell):
        ell = np.asarray(ell, dtype=np.float64)
        if ell.size == 0:
            return Accum()
        m = float(np.max(ell))
        e = np.exp(ell - m)
        return Accum(m, math.fsum(e.tolist()), math.fsum((e * e).tolist()), int(ell.size))

    def merge(self, o: "Accum") -> "Accum":
        if o.n == 0:
            return self
        if self.n == 0:
            return o
        m = max(self.m, o.m)
        a, b = math.exp(self.m - m), math.exp(o.m - m)
        return Accum(m, math.fsum([self.s1 * a, o.s1 * b]), math.fsum([self.s2 * a * a, o.s2 * b * b]),
                     self.n + o.n)

    def result(self):
        """(lnL_marg, n_eff = sum w / max w, Kish size, standard error of lnL_marg)."""
        if self.n == 0:
            return (-math.inf, 0.0, 0.0, math.inf)
        lnm = self.m + math.log(self.s1) - math.log(self.n)
        n_eff = self.s1          # max w = e^{max l - m} = 1
        kish = self.s1 * self.s1 / self.s2
        if self.n > 1:
            var = max(self.n * self.s2 / (self.s1 * self.s1) - 1.0, 0.0) / (self.n - 1)
        else:
            var = math.inf
        return lnm, n_eff, kish, math.sqrt(var)


def rebuild_tables(ell, bins, n_bins, beta, floor_eps):
    """New float32 CDF tables from one round's log weights and bins (see module doc)."""
    ell = np.asarray(ell, dtype=np.float64)
    h = np.zeros((ADAPT_DIMS, n_bins))
    wb = np.exp(beta * (ell - ell.max()))
    for d in range(ADAPT_DIMS):
        np.add.at(h[d], bins[d], wb)
    out = np.empty((ADAPT_DIMS, n_bins + 1), dtype=np.float32)
    for d in range(ADAPT_DIMS):
        p = (1.0 - floor_eps) * h[d] / h[d].sum() + floor_eps / n_bins
        c = np.concatenate([[0.0], np.cumsum(p)])
        c = c / c[-1]
        out[d] = c.astype(np.float32)
        out[d, -1] = 1.0
        out[d, 0] = 0.0
    return out, h


def uniform_time_table(n_bins: int):
    """The time table of a time-marginalised adaptive run: the uniform density built the way
    every rebuilt table is (running FP64 sum of the bin masses, normalised, rounded to FP32)."""
    c = 0.0
    out = np.empty(n_bins + 1, dtype=np.float32)
    out[0] = 0.0
    tot = 0.0
    for _ in range(n_bins):
        tot += 1.0 / n_bins
    for b in range(n_bins):
        c += 1.0 / n_bins
        out[b + 1] = np.float32(c / tot)
    out[n_bins] = 1.0
    return out


def marginalize(pt, seed, point, prior: Prior, n_per_round, max_evals, n_eff_target,
                adaptive=False, n_bins=100, beta=0.3, floor_eps=0.1, tables=None, interp=3,
                max_rounds=None, keep=False, adapt_rounds=-1, strata=(1, 1, 1), time_marg=False):
    """Round loop of Eq. (lnLmarg) with the n_eff stopping rule of Sec. II.C.

    adaptive=False: plain prior sampling.  adaptive=True: round 0 uses `tables`
    (default: the prior's own uniform tables); after round r < adapt_rounds (all rounds
    if adapt_rounds < 0) the tables are rebuilt from that round, otherwise kept.  Returns a dict with lnL_marg, n_eff, kish, sigma, n_evals,
    rounds, with the adaptive proposal "tables_next" (the tables a further round would use: a
    warm start for another point), and per-round data if keep."""
    acc = Accum()
    rnd = 0
    hist = []
    if adaptive and tables is None:
        tables = uniform_tables(n_bins)
    while True:
        idx = np.arange(min(n_per_round, max_evals - acc.n), dtype=np.uint64)
        th, bins, lpq = draw(seed, point, rnd, idx, prior, tables if adaptive else None, strata, len(idx))
        if time_marg:
            # Eq. (lnL:tmarg): the draw's t is unused, the event time is integrated by quadrature
            ell = lnL_tmarg(pt, th["ra"], np.arcsin(th["sindec"]), th["psi"], th["phi"], np.arccos(th["cosi"]),
                            th["dist"], interp=interp) + lpq
        else:
            ell = lnL_samples(pt, th, interp) + lpq
        acc = acc.merge(Accum.of(ell))
        lnm, n_eff, kish, sig = acc.result()
        if keep:
            hist.append(dict(ell=ell, bins=bins, tables=None if tables is None else tables.copy()))
        rnd += 1
        if n_eff >= n_eff_target or acc.n >= max_evals or (max_rounds and rnd >= max_rounds):
            break
        if adaptive and (adapt_rounds < 0 or rnd - 1 < adapt_rounds):
            tables, _ = rebuild_tables(ell, bins, n_bins, beta, floor_eps)
            if time_marg:
                tables[2] = uniform_time_table(n_bins)
    lnm, n_eff, kish, sig = acc.result()
    out = dict(lnL_marg=lnm, n_eff=n_eff, kish=kish, sigma=sig, n_evals=acc.n, rounds=rnd, acc=acc)
    if adaptive:
        # the proposal a further round would draw from (Sec. II.C: the integrator carried over to
        # the next intrinsic point): the last round's rebuild when that round adapts
        if adapt_rounds < 0 or rnd - 1 < adapt_rounds:
            nxt, _ = rebuild_tables(ell, bins, n_bins, beta, floor_eps)
            if time_marg:
                nxt[2] = uniform_time_table(n_bins)
            out["tables_next"] = nxt
        else:
            out["tables_next"] = tables.copy()
    if keep:
        out["history"] = hist
    return out


def marginalize_learned(pt, seed, point, prior: Prior, head, n_per_round, max_evals, n_eff_target,
                        fallback_neff=0.0, n_bins=100, beta=0.3, floor_eps=0.1, max_rounds=None,
                        time_marg=False, interp=3):
    """Round loop of Eq. (lnLmarg) with the learned proposal (oracle.mdn.sample, uniforms 0..9 of
    each draw's stream) and its fallback to the adaptive sampler.

    After a learned round whose own draws have n_eff = sum w / max w (that round alone) below
    fallback_neff, the point's remaining rounds draw from the adaptive proposal, unstratified,
    starting from the prior's tables and rebuilt from each adaptive round; every round enters the
    pooled estimate with its own q.  Returns the marginalize() keys plus "fallback_round" (the first
    adaptive round, -1 if none) and "round_neff" (each round's own n_eff)."""
    from .mdn import sample
    acc = Accum()
    rnd, fb_round = 0, -1
    learned = True
    round_neff = []
    tables = uniform_tables(n_bins)
    head = np.atleast_2d(np.asarray(head, dtype=np.float64))
    while True:
        idx = np.arange(min(n_per_round, max_evals - acc.n), dtype=np.uint64)
        if learned:
            th, lpq = sample(uniforms(seed, point, rnd, idx, 10), head, prior, time_marg)
            bins = None
        else:
            th, bins, lpq = draw(seed, point, rnd, idx, prior, tables, (1, 1, 1), len(idx))
        if time_marg:
            ell = lnL_tmarg(pt, th["ra"], np.arcsin(th["sindec"]), th["psi"], th["phi"], np.arccos(th["cosi"]),
                            th["dist"], interp=interp) + lpq
        else:
            ell = lnL_samples(pt, th, interp) + lpq
        this_round = Accum.of(ell)
        round_neff.append(this_round.s1)
        acc = acc.merge(this_round)
        lnm, n_eff, kish, sig = acc.result()
        rnd += 1
        if n_eff >= n_eff_target or acc.n >= max_evals or (max_rounds and rnd >= max_rounds):
            break
        if learned:
            if fallback_neff > 0.0 and this_round.s1 < fallback_neff:   # s1 = the round's sum w / max w
                learned = False
                fb_round = rnd
        else:
            tables, _ = rebuild_tables(ell, bins, n_bins, beta, floor_eps)
            if time_marg:
                tables[2] = uniform_time_table(n_bins)
    lnm, n_eff, kish, sig = acc.result()
    return dict(lnL_marg=lnm, n_eff=n_eff, kish=kish, sigma=sig, n_evals=acc.n, rounds=rnd, acc=acc,
                fallback_round=fb_round, round_neff=round_neff)
