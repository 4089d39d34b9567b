"""GPU: the canonical-mode quadratic forms (over the 21 l <= 4 modes, absent ones with zero
coefficients; used from 13 modes on) -- the grouped form, with or without the pairs that vanish
when each mode lives on one sign of frequency, and the positive form of mirror-symmetric points --
with coefficients from kernel parameters (single-point runs) or shared memory (batched runs)."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import mc

from test_parity_gpu import _tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p_full():
    return W.make_point(W.cfg_full(), 2)


def _ms(pt):
    return np.array([m for _, m in np.asarray(pt["lm"]).tolist()])


def _fill_vanishing(pt, value):
    """The point with the pairs that vanish for one-sign modes (U between opposite-sign m, V
    between same-sign m) set to `value` (Hermitian / symmetric)."""
    ms = _ms(pt)
    opp = np.outer(ms, ms) < 0
    same = np.outer(ms, ms) > 0
    U, V = pt["U"].copy(), pt["V"].copy()
    assert np.all(U[:, opp] == 0) and np.all(V[:, same] == 0), "workload is not one-sign"
    U[:, opp] = value
    V[:, same] = value
    return dict(pt, U=U, V=V)


def _two_sided(pt, eps):
    """Every mode given content on the other sign of frequency too, h'_a(f) = h_a(f) + eps
    conj(h_a(-f)) (as for precessing sources), with U and V recomputed from these modes by
    Eq. (QUV): a Gram matrix and its mirror companion, so no pair vanishes and U stays positive."""
    h = pt["hlm"] + eps * np.conj(pt["hlm"][:, np.asarray(pt["mirror"])])
    two = dict(pt, hlm=h)
    K = pt["data"].shape[0]
    w, df, mirror = pt["weight"], pt["df"], np.asarray(pt["mirror"])
    U = np.stack([2.0 * df * (np.conj(h) * w[k]) @ h.T for k in range(K)])
    V = np.stack([2.0 * df * (h[:, mirror] * w[k]) @ h.T for k in range(K)])
    U = 0.5 * (U + np.conj(np.transpose(U, (0, 2, 1))))
    V = 0.5 * (V + np.transpose(V, (0, 2, 1)))
    return dict(two, U=U, V=V)


def _break_mirror(pt):
    """The point with one U entry of the (4, 4) mode changed by 1e-6 of itself in one detector but
    not in its mirror (4, -4): still one-sign (the sparse pattern is kept), no longer
    mirror-symmetric, so the host uses the grouped form instead of the positive mirror form."""
    U = pt["U"].copy()
    a = [tuple(x) for x in np.asarray(pt["lm"]).tolist()].index((4, 4))
    U[0, a, a] *= 1.0 + 1e-6
    return dict(pt, U=U)


def _single(lib, pt, n, seed):
    import torch
    h = lib.rift_ile_create(pt)
    dbg = torch.empty(n, dtype=torch.float32, device="cuda")
    res = lib.rift_ile_marginalize(h, seed=seed, n_per_round=n, max_evals=n, dbg_ell=dbg, strata=(8, 4, 8))
    lib.rift_ile_destroy(h)
    return dbg.cpu().numpy(), res


def _batched(lib, pt, n, seed):
    h = lib.rift_ile_batch_create([pt])
    rows, _, res = lib.rift_ile_samples(h, n, seed=seed, n_per_round=n, max_evals=n, strata=(8, 4, 8))
    lib.rift_ile_destroy(h)
    r = rows[0].cpu().numpy()
    return r[:, 7] + r[:, 8], res


def test_skipping_vanishing_pairs_changes_no_bit(lib, cuda, p_full):
    """A coefficient of 1e-30 where the one-sign workload has exact zeros makes the host keep every
    pair; its products are far below an ulp of the sums, so both forms must agree bit for bit."""
    sparse = _break_mirror(p_full)
    dense = _fill_vanishing(sparse, 1e-30)
    n = 400_000
    a, ra = _single(lib, sparse, n, 91)
    b, rb = _single(lib, dense, n, 91)
    assert np.array_equal(a, b)
    assert ra["lnL_marg"] == rb["lnL_marg"]
    a, _ = _batched(lib, sparse, n, 92)
    b, _ = _batched(lib, dense, n, 92)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("path", ["single", "batched"])
def test_dense_grouped_form_matches_oracle(lib, cuda, p_full, path):
    """Modes on both signs of frequency (every pair present): per sample against the oracle on
    random and highest-weight draws."""
    pt = _two_sided(p_full, 0.1)
    ms = _ms(pt)
    assert np.abs(pt["U"][:, np.outer(ms, ms) < 0]).max() > 1e-3 * np.abs(pt["U"]).max()
    n = 1_000_000
    got, res = (_single if path == "single" else _batched)(lib, pt, n, 93)
    got = got.astype(np.float64)
    r = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.argsort(got)[-200:], r.integers(0, n, 2000)])).astype(np.uint64)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    S = tuple(res["strata"] if path == "single" else res[0]["strata"])
    th, _, lq = mc.draw(93, 0, 0, idx, pr, None, S, n)
    want = mc.lnL_samples(pt, th) + lq
    th64 = dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=th["t"], psi=th["psi"], phi=th["phi"],
                incl=np.arccos(th["cosi"]), dist=th["dist"])
    err = np.abs(got[idx.astype(np.int64)] - want)
    assert np.all(err <= _tol(pt, th64)), err.max()


@pytest.mark.parametrize("path", ["single", "batched"])
def test_partial_mode_set_matches_oracle(lib, cuda, path):
    """15 of the 21 modes in a shuffled caller order (the layout zero-fills the six absent ones)."""
    r = np.random.default_rng(8)
    modes = [(l, m) for l in (2, 3, 4) for m in range(-l, l + 1)]
    keep = [modes[i] for i in r.permutation(21)[:15]]
    if (2, 2) not in keep:
        keep[0] = (2, 2)
    if (2, -2) not in keep:
        keep[1] = (2, -2)
    spec = W.cfg_full()
    spec.modes = keep
    pt = W.make_point(spec, 11)
    assert len(np.asarray(pt["lm"])) == 15
    n = 400_000
    got, res = (_single if path == "single" else _batched)(lib, pt, n, 94)
    got = got.astype(np.float64)
    idx = np.unique(np.concatenate([np.argsort(got)[-200:], r.integers(0, n, 2000)])).astype(np.uint64)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    S = tuple(res["strata"] if path == "single" else res[0]["strata"])
    th, _, lq = mc.draw(94, 0, 0, idx, pr, None, S, n)
    want = mc.lnL_samples(pt, th) + lq
    th64 = dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=th["t"], psi=th["psi"], phi=th["phi"],
                incl=np.arccos(th["cosi"]), dist=th["dist"])
    err = np.abs(got[idx.astype(np.int64)] - want)
    assert np.all(err <= _tol(pt, th64)), err.max()


@pytest.mark.parametrize("path", ["single", "batched"])
def test_mirror_form_matches_oracle_on_edge_on_draws(lib, cuda, p_full, path):
    """The full-size point is mirror-symmetric (non-precessing modes), so its quadratic form is the
    positive form 2 beta^H U beta.  Per sample against the oracle where the general form cancels
    most: nearly edge-on draws (|cos incl| < 0.15) of a 2e6-draw round, the 2000 loudest of them
    and 18000 at random, all within the per-sample tolerance."""
    n = 2_000_000
    pr = mc.Prior(p_full["t_lo"], p_full["t_hi"])
    got, res = (_single if path == "single" else _batched)(lib, p_full, n, 95)
    got = got.astype(np.float64)
    S = tuple(res["strata"] if path == "single" else res[0]["strata"])
    th_all, _, _ = mc.draw(95, 0, 0, np.arange(n, dtype=np.uint64), pr, None, S, n)
    edge = np.where(np.abs(th_all["cosi"]) < 0.15)[0]
    r = np.random.default_rng(3)
    idx = np.unique(np.concatenate([edge[np.argsort(got[edge])[-2000:]], r.choice(edge, 18000, replace=False)]))
    idx = idx.astype(np.uint64)
    th, _, lq = mc.draw(95, 0, 0, idx, pr, None, S, n)
    want = mc.lnL_samples(p_full, th) + lq
    th64 = dict(ra=th["ra"], dec=np.arcsin(th["sindec"]), t=th["t"], psi=th["psi"], phi=th["phi"],
                incl=np.arccos(th["cosi"]), dist=th["dist"])
    q = np.abs(got[idx.astype(np.int64)] - want) / _tol(p_full, th64)
    assert q.max() <= 1.0, q.max()
