"""GPU: the grouped quadratic form (over the 21 canonical l <= 4 modes, absent ones with zero
coefficients; used from 13 modes on), in its forms: coefficients from kernel parameters
(single-point runs) or shared memory (batched runs), with or without the pairs that vanish when
each mode lives on one sign of frequency."""
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
    dense = _fill_vanishing(p_full, 1e-30)
    n = 400_000
    a, ra = _single(lib, p_full, n, 91)
    b, rb = _single(lib, dense, n, 91)
    assert np.array_equal(a, b)
    assert ra["lnL_marg"] == rb["lnL_marg"]
    a, _ = _batched(lib, p_full, n, 92)
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
