"""GPU parity of the time-marginalised likelihood, Eq. (lnL:tmarg), against the FP64 oracle.

Per draw the tolerance is that of the per-sample likelihood, 1e-3 * max(1, <h|h>/900): the
log-sum-exp over the time grid is dominated by its largest terms, whose errors it inherits."""
from __future__ import annotations

import math

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L
from oracle import tmarg as TM

pytestmark = pytest.mark.gpu


def _draws(n, seed):
    r = np.random.default_rng(seed)
    th = dict(ra=r.uniform(0, 2 * np.pi, n), dec=np.arcsin(r.uniform(-1, 1, n)), psi=r.uniform(0, np.pi, n),
              phi=r.uniform(0, 2 * np.pi, n), incl=np.arccos(r.uniform(-1, 1, n)),
              dist=np.cbrt(r.uniform(1, 1000.0 ** 3, n)))
    return {k: v.astype(np.float32) for k, v in th.items()}


def _tol(pt, th64):
    z = dict(pt)
    z["Q"] = np.zeros_like(pt["Q"])
    hh = -2.0 * L.lnL_factorised(z, t=np.zeros_like(th64["ra"]), **th64)
    return 1e-3 * np.maximum(1.0, hh / 900.0)


def _gpu(lib, h, th):
    import torch
    d = {k: torch.as_tensor(v, device="cuda") for k, v in th.items()}
    out = lib.rift_ile_lnL_tmarg(h, d["ra"], d["dec"], d["psi"], d["phi"], d["incl"], d["dist"])
    torch.cuda.synchronize()
    lib.rift_ile_check(h)
    return out.cpu().numpy().astype(np.float64)


def _break_q(pt, modes=None):
    """The point with the Q of each listed mode (default: every m < 0 mode) in detector 0 changed by
    1e-6 of the largest |Q| at one sample: Q_abar = sigma conj(Q_a) no longer holds for those pairs,
    so the kernels read them from their own rows (all of them: the full rows)."""
    Q = pt["Q"].copy()
    lm = [tuple(x) for x in np.asarray(pt["lm"]).tolist()]
    for mode in (modes if modes is not None else [x for x in lm if x[1] < 0]):
        Q[0, lm.index(mode), Q.shape[2] // 2] += 1e-6 * np.abs(Q).max()
    return dict(pt, Q=Q)


def test_merged_rows_are_taken_exactly_when_a_pair_is_reflection_symmetric(lib, cuda):
    """Real data and mirror-symmetric modes give Q_abar(t) = sigma_a conj(Q_a(t)) (Eq. (QUV)): the
    workload's points read merged rows; a perturbed Q whose only pair is (2, +-2), or a mode set
    without any mirror pair, does not."""
    for spec in (W.cfg_small(), W.cfg_full()):
        pt = W.make_point(spec, 8)
        h = lib.rift_ile_create(pt)
        assert lib.rift_ile_forms(h) & lib.FORM_QHALF
        lib.rift_ile_destroy(h)
    for modes, want in (([(2, -2), (2, 1), (2, 2)], False), ([(2, -2), (2, 1), (2, 2), (3, -3), (3, 3)], True)):
        spec = W.cfg_small()
        spec.modes = modes
        h = lib.rift_ile_create(_break_q(W.make_point(spec, 8), [(2, -2)]))
        assert bool(lib.rift_ile_forms(h) & lib.FORM_QHALF) == want, modes
        lib.rift_ile_destroy(h)
    spec = W.cfg_small()
    spec.modes = [(2, 1), (2, 2), (3, 3)]
    h = lib.rift_ile_create(W.make_point(spec, 8))
    assert not lib.rift_ile_forms(h) & lib.FORM_QHALF
    lib.rift_ile_destroy(h)


@pytest.mark.parametrize("which,n,interp,broken", [("small", 1500, 3, False), ("small", 400, 1, False),
                                                   ("small", 400, 0, False), ("full", 160, 3, False),
                                                   ("small", 400, 3, True), ("full", 160, 3, True)])
def test_tmarg_array_parity(lib, cuda, which, n, interp, broken):
    """Per draw against the oracle, with the half rows (the workload's points) and with the full
    rows (broken: Q no longer reflection symmetric)."""
    spec = W.cfg_small() if which == "small" else W.cfg_full()
    pt = W.make_point(spec, 8)
    if broken:
        pt = _break_q(pt)
    h = lib.rift_ile_create(pt, interp=interp)
    assert bool(lib.rift_ile_forms(h) & lib.FORM_QHALF) != broken
    th = _draws(n, 9)
    th64 = {k: v.astype(np.float64) for k, v in th.items()}
    got = _gpu(lib, h, th)
    want = TM.lnL_tmarg(pt, interp=interp, **th64)
    err = np.abs(got - want)
    tol = _tol(pt, th64)
    i = int(np.argmax(err / tol))
    assert np.all(err <= tol), (float(err[i]), float(tol[i]), float(want[i]), i)
    lib.rift_ile_destroy(h)


def test_tmarg_partly_merged_rows_match_oracle(lib, cuda):
    """A point whose (3, +-3) pair merges and whose (2, -2) keeps its own row (slots of both kinds),
    per draw against the oracle."""
    spec = W.cfg_small()
    spec.modes = [(2, -2), (2, 1), (2, 2), (3, -3), (3, 3)]
    pt = _break_q(W.make_point(spec, 8), [(2, -2)])
    h = lib.rift_ile_create(pt)
    assert lib.rift_ile_forms(h) & lib.FORM_QHALF
    th = _draws(600, 11)
    th64 = {k: v.astype(np.float64) for k, v in th.items()}
    err = np.abs(_gpu(lib, h, th) - TM.lnL_tmarg(pt, **th64))
    assert np.all(err <= _tol(pt, th64)), float(err.max())
    lib.rift_ile_destroy(h)


def test_tmarg_near_the_peak(lib, cuda):
    """Draws concentrated where L_margT is largest (the terms that dominate lnL_marg)."""
    pt = W.make_point(W.cfg_small(), 8)
    h = lib.rift_ile_create(pt)
    th = _draws(4000, 10)
    th64 = {k: v.astype(np.float64) for k, v in th.items()}
    got = _gpu(lib, h, th)
    top = np.argsort(got)[-200:]
    sub = {k: v[top] for k, v in th64.items()}
    want = TM.lnL_tmarg(pt, **sub)
    err = np.abs(got[top] - want)
    assert np.all(err <= _tol(pt, sub)), float(err.max())
    lib.rift_ile_destroy(h)


def _marg(lib, h, n, **kw):
    import torch
    dbg = torch.full((kw["max_evals"],), float("nan"), dtype=torch.float32, device="cuda")
    r = lib.rift_ile_marginalize(h, dbg_ell=dbg, time_marg=1, n_per_round=n, **kw)
    torch.cuda.synchronize()
    return r, dbg.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("broken", [False, True])
def test_tmarg_marginalize_matches_oracle(lib, cuda, broken):
    """Same Philox draws on both sides (the t uniform unused), sky strata 4 x 2: per-draw log weights
    within the per-draw tolerance, lnL_marg within 1e-4 (half rows, and full rows when broken)."""
    from oracle import mc
    pt = W.make_point(W.cfg_small(), 8)
    if broken:
        pt = _break_q(pt)
    h = lib.rift_ile_create(pt)
    n, S = 1500, (4, 2, 1)
    res, ell = _marg(lib, h, n, seed=71, max_evals=2 * n, strata=S)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    ref = mc.marginalize(pt, 71, 0, pr, n, 2 * n, 1e300, strata=S, time_marg=True, keep=True)
    want = np.concatenate([hh["ell"] for hh in ref["history"]])
    th0, _, _ = mc.draw(71, 0, 0, np.arange(n, dtype=np.uint64), pr, None, S, n)
    th1, _, _ = mc.draw(71, 0, 1, np.arange(n, dtype=np.uint64), pr, None, S, n)
    th64 = {k: np.concatenate([th0[k], th1[k]]) for k in th0}
    tol = _tol(pt, dict(ra=th64["ra"], dec=np.arcsin(th64["sindec"]), psi=th64["psi"], phi=th64["phi"],
                        incl=np.arccos(th64["cosi"]), dist=th64["dist"]))
    assert np.all(np.abs(ell - want) <= tol), float(np.max(np.abs(ell - want) / tol))
    assert abs(res["lnL_marg"] - ref["lnL_marg"]) < 1e-4, (res["lnL_marg"], ref["lnL_marg"])
    assert res["n_evals"] == 2 * n and res["strata"] == S
    lib.rift_ile_destroy(h)


def test_tmarg_adaptive_fixed_tables_matches_oracle(lib, cuda):
    """Adaptive (ra, sin dec) tables given, time table uniform, no rebuild: identical draws."""
    from oracle import mc
    pt = W.make_point(W.cfg_small(), 8)
    nb = 32
    r = np.random.default_rng(4)
    tab = np.empty((3, nb + 1), dtype=np.float32)
    for d in range(2):
        p = r.uniform(0.2, 3.0, nb)
        c = np.concatenate([[0.0], np.cumsum(p / p.sum())])
        tab[d] = c.astype(np.float32)
        tab[d, 0], tab[d, -1] = 0.0, 1.0
    tab[2] = mc.uniform_time_table(nb)
    h = lib.rift_ile_create(pt)
    n = 1200
    res, _ = _marg(lib, h, n, seed=72, max_evals=n, proposal="adaptive", n_bins=nb, tables=tab, adapt_rounds=0,
                   strata=(2, 2, 1))
    ref = mc.marginalize(pt, 72, 0, mc.Prior(pt["t_lo"], pt["t_hi"]), n, n, 1e300, adaptive=True, n_bins=nb,
                         tables=tab, adapt_rounds=0, strata=(2, 2, 1), time_marg=True)
    assert abs(res["lnL_marg"] - ref["lnL_marg"]) < 1e-4, (res["lnL_marg"], ref["lnL_marg"])
    lib.rift_ile_destroy(h)


def test_tmarg_estimate_agrees_with_sampled_time(lib, cuda):
    """Both estimators target the same L_marg (time integral by quadrature or by sampling): on a
    weak signal, where both converge, they agree within their Monte Carlo errors."""
    spec = W.cfg_small()
    spec.snr = 4.0
    pt = W.make_point(spec, 12)
    h = lib.rift_ile_create(pt)
    a = lib.rift_ile_marginalize(h, seed=73, n_per_round=1_000_000, max_evals=4_000_000)
    b = lib.rift_ile_marginalize(h, seed=74, n_per_round=20000, max_evals=80000, time_marg=1)
    sig = math.hypot(a["sigma"], b["sigma"])
    assert abs(a["lnL_marg"] - b["lnL_marg"]) < 4 * sig + 0.01, (a, b)
    assert b["n_eff"] > 50
    lib.rift_ile_destroy(h)


def test_tmarg_batch_equals_single_point_runs(lib, cuda):
    """The batched graph runner with the time quadrature gives every point exactly its
    single-point result (same draws, same rounds, same stopping)."""
    specs = W.batch_specs(3, seed=8, t_range=(800, 1200))
    pts = [W.make_point(sp, 20 + i) for i, sp in enumerate(specs)]
    hb = lib.rift_ile_batch_create(pts)
    assert all(lib.rift_ile_forms(hb, i) & lib.FORM_QHALF for i in range(3))
    kw = dict(seed=81, n_per_round=4000, max_evals=12000, n_eff_target=1e300, time_marg=1, proposal="adaptive",
              n_bins=32)
    batch = lib.rift_ile_batch_marginalize(hb, **kw)
    for i, p in enumerate(pts):
        h = lib.rift_ile_create(p)
        one = lib.rift_ile_marginalize(h, point_id=i, **kw)
        assert batch[i]["n_evals"] == one["n_evals"] and batch[i]["rounds"] == one["rounds"]
        assert batch[i]["lnL_marg"] == one["lnL_marg"], (i, batch[i]["lnL_marg"], one["lnL_marg"])
        lib.rift_ile_destroy(h)
    lib.rift_ile_destroy(hb)


def test_tmarg_mixed_batch_equals_single_point_runs(lib, cuda):
    """A batch whose points do not all have merged rows runs the kernel that chooses per point and
    scans each draw's own rows: the point without them gets exactly its single-point result, the
    others theirs within 1e-4 (alone they take the GEMM form of the scan, which sums in another
    order)."""
    specs = W.batch_specs(3, seed=9, t_range=(800, 1200))
    pts = [W.make_point(sp, 30 + i) for i, sp in enumerate(specs)]
    pts[1] = _break_q(pts[1])
    hb = lib.rift_ile_batch_create(pts)
    assert [bool(lib.rift_ile_forms(hb, i) & lib.FORM_QHALF) for i in range(3)] == [True, False, True]
    kw = dict(seed=82, n_per_round=3000, max_evals=6000, n_eff_target=1e300, time_marg=1, proposal="adaptive",
              n_bins=32)
    batch = lib.rift_ile_batch_marginalize(hb, **kw)
    for i, p in enumerate(pts):
        h = lib.rift_ile_create(p)
        one = lib.rift_ile_marginalize(h, point_id=i, **kw)
        if i == 1:
            assert batch[i]["lnL_marg"] == one["lnL_marg"], (i, batch[i]["lnL_marg"], one["lnL_marg"])
        else:
            assert abs(batch[i]["lnL_marg"] - one["lnL_marg"]) < 1e-4, (i, batch[i]["lnL_marg"], one["lnL_marg"])
        lib.rift_ile_destroy(h)
    lib.rift_ile_destroy(hb)


def test_tmarg_learned_matches_oracle(lib, cuda):
    """Learned proposal with the time quadrature: the mixture's time coordinate is integrated out
    (dropped from each diagonal component), the weight is that of the other four coordinates."""
    from oracle import mc, mdn
    from oracle import philox as P
    pt = W.make_point(W.cfg_small(), 8)
    a, b = mdn.bounds(pt["t_lo"], pt["t_hi"], 1.0, 1000.0)
    r = np.random.default_rng(5)
    head = np.zeros(88, dtype=np.float32)
    head[:8] = r.normal(0, 1, 8)
    head[8:48] = r.normal(0, 1.0, 40)
    head[48:88] = r.uniform(-1.0, 0.5, 40)
    h = lib.rift_ile_create(pt)
    lib.rift_ile_set_proposal_head(h, head[None])
    n = 1500
    res = lib.rift_ile_marginalize(h, seed=91, n_per_round=n, max_evals=n, proposal="learned", time_marg=1)
    u = P.uniforms(91, 0, 0, np.arange(n, dtype=np.uint64), 10)
    th, lq = mdn.sample(u, head.astype(np.float64)[None], mc.Prior(pt["t_lo"], pt["t_hi"]), time_marg=True)
    ell = TM.lnL_tmarg(pt, th["ra"], np.arcsin(th["sindec"]), th["psi"], th["phi"], np.arccos(th["cosi"]),
                       th["dist"]) + lq
    want = mc.Accum.of(ell).result()
    assert abs(res["lnL_marg"] - want[0]) < 1e-4, (res["lnL_marg"], want[0], res["n_eff"])
    lib.rift_ile_destroy(h)


def test_tmarg_resume_and_static_scratch(lib, cuda):
    """Checkpoint/resume and the allocation-free entry point carry the time quadrature too."""
    pt = W.make_point(W.cfg_small(), 8)
    h = lib.rift_ile_create(pt)
    kw = dict(seed=95, n_per_round=1000, max_evals=4000, n_eff_target=1e300, time_marg=1, proposal="adaptive",
              n_bins=24)
    full = lib.rift_ile_marginalize(h, **kw)
    part = lib.rift_ile_marginalize(h, save=True, max_rounds=2, **kw)
    rest = lib.rift_ile_marginalize(h, resume=part["state"], **kw)
    assert rest["lnL_marg"] == full["lnL_marg"] and rest["n_evals"] == full["n_evals"]
    with pytest.raises(lib.RiftError):   # a sampled-time run cannot resume a time-marginalised one
        lib.rift_ile_marginalize(h, resume=part["state"], **dict(kw, time_marg=0))
    st = lib.rift_ile_marginalize_static(h, **kw)
    assert st["lnL_marg"] == full["lnL_marg"] and st["n_evals"] == full["n_evals"]
    lib.rift_ile_destroy(h)


def test_adaptive_time_marginalised_run_reaches_neff_target_on_a_physical_injection(lib, cuda):
    """A physical injection (H1, L1, V1; l = 2; SNR 10): the time-marginalised estimator with the
    adaptive (ra, sin dec) proposal reaches n_eff >= 1000, and independent runs agree to 0.05."""
    from test_oracle_warm import phys_point
    pt = phys_point(41, snr=10.0)
    h = lib.rift_ile_create(pt)
    kw = dict(n_per_round=1_000_000, max_evals=200_000_000, n_eff_target=1000, proposal="adaptive", n_bins=64,
              beta=0.3, time_marg=1)
    a = lib.rift_ile_marginalize(h, seed=5, **kw)
    b = lib.rift_ile_marginalize(h, seed=6, **kw)
    lib.rift_ile_destroy(h)
    for r in (a, b):
        assert r["n_eff"] >= 1000 and r["n_evals"] < 200_000_000, r
    assert abs(a["lnL_marg"] - b["lnL_marg"]) < 0.05, (a["lnL_marg"], b["lnL_marg"])
    assert abs(a["lnL_marg"] - b["lnL_marg"]) < 4 * np.hypot(a["sigma"], b["sigma"])
