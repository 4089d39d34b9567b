"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each check is independent of the oracle's own formulas: published known-answer
vectors, closed forms, invariants, the brute-force definition of the likelihood,
exact special cases, and planted mistakes that must be caught.
"""
from __future__ import annotations

import math
from pathlib import Path

import numpy as np
import pytest

import workload as W
from oracle import geometry as G
from oracle import likelihood as L
from oracle import mc
from oracle import philox as P
from oracle import swsh as S

GOLD = Path(__file__).resolve().parent / "golden"


def _rng(seed=0):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- Philox / uniforms
def test_philox_known_answers():
    for line in (GOLD / "philox4x32_10_kat.txt").read_text().splitlines():
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = P.philox4x32_10([np.array([x]) for x in v[:4]], [np.array([x]) for x in v[4:6]])[:, 0]
        assert [int(x) for x in out] == v[6:], line


def test_uniforms_exact_in_float32_and_open_interval():
    x = np.array([0, 1, 511, 512, 2**31, 2**32 - 1], dtype=np.uint64)
    u = P.bits_to_uniform(x)
    assert np.all(u > 0) and np.all(u < 1)
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 0.5 * 2.0**-23 and u[-1] == 1.0 - 0.5 * 2.0**-23
    uu = P.uniforms(5, 3, 2, np.arange(1000, dtype=np.uint64), 8)
    assert np.array_equal(uu.astype(np.float32).astype(np.float64), uu)
    # sin dec = 2u - 1 and 1 - u are exact in float32 for these uniforms
    sd = 2.0 * uu[1] - 1.0
    assert np.array_equal(sd.astype(np.float32).astype(np.float64), sd)


def test_uniform_statistics():
    u = P.uniforms(123, 0, 0, np.arange(200000, dtype=np.uint64), 8)
    assert np.all(np.abs(u.mean(axis=1) - 0.5) < 0.005)
    assert np.all(np.abs(u.var(axis=1) - 1.0 / 12.0) < 0.002)
    c = np.corrcoef(u)
    assert np.max(np.abs(c - np.eye(8))) < 0.01


# ---------------------------------------------------------------- sidereal time
def test_gmst_j2000_and_sidereal_day():
    vals = dict(l.split() for l in (GOLD / "gmst_j2000.txt").read_text().splitlines() if l and not l.startswith("#"))
    d = float(vals["jd_ut1"]) - 2451545.0
    assert abs(math.degrees(G.gmst_from_days(d)) - float(vals["gmst_deg"])) < 1e-7
    g0 = G.gmst_from_gps(W.T_REF_GPS)
    g1 = G.gmst_from_gps(W.T_REF_GPS + 86164.0905)   # one sidereal day
    assert abs((g1 - g0 + np.pi) % (2 * np.pi) - np.pi) < 1e-5
    g2 = G.gmst_from_gps(W.T_REF_GPS + 43082.04525)  # half a sidereal day
    assert abs(abs((g2 - g0) % (2 * np.pi)) - np.pi) < 1e-5


# ---------------------------------------------------------------- detector response
def _sky(n, seed=1):
    r = _rng(seed)
    return r.uniform(0, 2 * np.pi, n), np.arcsin(r.uniform(-1, 1, n)), r.uniform(0, np.pi, n)


@pytest.mark.parametrize("det", ["H1", "L1", "V1"])
def test_response_psi_invariants(det):
    d, _ = W.detector(det)
    ra, dec, psi = _sky(500)
    g = 1.234
    F = G.complex_antenna(d, ra, dec, psi, g)
    Fq = G.complex_antenna(d, ra, dec, psi + np.pi / 2, g)
    Fh = G.complex_antenna(d, ra, dec, psi + np.pi, g)
    F0 = G.complex_antenna(d, ra, dec, np.zeros_like(psi), g)
    assert np.allclose(np.abs(F), np.abs(F0), rtol=0, atol=1e-13)       # F+^2 + Fx^2 psi-invariant
    assert np.allclose(Fq, -F, atol=1e-13)
    assert np.allclose(Fh, F, atol=1e-13)
    assert np.allclose(F, np.exp(2j * psi) * F0, atol=1e-13)            # spin-2 rotation
    assert np.all(np.abs(F) <= 1.0 + 1e-12)


def test_response_polar_detector_closed_form():
    """L-shaped detector at the north pole with arms along Earth-fixed x, y:
    F+^2 + Fx^2 = (1 + cos^2 th)^2 / 4 cos^2 2ph + cos^2 th sin^2 2ph, th = pi/2 - dec, ph = ra - GMST."""
    d = 0.5 * (np.diag([1.0, 0, 0]) - np.diag([0, 1.0, 0]))
    ra, dec, psi = _sky(300, 2)
    g = 0.77
    F = G.complex_antenna(d, ra, dec, psi, g)
    th, ph = np.pi / 2 - dec, ra - g
    want = 0.25 * (1 + np.cos(th) ** 2) ** 2 * np.cos(2 * ph) ** 2 + np.cos(th) ** 2 * np.sin(2 * ph) ** 2
    assert np.allclose(np.abs(F) ** 2, want, atol=1e-13)
    # source overhead: |F| = 1
    assert abs(abs(G.complex_antenna(d, 0.3, np.pi / 2, 0.4, g)) - 1.0) < 1e-13


def test_delay_sign_and_bound():
    pos = np.array([0.0, 0.0, 6.4e6])
    # source straight above the vertex: the vertex is reached first (negative delay)
    assert G.delay(pos, 0.1, np.pi / 2, 0.0) == pytest.approx(-6.4e6 / G.C_LIGHT, rel=1e-14)
    assert G.delay(pos, 0.1, -np.pi / 2, 0.0) == pytest.approx(6.4e6 / G.C_LIGHT, rel=1e-14)
    _, x = W.detector("H1")
    ra, dec, _ = _sky(1000, 3)
    dl = G.delay(x, ra, dec, 0.5)
    assert np.max(np.abs(dl)) <= W.max_light_delay(x) + 1e-15


# ---------------------------------------------------------------- spin-weighted harmonics
def test_swsh_l2_closed_forms():
    r = _rng(4)
    th, ph = r.uniform(0, np.pi, 200), r.uniform(0, 2 * np.pi, 200)
    c = np.cos(th)
    want = {2: np.sqrt(5 / (64 * np.pi)) * (1 + c) ** 2 * np.exp(2j * ph),
            1: np.sqrt(5 / (16 * np.pi)) * np.sin(th) * (1 + c) * np.exp(1j * ph),
            0: np.sqrt(15 / (32 * np.pi)) * np.sin(th) ** 2 + 0j,
            -1: np.sqrt(5 / (16 * np.pi)) * np.sin(th) * (1 - c) * np.exp(-1j * ph),
            -2: np.sqrt(5 / (64 * np.pi)) * (1 - c) ** 2 * np.exp(-2j * ph)}
    for m, w in want.items():
        assert np.allclose(S.swsh(-2, 2, m, th, ph), w, atol=1e-14), m


@pytest.mark.parametrize("l", [2, 3, 4])
def test_swsh_addition_theorem(l):
    r = _rng(5)
    th, ph = r.uniform(0, np.pi, 100), r.uniform(0, 2 * np.pi, 100)
    tot = sum(np.abs(S.swsh(-2, l, m, th, ph)) ** 2 for m in range(-l, l + 1))
    assert np.allclose(tot, (2 * l + 1) / (4 * np.pi), atol=1e-13)


def test_swsh_orthonormal_by_quadrature():
    x, w = np.polynomial.legendre.leggauss(40)     # cos theta nodes
    th = np.arccos(x)
    nph = 24
    ph = 2 * np.pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    Wt = np.repeat(w[:, None], nph, axis=1) * (2 * np.pi / nph)
    modes = W.ALL_MODES
    Y = np.stack([S.swsh(-2, l, m, TH, PH) for (l, m) in modes])
    gram = np.einsum("aij,bij,ij->ab", np.conj(Y), Y, Wt)
    assert np.allclose(gram, np.eye(len(modes)), atol=1e-12)


def test_swsh_conjugation_relation():
    """conj(sY_lm) = (-1)^(s+m) (-s)Y_{l,-m}: relates the s = -2 family to s = +2."""
    r = _rng(6)
    th, ph = r.uniform(0, np.pi, 50), r.uniform(0, 2 * np.pi, 50)
    for (l, m) in W.ALL_MODES:
        lhs = np.conj(S.swsh(-2, l, m, th, ph))
        rhs = (-1) ** (-2 + m) * S.swsh(2, l, -m, th, ph)
        assert np.allclose(lhs, rhs, atol=1e-14), (l, m)


# ---------------------------------------------------------------- likelihood
@pytest.fixture(scope="module")
def small_point():
    spec = W.cfg_small()
    spec.seg_len = 2.0
    return W.make_point(spec, 21)


@pytest.fixture(scope="module")
def hm_point():
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.ALL_MODES), fs=4096.0, seg_len=2.0, snr=20.0)
    return W.make_point(spec, 22)


def _draws(n, seed, t_half=0.05):
    r = _rng(seed)
    return dict(ra=r.uniform(0, 2 * np.pi, n), dec=np.arcsin(r.uniform(-1, 1, n)), t=r.uniform(-t_half, t_half, n),
                psi=r.uniform(0, np.pi, n), phi=r.uniform(0, 2 * np.pi, n), incl=np.arccos(r.uniform(-1, 1, n)),
                dist=r.uniform(30, 800, n))


@pytest.mark.parametrize("which", ["small_point", "hm_point"])
def test_factorised_equals_bruteforce(which, request):
    """Eq. (def:lnL:Decomposed) with exact Q(t) equals Eq. (lnL) built from Eq. (overlap)."""
    pt = request.getfixturevalue(which)
    th = _draws(6, 7)
    fac = L.lnL_factorised(pt, **th, exact=True)
    for i in range(6):
        bf = L.lnL_bruteforce(pt, **{k: v[i] for k, v in th.items()})
        assert abs(fac[i] - bf) <= 1e-10 * max(1.0, abs(bf)), (i, fac[i], bf)


def _mutated_lnL(pt, th, mutation):
    """Planted mistakes, applied to a copy of the factorised formula."""
    gm, tens, pos = L._geometry(pt)
    modes = [tuple(v) for v in np.asarray(pt["lm"]).tolist()]
    Y = L.ylm_m2(modes, th["incl"], th["phi"])
    x = pt["d_ref_mpc"] / th["dist"]
    lin = quad = 0.0
    for k in range(tens.shape[0]):
        F = G.complex_antenna(tens[k], th["ra"], th["dec"], th["psi"], gm)
        tk = th["t"] + G.delay(pos[k], th["ra"], th["dec"], gm)
        if mutation == "delay_sign":
            tk = th["t"] - G.delay(pos[k], th["ra"], th["dec"], gm)
        Qk = L.q_exact(pt, k, tk)
        Fl = np.conj(F) if mutation == "paper_literal" else F
        lin += np.real(Fl * np.sum(np.conj(Y) * Qk, -1))
        A = np.real(np.einsum("na,ab,nb->n", np.conj(Y), pt["U"][k], Y))
        Vk = pt["V"][k].T.conj() if mutation == "V_conj" else pt["V"][k]
        B = np.einsum("na,ab,nb->n", Y, Vk, Y)
        Fq = F if mutation == "paper_literal" else np.conj(F)
        if mutation == "drop_V":
            B = 0 * B
        quad += np.abs(F) ** 2 * A + np.real(Fq ** 2 * B)
    pref = 0.5 if mutation == "half_not_quarter" else 0.25
    return x * lin - pref * x * x * quad


@pytest.mark.parametrize("mutation", ["paper_literal", "drop_V", "V_conj", "half_not_quarter", "delay_sign"])
def test_planted_mistakes_are_caught(hm_point, mutation):
    th = {k: v for k, v in _draws(4, 8).items()}
    bf = np.array([L.lnL_bruteforce(hm_point, **{k: v[i] for k, v in th.items()}) for i in range(4)])
    mut = _mutated_lnL(hm_point, th, mutation)
    assert np.max(np.abs(mut - bf)) > 1e-3 * max(1.0, np.max(np.abs(bf))), mutation


def test_zero_noise_peak_and_cauchy_schwarz():
    """Zero-noise data: lnL(theta_inj) = rho^2/2 exactly, and lnL <= rho^2/2 everywhere."""
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.ALL_MODES), fs=4096.0, seg_len=2.0, snr=20.0, noise=False)
    inj = dict(ra=1.1, dec=-0.3, t=0.012, psi=0.4, phi=2.0, incl=0.9, dist=300.0)
    tens = np.stack([W.detector(d)[0] for d in spec.dets])
    pos = np.stack([W.detector(d)[1] for d in spec.dets])
    coef, tk = L.injection((tens, pos), spec.modes, **inj, d_ref=spec.d_ref, t_ref_gps=spec.t_ref_gps)
    pt = W.make_point(spec, 31, injection=(coef, tk))
    peak = L.lnL_factorised(pt, **{k: np.array([v]) for k, v in inj.items()}, exact=True)[0]
    assert abs(peak - 0.5 * spec.snr ** 2) < 1e-9 * spec.snr ** 2
    th = _draws(2000, 9)
    vals = L.lnL_factorised(pt, **th)
    assert np.max(vals) < 0.5 * spec.snr ** 2
    # perturbing any coordinate lowers the exact likelihood
    for key, step in (("ra", 1e-3), ("dec", 1e-3), ("t", 1e-4), ("psi", 1e-2), ("phi", 1e-2), ("incl", 1e-2),
                      ("dist", 3.0)):
        for sgn in (-1, 1):
            th2 = {k: np.array([v]) for k, v in inj.items()}
            th2[key] = th2[key] + sgn * step
            assert L.lnL_factorised(pt, **th2, exact=True)[0] < peak, key


def test_lnL_quadratic_in_inverse_distance(small_point):
    th = _draws(5, 10)
    a = L.lnL_factorised(small_point, **{**th, "dist": np.full(5, 100.0)})   # x = 1
    b = L.lnL_factorised(small_point, **{**th, "dist": np.full(5, 50.0)})    # x = 2
    c = L.lnL_factorised(small_point, **{**th, "dist": np.full(5, 200.0)})   # x = 1/2
    # lnL(x) = A x - B x^2 -> from x = 1, 2: B = (2 a - b) / 2, A = a + B
    B = (2 * a - b) / 2
    A = a + B
    assert np.allclose(c, A * 0.5 - B * 0.25, rtol=1e-12, atol=1e-10)


def test_psi_period_pi_and_22_symmetry(small_point):
    th = _draws(20, 11)
    a = L.lnL_factorised(small_point, **th)
    b = L.lnL_factorised(small_point, **{**th, "psi": th["psi"] + np.pi})
    assert np.allclose(a, b, atol=1e-9)
    # a mode set with |m| = 2 only: lnL(psi + pi/2, phi + pi/2) = lnL(psi, phi)
    pt2 = dict(small_point)
    keep = [i for i, (l, m) in enumerate(pt2["lm"].tolist()) if abs(m) == 2]
    pt2["lm"] = pt2["lm"][keep]
    pt2["Q"] = pt2["Q"][:, keep]
    pt2["U"] = pt2["U"][:, keep][:, :, keep]
    pt2["V"] = pt2["V"][:, keep][:, :, keep]
    c = L.lnL_factorised(pt2, **th)
    d = L.lnL_factorised(pt2, **{**th, "psi": th["psi"] + np.pi / 2, "phi": th["phi"] + np.pi / 2})
    assert np.allclose(c, d, atol=1e-9)


def test_zero_inner_products_give_zero(small_point):
    pt = dict(small_point)
    pt["Q"] = np.zeros_like(pt["Q"])
    pt["U"] = np.zeros_like(pt["U"])
    pt["V"] = np.zeros_like(pt["V"])
    assert np.all(L.lnL_factorised(pt, **_draws(50, 12)) == 0.0)
    r = mc.marginalize(pt, 3, 0, mc.Prior(-0.05, 0.05), 1000, 1000, 1e300)
    assert r["lnL_marg"] == 0.0 and r["n_eff"] == 1000


def test_interpolation_exact_on_cubics():
    r = _rng(13)
    coefs = r.normal(size=(3, 4)) + 1j * r.normal(size=(3, 4))
    j = np.arange(40.0)
    grid = np.stack([np.polyval(c, j) for c in coefs])
    s = r.uniform(1.0, 36.9, 200)
    got = L.q_interp(grid, s, 3)
    want = np.stack([np.polyval(c, s) for c in coefs], axis=-1)
    assert np.allclose(got, want, rtol=1e-12, atol=1e-9)
    lin = L.q_interp(grid[:, :], s, 1)
    assert np.allclose(lin[:, 0], (1 - (s - np.floor(s))) * grid[0, np.floor(s).astype(int)] +
                       (s - np.floor(s)) * grid[0, np.floor(s).astype(int) + 1])
    with pytest.raises(ValueError):
        L.q_interp(grid, np.array([0.5]), 3)


def test_interpolated_matches_exact_within_interpolation_error(small_point):
    th = _draws(200, 14)
    a = L.lnL_factorised(small_point, **th)
    b = L.lnL_factorised(small_point, **th, exact=True)
    assert np.max(np.abs(a - b)) < 0.05 * max(1.0, np.max(np.abs(b)))


# ---------------------------------------------------------------- Monte Carlo
def test_accumulator_matches_sorted_exact_sum_and_merges():
    r = _rng(15)
    ell = np.concatenate([r.normal(0, 30, 3000), [700.0, -800.0, 699.5]])
    a = mc.Accum.of(ell)
    m = ell.max()
    exact = math.fsum(sorted(np.exp(ell - m).tolist()))
    assert abs(a.result()[0] - (m + math.log(exact) - math.log(ell.size))) < 1e-13
    # shards merged in different orders give the same state
    idx = r.permutation(ell.size)
    shards = np.array_split(ell[idx], 7)
    parts = [mc.Accum.of(s) for s in shards]
    fwd = mc.Accum()
    for p in parts:
        fwd = fwd.merge(p)
    bwd = mc.Accum()
    for p in reversed(parts):
        bwd = bwd.merge(p)
    for x, y in zip(fwd.result(), bwd.result()):
        assert abs(x - y) <= 1e-12 * max(1.0, abs(x))
    assert abs(fwd.result()[0] - a.result()[0]) < 1e-12


def test_constant_likelihood_gives_constant_and_full_neff():
    ell = np.full(5000, 3.25)
    r = mc.Accum.of(ell).result()
    assert abs(r[0] - 3.25) < 1e-14 and abs(r[1] - 5000) < 1e-9 and abs(r[2] - 5000) < 1e-9


def test_prior_transform_ranges_and_distance_law():
    pr = mc.Prior(-0.05, 0.05, 1.0, 1000.0)
    u = P.uniforms(9, 0, 0, np.arange(100000, dtype=np.uint64), 8)
    th = mc.prior_transform(u, pr)
    assert th["ra"].min() > 0 and th["ra"].max() < 2 * np.pi
    assert th["t"].min() > -0.05 and th["t"].max() < 0.05
    assert th["dist"].min() >= 1.0 and th["dist"].max() <= 1000.0
    # p(D) ~ D^2: P(D < 500) = (500^3 - 1) / (1000^3 - 1)
    assert abs(np.mean(th["dist"] < 500.0) - (500.0 ** 3 - 1) / (1000.0 ** 3 - 1)) < 0.005


def test_inverse_cdf_uniform_table_and_weights():
    nb = 50
    tab = mc.uniform_tables(nb)[0]
    u = P.uniforms(4, 0, 0, np.arange(20000, dtype=np.uint64), 1)[0]
    x, b, pb = mc.inverse_cdf(tab, u)
    assert np.allclose(x, u, atol=1e-7) and np.all(b == np.floor(u * nb))
    # a peaked table: sampled density follows the table, weights p/q average to 1
    c = np.concatenate([[0.0], np.cumsum(np.linspace(1, 10, nb))])
    c = (c / c[-1]).astype(np.float32)
    c[-1] = 1.0
    x, b, pb = mc.inverse_cdf(c, u)
    hist = np.bincount(b, minlength=nb) / u.size
    assert np.max(np.abs(hist - np.diff(c.astype(np.float64)))) < 0.005
    assert abs(np.mean(1.0 / (nb * pb)) - 1.0) < 0.02


def test_distance_marginal_against_quadrature(small_point):
    """Only D varies: Monte Carlo over p(D) ~ D^2 vs Gauss-Legendre quadrature of the same integral."""
    th0 = {k: v[0] for k, v in _draws(1, 16).items()}
    dlo, dhi = 20.0, 1000.0
    xg, wg = np.polynomial.legendre.leggauss(400)
    D = 0.5 * (dhi - dlo) * xg + 0.5 * (dhi + dlo)
    lnl = L.lnL_factorised(small_point, **{k: np.full(D.size, v) for k, v in th0.items() if k != "dist"}, dist=D)
    pD = 3 * D ** 2 / (dhi ** 3 - dlo ** 3)
    m = lnl.max()
    quad = m + math.log(np.sum(0.5 * (dhi - dlo) * wg * pD * np.exp(lnl - m)))
    u = P.uniforms(17, 0, 0, np.arange(200000, dtype=np.uint64), 8)[6]
    Ds = np.cbrt(dlo ** 3 + u * (dhi ** 3 - dlo ** 3))
    lm = L.lnL_factorised(small_point, **{k: np.full(Ds.size, v) for k, v in th0.items() if k != "dist"}, dist=Ds)
    est, neff, kish, sig = mc.Accum.of(lm).result()
    assert abs(est - quad) < 4 * sig + 1e-6


def _physical_point(snr, seed=41):
    spec = W.PointSpec(dets=("H1", "L1", "V1"), modes=list(W.L2_MODES), fs=4096.0, snr=snr, t_half=0.02,
                       seg_len=4.0)
    tens = np.stack([W.detector(d)[0] for d in spec.dets])
    pos = np.stack([W.detector(d)[1] for d in spec.dets])
    coef, tk = L.injection((tens, pos), spec.modes, ra=2.0, dec=0.5, t=0.003, psi=0.3, phi=1.0, incl=0.6,
                           dist=300.0, d_ref=spec.d_ref, t_ref_gps=spec.t_ref_gps)
    return W.make_point(spec, seed, injection=(coef, tk))


def test_adaptive_is_unbiased_against_plain():
    """Adaptive proposal vs plain prior sampling on a weak physical signal (SNR 4, where both
    estimators are well resolved): the same lnL_marg within the combined MC error."""
    pt = _physical_point(4.0)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    plain = mc.marginalize(pt, 101, 0, pr, 100000, 400000, 1e300)
    ad = mc.marginalize(pt, 102, 0, pr, 50000, 400000, 1e300, adaptive=True, n_bins=50)
    assert plain["n_eff"] > 30 and ad["n_eff"] > 30
    s = math.hypot(plain["sigma"], ad["sigma"])
    assert abs(plain["lnL_marg"] - ad["lnL_marg"]) < 5 * s + 0.005


def test_rebuild_tables_properties():
    r = _rng(18)
    ell = r.normal(0, 3, 5000)
    bins = r.integers(0, 20, size=(3, 5000))
    tab, h = mc.rebuild_tables(ell, bins, 20, 0.8, 0.1)
    for d in range(3):
        c = tab[d].astype(np.float64)
        assert c[0] == 0.0 and c[-1] == 1.0 and np.all(np.diff(c) > 0)
        p = np.diff(c)
        assert np.all(p >= 0.1 / 20 * (1 - 1e-6))


def test_rebuild_tables_hand_computed():
    """The adaptive rebuild (tempered weights exp(beta (l - max l)) summed per bin, floor-mixed
    p_b = (1 - eps) h_b / sum h + eps / n_bins, float32 CDF) on five samples worked out by hand:
    beta = 1/2, eps = 1/5, 4 bins, log weights 3000 + {2 ln 2, 0, 0, -2 ln 2, 2 ln 2}, so the
    tempered weights are {1, 1/2, 1/2, 1/4, 1}.  The offset 3000 overflows exp(beta l) unless the
    maximum is taken out first."""
    l2 = math.log(2.0)
    ell = 3000.0 + np.array([2 * l2, 0.0, 0.0, -2 * l2, 2 * l2])
    bins = np.array([[0, 1, 1, 3, 0],      # ra: h = (2, 1, 0, 1/4)
                     [2, 2, 2, 2, 2],      # sin dec: all in bin 2, h = (0, 0, 13/4, 0)
                     [3, 0, 1, 2, 0]])     # t: h = (3/2, 1/2, 1/4, 1)
    tab, _ = mc.rebuild_tables(ell, bins, 4, 0.5, 0.2)
    # ra: p = (4/5) h / (13/4) + 1/20 = (141, 77, 13, 29) / 260
    want0 = np.array([0, 141, 218, 231, 260]) / 260.0
    # sin dec: p = (1/20, 1/20, 4/5 + 1/20, 1/20)
    want1 = np.array([0, 1, 2, 19, 20]) / 20.0
    # t: sum h = 13/4, p = (16/65)(3/2, 1/2, 1/4, 1) + 1/20 = (109, 45, 29, 77) / 260
    want2 = np.array([0, 109, 154, 183, 260]) / 260.0
    for d, want in enumerate((want0, want1, want2)):
        assert np.array_equal(tab[d], want.astype(np.float32)), (d, tab[d], want)


# ---------------------------------------------------------------- stratified rounds
def test_cell_mapping_contiguous_and_balanced():
    for n, C in ((23, 4), (100000, 1024), (1024, 1024), (5000, 7)):
        c, n_c = mc.cell_of(np.arange(n), n, C)
        assert np.all(np.diff(c) >= 0) and c.min() == 0 and c.max() == C - 1
        counts = np.bincount(c, minlength=C)
        assert np.array_equal(counts, n_c[np.searchsorted(c, np.arange(C))])
        assert counts.max() - counts.min() <= 1 and counts.sum() == n


def test_stratified_estimator_exact_for_cellwise_constant_weights():
    """A weight that is constant on every cell is integrated exactly by the stratified round,
    whatever the (uneven) number of samples per cell -- this fixes the ln(n / (C n_c)) term."""
    S = (4, 2, 8)
    C = 64
    r = _rng(19)
    g = r.uniform(0.1, 3.0, C)                       # weight of each cell
    for n in (64, 1000, 4097):
        u = P.uniforms(3, 0, 0, np.arange(n, dtype=np.uint64), 8)
        us, corr = mc.stratify(u, np.arange(n), n, S)
        cell = (np.floor(us[0] * S[0]) + S[0] * (np.floor(us[1] * S[1]) + S[1] * np.floor(us[2] * S[2]))).astype(int)
        ell = np.log(g[cell]) + corr
        est = mc.Accum.of(ell).result()[0]
        assert abs(est - math.log(g.mean())) < 1e-12, n


def test_stratified_uniforms_stay_in_their_cells_and_rounds_below_C_are_plain():
    S = (8, 4, 2)
    n = 1000
    u = P.uniforms(4, 0, 0, np.arange(n, dtype=np.uint64), 8)
    us, _ = mc.stratify(u, np.arange(n), n, S)
    c, _ = mc.cell_of(np.arange(n), n, 64)
    assert np.array_equal(np.floor(us[0] * 8), c % 8)
    assert np.array_equal(np.floor(us[2] * 2), c // 32)
    assert np.array_equal(us[3:], u[3:])
    u2, corr = mc.stratify(u[:, :40], np.arange(40), 40, S)  # 40 < 64 cells: not stratified
    assert np.array_equal(u2, u[:, :40]) and np.all(corr == 0)
    with pytest.raises(ValueError):
        mc.effective_strata(100, (3, 1, 1))


def test_stratified_marginalisation_agrees_with_plain():
    pt = _physical_point(4.0)
    pr = mc.Prior(pt["t_lo"], pt["t_hi"])
    plain = mc.marginalize(pt, 201, 0, pr, 100000, 300000, 1e300)
    strat = mc.marginalize(pt, 202, 0, pr, 100000, 300000, 1e300, strata=(16, 8, 8))
    s = math.hypot(plain["sigma"], strat["sigma"])
    assert abs(plain["lnL_marg"] - strat["lnL_marg"]) < 5 * s + 0.005


# ---------------------------------------------------------------- reflection-symmetric modes
def test_positive_quadratic_form_of_mirror_symmetric_modes():
    """The identity the kernels use for points whose modes carry the reflection symmetry of
    non-precessing sources, conj(h_a(-f)) = sigma_a h_mirror(a)(f): the detector strain is
    x sum_a beta_a h_a with beta_a = (conj(F) Y_a + sigma_a F conj(Y_mirror(a))) / 2, so the
    quadratic form of Eq. (def:lnL:Decomposed) is 2 beta^H U beta.  The synthetic full-size point
    has the symmetry (sigma = -1 for odd l, m != 0; its m = 0 modes are real), which shows in its
    inputs as V_ab = sigma_a U_mirror(a),b; on random draws the positive form equals the oracle's
    general form (-4 lnL / x^2 with Q = 0) to 1e-12."""
    pt = W.make_point(W.cfg_full(), 2)
    modes = [tuple(x) for x in np.asarray(pt["lm"]).tolist()]
    mir = np.array([modes.index((l, -m)) for l, m in modes])
    sig = np.array([(-1.0 if (l % 2 and m != 0) else 1.0) for l, m in modes])
    U, V = pt["U"], pt["V"]
    scale = np.abs(U).max()
    assert np.abs(V - sig[None, :, None] * U[:, mir, :]).max() < 1e-12 * scale
    r = _rng(31)
    n = 200
    th = dict(ra=r.uniform(0, 2 * np.pi, n), dec=np.arcsin(r.uniform(-1, 1, n)), t=np.zeros(n),
              psi=r.uniform(0, np.pi, n), phi=r.uniform(0, 2 * np.pi, n), incl=np.arccos(r.uniform(-1, 1, n)),
              dist=np.full(n, 100.0))
    silent = dict(pt, Q=np.zeros_like(pt["Q"]))
    general = -4.0 * L.lnL_factorised(silent, **th)          # x = d_ref / D = 1
    Y = S.ylm_m2(modes, th["incl"], th["phi"])                # (n, M)
    gm = G.gmst_from_gps(pt["t_ref_gps"])
    pos = np.zeros(n)
    for k in range(U.shape[0]):
        F = G.complex_antenna(pt["det_tensor"][k], th["ra"], th["dec"], th["psi"], gm)
        beta = 0.5 * (np.conj(F)[:, None] * Y + sig[None, :] * F[:, None] * np.conj(Y[:, mir]))
        pos += 2.0 * np.real(np.einsum("na,ab,nb->n", np.conj(beta), U[k], beta))
    assert np.all(pos >= 0)
    assert np.max(np.abs(pos - general)) < 1e-12 * np.max(np.abs(general))


def test_merged_rows_of_real_data():
    """Real data and modes with conj(h_a(-f)) = sigma h_abar(f) give Q_abar(t) = sigma conj(Q_a(t))
    from Eq. (QUV) (the direct sums of the oracle), so the likelihood is unchanged when every m < 0
    row is replaced by sigma conj(row of its mirror); data made complex break the relation."""
    from oracle import quv as QUV
    pt = W.make_point(W.cfg_small(), 8)
    Q = QUV.quv(pt)[0]
    lm = [tuple(x) for x in np.asarray(pt["lm"]).tolist()]
    qmax = np.abs(Q).max()
    Q2 = Q.copy()
    for i, (l, m) in enumerate(lm):
        if m < 0:
            continue
        j = lm.index((l, -m))
        errs = [np.abs(Q[:, j] - s * np.conj(Q[:, i])).max() for s in (1.0, -1.0)]
        assert min(errs) <= 1e-12 * qmax, (l, m, errs)
        if m > 0:
            Q2[:, j] = (1.0, -1.0)[int(np.argmin(errs))] * np.conj(Q[:, i])
    r = np.random.default_rng(3)
    n = 200
    th = dict(ra=r.uniform(0, 2 * np.pi, n), dec=np.arcsin(r.uniform(-1, 1, n)), t=r.uniform(-0.04, 0.04, n),
              psi=r.uniform(0, np.pi, n), phi=r.uniform(0, 2 * np.pi, n), incl=np.arccos(r.uniform(-1, 1, n)),
              dist=r.uniform(50.0, 500.0, n))
    a = L.lnL_factorised(dict(pt, Q=Q), **th)
    b = L.lnL_factorised(dict(pt, Q=Q2), **th)
    assert np.max(np.abs(a - b)) <= 1e-9 * max(1.0, np.max(np.abs(a)))
    Qc = QUV.quv(dict(pt, data=pt["data"] * np.exp(0.3j)))[0]
    i, j = lm.index((2, 2)), lm.index((2, -2))
    assert min(np.abs(Qc[:, j] - s * np.conj(Qc[:, i])).max() for s in (1.0, -1.0)) > 1e-3 * np.abs(Qc).max()
