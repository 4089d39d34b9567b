"""GPU parity of the extrinsic posterior samples (weighted export, systematic resampling, event
time of time-marginalised draws) against the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L
from oracle import mc
from oracle import posterior as PO

pytestmark = pytest.mark.gpu

TOL_LNL = 1e-3


@pytest.fixture(scope="module")
def p_small():
    return W.make_point(W.cfg_small(), 1)


def _hh(pt, cols):
    z = dict(pt, Q=np.zeros_like(pt["Q"]))
    t = cols["t"] if not np.any(np.isnan(cols["t"])) else np.zeros_like(cols["ra"])
    return -2.0 * L.lnL_factorised(z, cols["ra"], cols["dec"], t, cols["psi"], cols["phi"], cols["incl"], cols["dist"])


def _tol(pt, cols):
    return TOL_LNL * np.maximum(1.0, _hh(pt, cols) / 900.0)


def _fixed_tables(nb=16):
    c = np.concatenate([[0.0], np.cumsum(np.linspace(1.0, 3.0, nb))])
    t = (c / c[-1]).astype(np.float32)
    t[-1] = 1.0
    return np.stack([t, t[::-1].copy() * 0 + t, t])


def _compare_rows(pt, got, ref, n, lnpq=True):
    """Exported rows against the oracle's draws of the same round."""
    g = got[:n].astype(np.float64)
    assert np.allclose(g[:, 0], ref["ra"], rtol=0, atol=4e-6)
    assert np.allclose(np.sin(g[:, 1]), np.sin(ref["dec"]), rtol=0, atol=2e-6)
    if np.all(np.isnan(ref["t"])):
        assert np.all(np.isnan(g[:, 2]))
    else:
        assert np.allclose(g[:, 2], ref["t"], rtol=0, atol=2e-8)
    assert np.allclose(g[:, 3], ref["psi"], rtol=0, atol=2e-6)
    assert np.allclose(g[:, 4], ref["phi"], rtol=0, atol=4e-6)
    assert np.allclose(np.cos(g[:, 5]), np.cos(ref["incl"]), rtol=0, atol=2e-6)
    assert np.allclose(g[:, 6], ref["dist"], rtol=2e-6, atol=0)
    assert np.all(np.abs(g[:, 7] - ref["lnL"]) <= _tol(pt, ref)), np.max(np.abs(g[:, 7] - ref["lnL"]))
    if lnpq:
        assert np.allclose(g[:, 8], ref["lnpq"], rtol=0, atol=2e-5)


@pytest.mark.parametrize("case", ["prior", "tables", "tmarg"])
def test_weighted_export_matches_oracle(lib, cuda, p_small, case):
    """Every draw of the last round (the second of two, ragged strata) against the oracle's draws."""
    n = 6000 if case == "tmarg" else 30000     # the oracle's quadrature costs J likelihoods per draw
    pr = mc.Prior(p_small["t_lo"], p_small["t_hi"])
    kw = dict(seed=61, n_per_round=n, max_evals=2 * n - 777, strata=(4, 2, 4))
    okw = {}
    if case == "tables":
        kw.update(proposal="adaptive", n_bins=16, tables=_fixed_tables(), adapt_rounds=0)
        okw = dict(adaptive=True, n_bins=16, tables=_fixed_tables(), adapt_rounds=0)
    if case == "tmarg":
        kw.update(time_marg=1, strata=(4, 2, 1))
    h = lib.rift_ile_create(p_small)
    cap = n + 5
    rows, counts, res = lib.rift_ile_samples(h, cap, **kw)
    ref = PO.last_round(p_small, 61, 0, pr, n, 2 * n - 777, 1e300, strata=kw["strata"],
                        time_marg=case == "tmarg", **okw)
    m = n - 777
    assert counts == [m] and res[0]["rounds"] == 2
    got = rows[0].cpu().numpy()
    _compare_rows(p_small, got, ref, m)
    assert np.all(np.isnan(got[m:]))
    assert abs(res[0]["lnL_marg"] - ref["result"]["lnL_marg"]) < 1e-4
    lib.rift_ile_destroy(h)


def test_export_counts_only_and_truncation(lib, cuda, p_small):
    h = lib.rift_ile_create(p_small)
    kw = dict(seed=62, n_per_round=5000, max_evals=5000)
    _, counts, _ = lib.rift_ile_samples(h, 0, **kw)
    assert counts == [5000]
    rows, counts, _ = lib.rift_ile_samples(h, 100, **kw)
    full, _, _ = lib.rift_ile_samples(h, 5000, **kw)
    assert counts == [5000]
    assert np.array_equal(rows[0].cpu().numpy(), full[0, :100].cpu().numpy())
    lib.rift_ile_destroy(h)


def _valid_slots(idx, C, tol):
    """Slot h may take row i when C_{i-1} <= target_h < C_i holds within tol * C_{n-1}."""
    H = idx.size
    tot = C[-1]
    target = (np.arange(H) + 0.5) * tot / H
    lo = np.where(idx > 0, C[np.maximum(idx - 1, 0)], 0.0)
    hi = C[idx]
    return (lo <= target + tol * tot) & (target < hi + tol * tot)


@pytest.mark.parametrize("case", ["prior", "tables"])
def test_posterior_resampling_matches_oracle(lib, cuda, p_small, case):
    """The resampled draws: each valid for the oracle's cumulative weights within the FP32 error
    of the log weights, nearly all identical to the oracle's choice, and each row the exported row
    of its draw bit for bit."""
    n, H = 40000, 3000
    kw = dict(seed=63, n_per_round=n, max_evals=n, strata=(2, 2, 2))
    okw = {}
    if case == "tables":
        kw.update(proposal="adaptive", n_bins=16, tables=_fixed_tables(), adapt_rounds=0)
        okw = dict(adaptive=True, n_bins=16, tables=_fixed_tables(), adapt_rounds=0)
    h = lib.rift_ile_create(p_small)
    rows, idx, res = lib.rift_ile_posterior(h, H, **kw)
    exp, _, _ = lib.rift_ile_samples(h, n, **kw)
    pr = mc.Prior(p_small["t_lo"], p_small["t_hi"])
    ref = PO.posterior(p_small, 63, 0, pr, n, n, 1e300, H, strata=(2, 2, 2), **okw)
    gi = idx[0].cpu().numpy().astype(np.int64)
    assert np.all((gi >= 0) & (gi < n)) and np.all(np.diff(gi) >= 0)
    _, C = PO.systematic_resample(ref["draws"]["ell"], H)
    assert np.all(_valid_slots(gi, C, 4e-3))
    assert np.mean(gi == ref["idx"]) > 0.98
    assert np.array_equal(rows[0].cpu().numpy(), exp[0].cpu().numpy()[gi, :8])
    lib.rift_ile_destroy(h)


def test_posterior_event_times_of_time_marginalised_draws(lib, cuda, p_small):
    """Time-marginalised run: each slot's event time is a valid inversion of the oracle's
    conditional at that slot's draw (with the same uniform), nearly always the same grid time, and
    lnL at that time matches the oracle."""
    n, H = 20000, 400
    kw = dict(seed=64, n_per_round=n, max_evals=n, strata=(4, 2, 1), time_marg=1)
    h = lib.rift_ile_create(p_small)
    rows, idx, res = lib.rift_ile_posterior(h, H, **kw)
    g = rows[0].cpu().numpy().astype(np.float64)
    u = PO.posterior_uniforms(64, 0, H)
    fs = float(p_small["fs"])
    same = 0
    want = np.empty(H)
    for hh in range(H):
        ra, dec, t, psi, phi, incl, dist, l = g[hh]
        j = int(round((t - p_small["t_lo"]) * fs - 0.5))
        assert abs(t - (p_small["t_lo"] + (j + 0.5) / fs)) < 1e-7
        jo, to, lo_, cdf = PO.time_draw(p_small, ra, dec, psi, phi, incl, dist, u[hh])
        below = cdf[j - 1] if j > 0 else 0.0
        assert below - 4e-3 <= u[hh] <= cdf[j] + 4e-3, (hh, j, jo)
        same += int(j == jo)
        want[hh] = L.lnL_factorised(p_small, ra, dec, t, psi, phi, incl, dist)[0]
    assert same >= 0.95 * H
    cols = {k: g[:, c] for c, k in enumerate(("ra", "dec", "t", "psi", "phi", "incl", "dist"))}
    assert np.all(np.abs(g[:, 7] - want) <= _tol(p_small, cols)), np.max(np.abs(g[:, 7] - want))
    lib.rift_ile_destroy(h)


def test_batch_posterior_equals_single_point_runs(lib, cuda):
    """A batch's posterior rows are those of single-point runs of each point with the same Philox
    point word, although the points stop at different rounds."""
    specs = [W.cfg_small() for _ in range(3)]
    pts = [W.make_point(s, 70 + i) for i, s in enumerate(specs)]
    kw = dict(seed=65, n_per_round=8192, max_evals=8192 * 6, n_eff_target=1.6, proposal="adaptive", n_bins=32,
              strata=(2, 2, 2))
    hb = lib.rift_ile_batch_create(pts)
    rb, ib, resb = lib.rift_ile_posterior(hb, 500, **kw)
    for p, pt in enumerate(pts):
        h1 = lib.rift_ile_create(pt)
        r1, i1, res1 = lib.rift_ile_posterior(h1, 500, point_id=p, **kw)
        assert res1[0]["rounds"] == resb[p]["rounds"]
        assert np.array_equal(i1[0].cpu().numpy(), ib[p].cpu().numpy())
        assert np.array_equal(r1[0].cpu().numpy(), rb[p].cpu().numpy(), equal_nan=True)
        lib.rift_ile_destroy(h1)
    lib.rift_ile_destroy(hb)


def test_posterior_rejects_bad_arguments(lib, cuda, p_small):
    h = lib.rift_ile_create(p_small)
    with pytest.raises(lib.RiftError):
        lib.rift_ile_posterior(h, 0, seed=1, n_per_round=1000, max_evals=1000)
    lib.rift_ile_destroy(h)


def _lnl_array(lib, h, rows, tmarg=False):
    """lnL of exported parameter rows by the array kernels (an independent device path)."""
    import torch
    d = {k: torch.as_tensor(np.ascontiguousarray(rows[:, c]), device="cuda")
         for c, k in enumerate(("ra", "dec", "t", "psi", "phi", "incl", "dist"))}
    if tmarg:
        out = lib.rift_ile_lnL_tmarg(h, d["ra"], d["dec"], d["psi"], d["phi"], d["incl"], d["dist"])
    else:
        out = lib.rift_ile_lnL(h, d["ra"], d["dec"], d["t"], d["psi"], d["phi"], d["incl"], d["dist"])
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tmarg", [0, 1])
def test_learned_proposal_rows_agree_with_the_array_kernels(lib, cuda, p_small, tmarg):
    """Rows re-drawn from the learned proposal: their lnL column is what the array kernels give at
    the exported parameters (the exported angles are the sampler's, rounded to float32)."""
    import test_mdn_gpu as M
    h = lib.rift_ile_create(p_small)
    lib.rift_ile_set_proposal_head(h, M._head(11, p_small)[None])
    n = 20000
    rows, counts, _ = lib.rift_ile_samples(h, n, seed=66, n_per_round=n, max_evals=n, proposal="learned",
                                          time_marg=tmarg)
    g = rows[0].cpu().numpy()
    assert counts == [n] and np.all(np.isfinite(g[:, [0, 1, 3, 4, 5, 6, 7, 8]]))
    assert np.all(np.isnan(g[:, 2])) == bool(tmarg)
    want = _lnl_array(lib, h, g.astype(np.float32), bool(tmarg))
    cols = {k: g[:, c].astype(np.float64) for c, k in enumerate(("ra", "dec", "t", "psi", "phi", "incl", "dist"))}
    if tmarg:
        cols["t"] = np.zeros(n)
    # float32 parameters move lnL by up to ~|d lnL / d theta| * ulp: a wider bar than the parity one
    assert np.all(np.abs(g[:, 7] - want) <= 10 * _tol(p_small, cols)), np.max(np.abs(g[:, 7] - want))
    lib.rift_ile_destroy(h)


def test_batch_export_counts_follow_each_points_last_round(lib, cuda):
    """Points stopping at different rounds: each exports the draws of its own last round."""
    pts = [W.make_point(W.cfg_small(), 80 + i) for i in range(3)]
    n = 8192
    kw = dict(seed=67, n_per_round=n, max_evals=n * 6 - 100, n_eff_target=1.6, proposal="adaptive", n_bins=32,
              strata=(2, 2, 2))
    hb = lib.rift_ile_batch_create(pts)
    rows, counts, res = lib.rift_ile_samples(hb, n, **kw)
    for p in range(3):
        want = n if res[p]["n_evals"] % n == 0 else res[p]["n_evals"] % n
        assert counts[p] == want, (p, counts[p], res[p])
        g = rows[p].cpu().numpy()
        assert np.all(np.isfinite(g[:counts[p], 7])) and np.all(np.isnan(g[counts[p]:]))
    lib.rift_ile_destroy(hb)


def test_posterior_slot_counts_and_rejections(lib, cuda, p_small):
    h = lib.rift_ile_create(p_small)
    kw = dict(seed=68, n_per_round=1000, max_evals=1000)
    rows, idx, _ = lib.rift_ile_posterior(h, 1, **kw)
    assert 0 <= int(idx[0, 0]) < 1000
    rows, idx, _ = lib.rift_ile_posterior(h, 5000, **kw)       # more slots than draws
    gi = idx[0].cpu().numpy()
    assert np.all((gi >= 0) & (gi < 1000)) and np.all(np.diff(gi) >= 0)
    with pytest.raises(lib.RiftError):
        lib.rift_ile_marginalize(h, want_tables=True, **kw)   # tables_out needs the adaptive proposal
    lib.rift_ile_destroy(h)
