"""GPU parity of the mode inner products of Eq. (QUV) against the FP64 direct-sum oracle.

Each element is compared within 3e-6 of its condition scale, the sum of the absolute values of
its terms (2 df sum |h| |d| w for Q, 2 df sum |h_a| |h_b| w for U and V): FP32 terms summed in
blocks of 32 into double-float totals stay well inside that."""
from __future__ import annotations

import numpy as np
import pytest

import workload as W
from oracle import likelihood as L
from oracle import quv as QUV

pytestmark = pytest.mark.gpu


def _scales(pt):
    w, h, d, df = pt["weight"], np.abs(pt["hlm"]), np.abs(pt["data"]), pt["df"]
    sq = 2 * df * np.einsum("mf,kf,kf->km", h, d, w)          # (K, M)
    su = 2 * df * np.einsum("af,bf,kf->kab", h, h, w)
    sv = 2 * df * np.einsum("af,bf,kf->kab", h[:, pt["mirror"]], h, w)
    return sq, su, sv


@pytest.mark.parametrize("which", ["small", "full"])
def test_quv_matches_oracle(lib, cuda, which):
    pt = W.make_point(W.cfg_small() if which == "small" else W.cfg_full(), 13)
    Q, U, V = lib.rift_quv(pt)
    Qo, Uo, Vo = QUV.quv(pt)
    sq, su, sv = _scales(pt)
    assert np.all(np.abs(Q - Qo) <= 3e-6 * sq[:, :, None]), float(np.max(np.abs(Q - Qo) / sq[:, :, None]))
    for name, A, B, S in (("U", U, Uo, su), ("V", V, Vo, sv)):
        bad = np.argwhere(~(np.abs(A - B) <= 3e-6 * S))   # NaN counts as a failure
        assert bad.size == 0, (name, bad[:4].tolist(), [(A[tuple(i)], B[tuple(i)], S[tuple(i)]) for i in bad[:4]])


def test_handle_from_frequency_domain_inputs(lib, cuda):
    """rift_ile_create_fd (Q, U, V formed on the device) gives the per-sample likelihood of the
    oracle's Q, U, V within the per-sample tolerance."""
    import torch
    pt = W.make_point(W.cfg_small(), 14)
    Qo, Uo, Vo = QUV.quv(pt)
    ref = dict(pt, Q=Qo, U=Uo, V=Vo)
    h = lib.rift_ile_create_fd(pt)
    r = np.random.default_rng(3)
    n = 4000
    th = dict(ra=r.uniform(0, 2 * np.pi, n), dec=np.arcsin(r.uniform(-1, 1, n)), t=r.uniform(pt["t_lo"], pt["t_hi"], n),
              psi=r.uniform(0, np.pi, n), phi=r.uniform(0, 2 * np.pi, n), incl=np.arccos(r.uniform(-1, 1, n)),
              dist=np.cbrt(r.uniform(1, 1000.0 ** 3, n)))
    th = {k: v.astype(np.float32) for k, v in th.items()}
    d = {k: torch.as_tensor(v, device="cuda") for k, v in th.items()}
    got = lib.rift_ile_lnL(h, d["ra"], d["dec"], d["t"], d["psi"], d["phi"], d["incl"], d["dist"]).cpu().numpy()
    th64 = {k: v.astype(np.float64) for k, v in th.items()}
    want = L.lnL_factorised(ref, **th64)
    z = dict(ref, Q=np.zeros_like(Qo))
    tol = 1e-3 * np.maximum(1.0, -2.0 * L.lnL_factorised(z, **th64) / 900.0)
    assert np.all(np.abs(got - want) <= tol), float(np.max(np.abs(got - want) / tol))
    lib.rift_ile_destroy(h)


def test_inconsistent_grids_are_refused(lib, cuda):
    pt = W.make_point(W.cfg_small(), 15)
    bad = dict(pt, fs=float(pt["fs"]) * 1.0001)
    with pytest.raises(lib.RiftError) as e:
        lib.rift_quv(bad)
    assert e.value.status == 1


def test_non_finite_inputs_are_refused(lib, cuda):
    pt = W.make_point(W.cfg_small(), 16)
    band = np.flatnonzero(pt["weight"][0])
    data = pt["data"].copy()
    data[0, band[10]] = np.nan
    with pytest.raises(lib.RiftError) as e:
        lib.rift_quv(dict(pt, data=data))
    assert e.value.status == 1
