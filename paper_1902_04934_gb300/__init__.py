"""Python binding of the GB300 extrinsic-likelihood library (argument marshalling only).

Every computation runs in the CUDA library built from ``csrc/`` (``_lib/librift_ile.so``);
this module only converts Python/numpy/torch arguments to the C ABI declared in
``include/rift_ile.h`` and back.  Importing it fails loudly when the library is
missing: there is no CPU fallback.

Functions carry the names of the C entry points:

* rift_ile_create(point) / rift_ile_batch_create(points) -> handle
* rift_ile_lnL(h, ra, dec, t, psi, phi, incl, dist, out=None)   (CUDA tensors)
* rift_ile_lnL_host(h, ...)                                       (numpy arrays)
* rift_ile_marginalize(h, **opts) -> dict
* rift_ile_batch_marginalize(h, **opts) -> list of dicts
* rift_ile_draw(h, round, n, tables=None, **opts) -> (theta, lpq, bins)
* rift_ile_destroy(h)
"""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
_LIBPATH = _PKG / "_lib" / "librift_ile.so"

STATUS = {0: "RIFT_OK", 1: "RIFT_EINVAL", 2: "RIFT_EWINDOW", 3: "RIFT_ENOMEM", 4: "RIFT_ECUDA",
          5: "RIFT_ETIMEOUT", 6: "RIFT_ENONFINITE", 7: "RIFT_ENOTCONVERGED", 8: "RIFT_EUNSUPPORTED"}
PROPOSAL = {"prior": 0, "adaptive": 1, "learned": 2}


class RiftError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [("n_det", C.c_int), ("det_tensor", C.c_void_p), ("det_pos", C.c_void_p),
                ("n_modes", C.c_int), ("lm", C.c_void_p), ("n_t", C.c_int), ("Q", C.c_void_p),
                ("q_t0_gps", C.c_void_p), ("fs", C.c_double), ("U", C.c_void_p), ("V", C.c_void_p),
                ("t_ref_gps", C.c_double), ("d_ref_mpc", C.c_double), ("t_lo", C.c_double),
                ("t_hi", C.c_double), ("interp", C.c_int), ("cuda_stream", C.c_void_p)]


class FdDesc(C.Structure):
    _fields_ = [("n_det", C.c_int), ("det_tensor", C.c_void_p), ("det_pos", C.c_void_p), ("n_modes", C.c_int),
                ("lm", C.c_void_p), ("n_f", C.c_int), ("nu", C.c_void_p), ("df", C.c_double), ("hlm", C.c_void_p),
                ("data", C.c_void_p), ("weight", C.c_void_p), ("mirror", C.c_void_p), ("n_t", C.c_int),
                ("q_t0_gps", C.c_void_p), ("fs", C.c_double), ("t_ref_gps", C.c_double), ("d_ref_mpc", C.c_double),
                ("t_lo", C.c_double), ("t_hi", C.c_double), ("interp", C.c_int), ("cuda_stream", C.c_void_p)]


class McOpts(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("point_id", C.c_uint32), ("n_per_round", C.c_uint32),
                ("max_evals", C.c_uint64), ("n_eff_target", C.c_double), ("d_lo", C.c_double),
                ("d_hi", C.c_double), ("proposal", C.c_int), ("n_bins", C.c_int), ("beta", C.c_double),
                ("floor_eps", C.c_double), ("adapt_rounds", C.c_int), ("tables", C.c_void_p),
                ("mdn", C.c_void_p), ("dbg_ell", C.c_void_p), ("dbg_tables", C.c_void_p),
                ("max_rounds", C.c_int), ("timing", C.c_int), ("strata", C.c_int * 3),
                ("resume", C.c_void_p), ("save", C.c_void_p), ("time_marg", C.c_int),
                ("tables_per_point", C.c_int), ("tables_out", C.c_void_p), ("fallback_neff", C.c_double),
                ("refine", C.c_int)]


MC_STATE_BYTES = 8192   # RIFT_MC_STATE_BYTES
REFINE_CAP = 64         # RIFT_REFINE_CAP


class McResult(C.Structure):
    _fields_ = [("lnL_marg", C.c_double), ("n_eff", C.c_double), ("n_eff_kish", C.c_double),
                ("sigma", C.c_double), ("n_evals", C.c_uint64), ("rounds", C.c_int), ("status", C.c_int),
                ("acc_max", C.c_double), ("acc_s1", C.c_double), ("acc_s2", C.c_double),
                ("kernel_ms", C.c_double), ("kernel_launches", C.c_int), ("strata", C.c_int * 3),
                ("fallback_round", C.c_int), ("n_refined", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["strata"] = tuple(self.strata)
        return d


class Tune(C.Structure):
    _fields_ = [("cell_samples", C.c_int), ("smem_split", C.c_int), ("ms", C.c_double)]


def _load():
    if not _LIBPATH.exists():
        raise ImportError(f"CUDA library {_LIBPATH} is not built; run __graft_entry__.build() "
                          "(paper_1902_04934_gb300._build.build()) first")
    lib = C.CDLL(str(_LIBPATH))
    P, S, I, U32, U64, D = C.c_void_p, C.c_size_t, C.c_int, C.c_uint32, C.c_uint64, C.c_double
    sig = {
        "rift_ile_create": (I, [C.POINTER(Desc), C.POINTER(P)]),
        "rift_ile_batch_create": (I, [C.POINTER(Desc), I, C.POINTER(P)]),
        "rift_ile_destroy": (None, [P]),
        "rift_status_str": (C.c_char_p, [I]),
        "rift_ile_last_error": (C.c_char_p, [P]),
        "rift_ile_n_points": (I, [P]),
        "rift_ile_forms": (C.c_uint, [P, I]),
        "rift_ile_lnL": (I, [P, S] + [P] * 8),
        "rift_ile_lnL_host": (I, [P, S] + [P] * 8),
        "rift_ile_lnL_tmarg": (I, [P, S] + [P] * 7),
        "rift_ile_check": (I, [P]),
        "rift_quv": (I, [P, P, P, P]),
        "rift_quv_last_error": (C.c_char_p, []),
        "rift_quv_kernel_ms": (None, [P]),
        "rift_mdn_forward_ms": (D, []),
        "rift_source_frame": (I, [I, P, P, I, P, D, D, S, P, P, P]),
        "rift_ile_create_fd": (I, [P, C.POINTER(P)]),
        "rift_ile_marginalize": (I, [P, C.POINTER(McOpts), C.POINTER(McResult)]),
        "rift_ile_batch_marginalize": (I, [P, C.POINTER(McOpts), C.POINTER(McResult)]),
        "rift_ile_marginalize_static": (I, [P, C.POINTER(McOpts), C.POINTER(McResult)]),
        "rift_ile_draw": (I, [P, C.POINTER(McOpts), U32, P, S, P, P, P]),
        "rift_mdn_create": (I, [U64, C.POINTER(P)]),
        "rift_mdn_destroy": (None, [P]),
        "rift_mdn_last_error": (C.c_char_p, [P]),
        "rift_mdn_set_params": (I, [P, P]),
        "rift_mdn_get_params": (I, [P, P, I]),
        "rift_mdn_forward": (I, [P, I, P, P]),
        "rift_mdn_loss_grad": (I, [P, I, P, P, P, I, P, C.POINTER(D), P]),
        "rift_mdn_train": (I, [P, I, P, P, P, I, P, I, I, D, P]),
        "rift_ile_batch_summary": (I, [P, P]),
        "rift_ile_set_proposal_head": (I, [P, P]),
        "rift_ile_boxes": (I, [P, D, D, P]),
        "rift_ile_batch_harvest": (I, [P, C.POINTER(McOpts), I, D, P, C.POINTER(McResult)]),
        "rift_ile_samples": (I, [P, C.POINTER(McOpts), S, P, C.POINTER(U64), C.POINTER(McResult)]),
        "rift_release_cached_memory": (None, []),
        "rift_cache_counters": (None, [P]),
        "rift_ile_posterior": (I, [P, C.POINTER(McOpts), I, P, P, C.POINTER(McResult)]),
        "rift_ile_get_tune": (I, [P, C.POINTER(Tune)]),
        "rift_ile_set_tune": (I, [P, C.POINTER(Tune)]),
        "rift_ile_autotune": (I, [P, C.POINTER(McOpts), I, C.POINTER(Tune)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()
LIB_PATH = str(_LIBPATH)


class Handle:
    """Owns a rift_ile* and keeps the host arrays of its descriptor alive during create."""

    def __init__(self, ptr, n_points):
        self.ptr = C.c_void_p(ptr)
        self.n_points = n_points

    def __del__(self):
        try:
            rift_ile_destroy(self)
        except Exception:
            pass


def _check(h, status):
    if status not in (0,):
        msg = _lib.rift_ile_last_error(h.ptr if h is not None else None)
        raise RiftError(status, (msg or b"").decode())


def _f64(a):
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _desc(pt, interp=3, stream=None, keep=None):
    K = int(np.asarray(pt["det_tensor"]).shape[0])
    lm = np.ascontiguousarray(np.asarray(pt["lm"], dtype=np.int32).reshape(-1, 2))
    Q = np.asarray(pt["Q"])
    M, T = Q.shape[1], Q.shape[2]
    arrs = dict(det_tensor=_f64(pt["det_tensor"]), det_pos=_f64(pt["det_pos"]), lm=lm,
                Q=np.ascontiguousarray(Q, dtype=np.complex128).view(np.float64),
                q_t0_gps=_f64(pt["q_t0_gps"]),
                U=np.ascontiguousarray(pt["U"], dtype=np.complex128).view(np.float64),
                V=np.ascontiguousarray(pt["V"], dtype=np.complex128).view(np.float64))
    if keep is not None:
        keep.append(arrs)
    d = Desc()
    d.n_det = K
    d.det_tensor = arrs["det_tensor"].ctypes.data
    d.det_pos = arrs["det_pos"].ctypes.data
    d.n_modes = M
    d.lm = arrs["lm"].ctypes.data
    d.n_t = T
    d.Q = arrs["Q"].ctypes.data
    d.q_t0_gps = arrs["q_t0_gps"].ctypes.data
    d.fs = float(pt["fs"])
    d.U = arrs["U"].ctypes.data
    d.V = arrs["V"].ctypes.data
    d.t_ref_gps = float(pt["t_ref_gps"])
    d.d_ref_mpc = float(pt["d_ref_mpc"])
    d.t_lo = float(pt["t_lo"])
    d.t_hi = float(pt["t_hi"])
    d.interp = int(interp)
    d.cuda_stream = stream
    return d


def _fd_desc(pt, interp=3, stream=None, keep=None):
    """Frequency-domain descriptor of a point dict with freqs, df, hlm, data, weight, mirror, n_t (nu,
    the integer bins of the grid with freqs = nu df, is taken from the dict when given)."""
    K = int(np.asarray(pt["det_tensor"]).shape[0])
    hlm = np.ascontiguousarray(np.asarray(pt["hlm"], dtype=np.complex128))
    M, nf = hlm.shape
    df = float(pt["df"])
    arrs = dict(det_tensor=_f64(pt["det_tensor"]), det_pos=_f64(pt["det_pos"]),
                lm=np.ascontiguousarray(np.asarray(pt["lm"], dtype=np.int32).reshape(-1, 2)),
                nu=np.ascontiguousarray(pt["nu"], dtype=np.int32) if "nu" in pt
                else np.ascontiguousarray(np.rint(np.asarray(pt["freqs"]) / df).astype(np.int32)),
                hlm=hlm.view(np.float64),
                data=np.ascontiguousarray(np.asarray(pt["data"], dtype=np.complex128)).view(np.float64),
                weight=_f64(pt["weight"]), mirror=np.ascontiguousarray(np.asarray(pt["mirror"], dtype=np.int32)),
                q_t0_gps=_f64(pt["q_t0_gps"]))
    if keep is not None:
        keep.append(arrs)
    d = FdDesc()
    d.n_det, d.n_modes, d.n_f, d.n_t = K, M, nf, int(pt["n_t"])
    for key in ("det_tensor", "det_pos", "lm", "nu", "hlm", "data", "weight", "mirror", "q_t0_gps"):
        setattr(d, key, arrs[key].ctypes.data)
    d.df, d.fs = df, float(pt["fs"])
    d.t_ref_gps, d.d_ref_mpc = float(pt["t_ref_gps"]), float(pt["d_ref_mpc"])
    d.t_lo, d.t_hi = float(pt["t_lo"]), float(pt["t_hi"])
    d.interp = int(interp)
    d.cuda_stream = stream
    return d


def rift_quv(pt, stream=None):
    """Eq. (QUV) on the device from the point's frequency-domain arrays: (Q, U, V) complex128."""
    keep = []
    d = _fd_desc(pt, 3, stream, keep)
    K, M, T = d.n_det, d.n_modes, d.n_t
    Q = np.empty((K, M, T), dtype=np.complex128)
    U = np.empty((K, M, M), dtype=np.complex128)
    V = np.empty((K, M, M), dtype=np.complex128)
    st = _lib.rift_quv(C.byref(d), Q.ctypes.data, U.ctypes.data, V.ctypes.data)
    if st != 0:
        raise RiftError(st, (_lib.rift_quv_last_error() or b"").decode())
    return Q, U, V


def rift_source_frame(det_tensor, det_pos, lm, t_ref_gps, d_ref_mpc, src):
    """Detector-frame coefficients and arrival times of sources: src (n, 7) rows (ra, dec, t, psi,
    phi, incl, D) -> coef (n, K, M) complex128 = (D_ref/D) conj(F_k) Y_lm, tk (n, K) = t + delay_k."""
    tens = np.ascontiguousarray(det_tensor, dtype=np.float64)
    pos = np.ascontiguousarray(det_pos, dtype=np.float64)
    modes = np.ascontiguousarray(np.asarray(lm).reshape(-1, 2), dtype=np.int32)
    s = np.ascontiguousarray(np.asarray(src, dtype=np.float64).reshape(-1, 7))
    n, K, M = s.shape[0], tens.shape[0], modes.shape[0]
    coef = np.empty((n, K, M), dtype=np.complex128)
    tk = np.empty((n, K), dtype=np.float64)
    st = _lib.rift_source_frame(K, tens.ctypes.data, pos.ctypes.data, M, modes.ctypes.data, float(t_ref_gps),
                                float(d_ref_mpc), n, s.ctypes.data, coef.ctypes.data, tk.ctypes.data)
    if st != 0:
        raise RiftError(st, "rift_source_frame failed")
    return coef, tk


def rift_quv_kernel_ms():
    """Device time (ms) of the Q kernel and of the U/V kernel of this thread's last rift_quv call."""
    out = (C.c_double * 2)()
    _lib.rift_quv_kernel_ms(out)
    return float(out[0]), float(out[1])


def rift_ile_create_fd(pt, interp=3, stream=None):
    """A handle whose Q, U, V are formed on the device from frequency-domain inputs."""
    keep = []
    d = _fd_desc(pt, interp, stream, keep)
    out = C.c_void_p()
    st = _lib.rift_ile_create_fd(C.byref(d), C.byref(out))
    if st != 0:
        raise RiftError(st, (_lib.rift_quv_last_error() or b"rift_ile_create_fd failed").decode())
    return Handle(out.value, 1)


def rift_ile_create(pt, interp=3, stream=None):
    keep = []
    d = _desc(pt, interp, stream, keep)
    out = C.c_void_p()
    st = _lib.rift_ile_create(C.byref(d), C.byref(out))
    if st != 0:
        raise RiftError(st, "rift_ile_create failed (see stderr)")
    return Handle(out.value, 1)


def rift_ile_batch_create(points, interp=3, stream=None):
    keep = []
    arr = (Desc * len(points))(*[_desc(p, interp, stream, keep) for p in points])
    out = C.c_void_p()
    st = _lib.rift_ile_batch_create(arr, len(points), C.byref(out))
    if st != 0:
        raise RiftError(st, "rift_ile_batch_create failed (see stderr)")
    return Handle(out.value, len(points))


def rift_ile_destroy(h):
    if h is not None and h.ptr:
        _lib.rift_ile_destroy(h.ptr)
        h.ptr = C.c_void_p(None)


FORM_GROUPED, FORM_SPARSE, FORM_MIRROR, FORM_QHALF = 1, 2, 4, 8


def rift_ile_forms(h, point=0):
    """Bits of the forms the kernels take for `point` (FORM_* above; 0 for a bad index)."""
    return int(_lib.rift_ile_forms(h.ptr, int(point)))


def _dptr(t, n):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    if t.numel() != n:
        raise ValueError("sample arrays differ in length")
    return t.data_ptr()


def rift_ile_lnL(h, ra, dec, t, psi, phi, incl, dist, out=None):
    """Device-buffer call: CUDA float32 tensors in, CUDA float32 tensor out (asynchronous)."""
    import torch
    n = ra.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=ra.device)
    ptrs = [_dptr(a, n) for a in (ra, dec, t, psi, phi, incl, dist, out)]
    _check(h, _lib.rift_ile_lnL(h.ptr, n, *ptrs))
    return out


def rift_ile_lnL_tmarg(h, ra, dec, psi, phi, incl, dist, out=None):
    """Time-marginalised lnL of device draws (CUDA float32 tensors; asynchronous), see the C header."""
    import torch
    n = ra.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=ra.device)
    ptrs = [_dptr(a, n) for a in (ra, dec, psi, phi, incl, dist, out)]
    _check(h, _lib.rift_ile_lnL_tmarg(h.ptr, n, *ptrs))
    return out


def rift_ile_lnL_host(h, ra, dec, t, psi, phi, incl, dist):
    """Host-buffer call: numpy float32 in, numpy float32 out (copies inside the library)."""
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (ra, dec, t, psi, phi, incl, dist)]
    n = arrs[0].shape[0]
    out = np.empty(n, dtype=np.float32)
    _check(h, _lib.rift_ile_lnL_host(h.ptr, n, *[a.ctypes.data for a in arrs], out.ctypes.data))
    return out


def rift_ile_check(h):
    _check(h, _lib.rift_ile_check(h.ptr))


def _opts(seed=1, point_id=0, n_per_round=100000, max_evals=100000, n_eff_target=1e300, d_lo=1.0,
          d_hi=1000.0, proposal="prior", n_bins=100, beta=0.3, floor_eps=0.1, adapt_rounds=-1,
          tables=None, mdn=None, dbg_ell=None, dbg_tables=None, max_rounds=0, timing=0, strata=(0, 0, 0),
          resume=None, save=None, time_marg=0, tables_out=None, fallback_neff=0.0, refine=0, keep=None):
    o = McOpts()
    o.seed = int(seed)
    o.point_id = int(point_id)
    o.n_per_round = int(n_per_round)
    o.max_evals = int(max_evals)
    o.n_eff_target = float(n_eff_target)
    o.d_lo = float(d_lo)
    o.d_hi = float(d_hi)
    o.proposal = PROPOSAL[proposal] if isinstance(proposal, str) else int(proposal)
    o.n_bins = int(n_bins)
    o.beta = float(beta)
    o.floor_eps = float(floor_eps)
    o.adapt_rounds = int(adapt_rounds)
    if tables is not None:
        tb = np.ascontiguousarray(tables, dtype=np.float32)
        if keep is not None:
            keep.append(tb)
        o.tables = tb.ctypes.data
        o.tables_per_point = 1 if tb.ndim == 3 else 0   # [n_points][3][n_bins+1]: one set per point
    o.mdn = mdn.ptr.value if mdn is not None else None
    o.dbg_ell = dbg_ell.data_ptr() if dbg_ell is not None else None
    o.dbg_tables = dbg_tables.data_ptr() if dbg_tables is not None else None
    o.max_rounds = int(max_rounds)
    o.timing = int(timing)
    for d in range(3):
        o.strata[d] = int(strata[d])
    o.time_marg = int(time_marg)
    o.fallback_neff = float(fallback_neff)
    o.refine = int(refine)
    if resume is not None:
        rb = C.create_string_buffer(bytes(resume), MC_STATE_BYTES)
        keep.append(rb)
        o.resume = C.cast(rb, C.c_void_p)
    if save is not None:
        keep.append(save)
        o.save = C.cast(save, C.c_void_p)
    if tables_out is not None:
        keep.append(tables_out)
        o.tables_out = tables_out.ctypes.data
    return o


def _tables_out(h, want, kw):
    """Host buffer for each point's proposal tables at return (adaptive runs), or None."""
    if not want:
        return None
    return np.zeros((h.n_points, 3, int(kw.get("n_bins", 100)) + 1), dtype=np.float32)


def rift_ile_marginalize(h, save=False, want_tables=False, **kw):
    """One point's marginalisation (see the C header).  resume=<bytes> continues a run whose
    state an earlier call returned with save=True (the dict's "state" entry); want_tables=True
    returns the adapted proposal as "tables" ([3][n_bins+1], to warm-start another point)."""
    keep = []
    buf = C.create_string_buffer(MC_STATE_BYTES) if save else None
    tout = _tables_out(h, want_tables, kw)
    o = _opts(keep=keep, save=buf, tables_out=tout, **kw)
    r = McResult()
    st = _lib.rift_ile_marginalize(h.ptr, C.byref(o), C.byref(r))
    if st not in (0, 7):
        _check(h, st)
    d = r.as_dict()
    if save:
        d["state"] = buf.raw
    if tout is not None:
        d["tables"] = tout[0]
    return d


def rift_ile_marginalize_static(h, **kw):
    """rift_ile_marginalize without device allocation (scratch in a static device array);
    for callers that may not allocate device memory at that point.  See the C header."""
    keep = []
    o = _opts(keep=keep, **kw)
    r = McResult()
    st = _lib.rift_ile_marginalize_static(h.ptr, C.byref(o), C.byref(r))
    if st not in (0, 7):
        _check(h, st)
    return r.as_dict()


def rift_ile_batch_marginalize(h, want_tables=False, **kw):
    """Every point of a batch handle; tables=<[n_points][3][n_bins+1]> starts each point from its
    own proposal, want_tables=True returns each point's adapted proposal as "tables"."""
    keep = []
    tout = _tables_out(h, want_tables, kw)
    o = _opts(keep=keep, tables_out=tout, **kw)
    res = (McResult * h.n_points)()
    st = _lib.rift_ile_batch_marginalize(h.ptr, C.byref(o), res)
    if st not in (0, 7):
        _check(h, st)
    out = [r.as_dict() for r in res]
    if tout is not None:
        for p, d in enumerate(out):
            d["tables"] = tout[p]
    return out


MDN_PARAMS = 105048
MDN_SUMMARY = 64
MDN_HEAD = 88


class Mdn:
    """Owns a rift_mdn*."""

    def __init__(self, ptr):
        self.ptr = C.c_void_p(ptr)

    def __del__(self):
        try:
            rift_mdn_destroy(self)
        except Exception:
            pass


def _mcheck(m, status):
    if status != 0:
        raise RiftError(status, (_lib.rift_mdn_last_error(m.ptr) or b"").decode())


def rift_mdn_create(seed=0):
    out = C.c_void_p()
    st = _lib.rift_mdn_create(int(seed), C.byref(out))
    if st != 0:
        raise RiftError(st, "rift_mdn_create failed")
    return Mdn(out.value)


def rift_mdn_destroy(m):
    if m is not None and m.ptr:
        _lib.rift_mdn_destroy(m.ptr)
        m.ptr = C.c_void_p(None)


def rift_mdn_set_params(m, params):
    a = np.ascontiguousarray(params, dtype=np.float32)
    assert a.size == MDN_PARAMS
    _mcheck(m, _lib.rift_mdn_set_params(m.ptr, a.ctypes.data))


def rift_mdn_get_params(m, which=0):
    a = np.empty(MDN_PARAMS, dtype=np.float32)
    _mcheck(m, _lib.rift_mdn_get_params(m.ptr, a.ctypes.data, int(which)))
    return a


def rift_mdn_forward(m, summ):
    """summ: CUDA float32 tensor (n, 64) -> head (n, 88)."""
    import torch
    n = summ.shape[0]
    out = torch.empty((n, MDN_HEAD), dtype=torch.float32, device=summ.device)
    _mcheck(m, _lib.rift_mdn_forward(m.ptr, n, summ.data_ptr(), out.data_ptr()))
    return out


def rift_mdn_forward_ms():
    """Device time (ms) of the kernel of this thread's last rift_mdn_forward call."""
    return float(_lib.rift_mdn_forward_ms())


def rift_mdn_loss_grad(m, summ, theta, w, box):
    """Device tensors summ (n,64), theta (n,H,5), w (n,H), box (n,2,5) -> (loss, grad numpy)."""
    n, H = theta.shape[0], theta.shape[1]
    loss = C.c_double()
    g = np.empty(MDN_PARAMS, dtype=np.float32)
    _mcheck(m, _lib.rift_mdn_loss_grad(m.ptr, n, summ.data_ptr(), theta.data_ptr(), w.data_ptr(), H,
                                       box.data_ptr(), C.byref(loss), g.ctypes.data))
    return loss.value, g


def rift_mdn_train(m, summ, theta, w, box, steps, batch, lr):
    n, H = theta.shape[0], theta.shape[1]
    losses = np.empty(max(1, steps), dtype=np.float64)
    _mcheck(m, _lib.rift_mdn_train(m.ptr, n, summ.data_ptr(), theta.data_ptr(), w.data_ptr(), H, box.data_ptr(),
                                   int(steps), int(batch), float(lr), losses.ctypes.data))
    return losses[:steps]


def rift_ile_batch_summary(h):
    import torch
    out = torch.empty((h.n_points, MDN_SUMMARY), dtype=torch.float32, device="cuda")
    _check(h, _lib.rift_ile_batch_summary(h.ptr, out.data_ptr()))
    return out


def rift_ile_set_proposal_head(h, head):
    a = np.ascontiguousarray(head, dtype=np.float32).reshape(h.n_points, MDN_HEAD)
    _check(h, _lib.rift_ile_set_proposal_head(h.ptr, a.ctypes.data))


def rift_ile_boxes(h, d_lo=1.0, d_hi=1000.0):
    out = np.empty((h.n_points, 2, 5), dtype=np.float32)
    _check(h, _lib.rift_ile_boxes(h.ptr, float(d_lo), float(d_hi), out.ctypes.data))
    return out


def rift_ile_batch_harvest(h, H, beta=0.5, **kw):
    """Run the batch and resample H samples per point from its last round -> (theta (np,H,5) CUDA, results)."""
    import torch
    keep = []
    o = _opts(keep=keep, **kw)
    theta = torch.empty((h.n_points, H, 5), dtype=torch.float32, device="cuda")
    res = (McResult * h.n_points)()
    st = _lib.rift_ile_batch_harvest(h.ptr, C.byref(o), int(H), float(beta), theta.data_ptr(), res)
    if st not in (0, 7):
        _check(h, st)
    return theta, [r.as_dict() for r in res]


SAMPLE_COLS = ("ra", "dec", "t", "psi", "phi", "incl", "dist", "lnL", "lnpq")
POSTERIOR_COLS = SAMPLE_COLS[:8]


def rift_ile_samples(h, cap, **kw):
    """Marginalise every point and export the draws of its last round with their weights ->
    (rows (np, cap, 9) CUDA float32 with columns SAMPLE_COLS, draws per point, results)."""
    import torch
    keep = []
    o = _opts(keep=keep, **kw)
    rows = torch.empty((h.n_points, int(cap), len(SAMPLE_COLS)), dtype=torch.float32, device="cuda")
    n = (C.c_uint64 * h.n_points)()
    res = (McResult * h.n_points)()
    st = _lib.rift_ile_samples(h.ptr, C.byref(o), int(cap), rows.data_ptr() if cap else None, n, res)
    if st not in (0, 7):
        _check(h, st)
    return rows, list(n), [r.as_dict() for r in res]


def rift_ile_posterior(h, H, **kw):
    """Marginalise every point and draw H equal-weight posterior samples from its last round ->
    (rows (np, H, 8) CUDA float32 with columns POSTERIOR_COLS, resampled draw (np, H) int32, results)."""
    import torch
    keep = []
    o = _opts(keep=keep, **kw)
    rows = torch.empty((h.n_points, int(H), len(POSTERIOR_COLS)), dtype=torch.float32, device="cuda")
    idx = torch.empty((h.n_points, int(H)), dtype=torch.int32, device="cuda")
    res = (McResult * h.n_points)()
    st = _lib.rift_ile_posterior(h.ptr, C.byref(o), int(H), rows.data_ptr(), idx.data_ptr(), res)
    if st not in (0, 7):
        _check(h, st)
    return rows, idx, [r.as_dict() for r in res]


def rift_release_cached_memory():
    """Give the device and pinned buffers cached from destroyed handles back to CUDA."""
    _lib.rift_release_cached_memory()


def rift_cache_counters():
    """Buffer-cache counters: (device requests, pinned host requests, cudaMalloc calls,
    cudaMallocHost calls) since the library was loaded."""
    out = (C.c_ulonglong * 4)()
    _lib.rift_cache_counters(out)
    return tuple(int(x) for x in out)


def rift_ile_get_tune(h):
    t = Tune()
    _check(h, _lib.rift_ile_get_tune(h.ptr, C.byref(t)))
    return dict(cell_samples=t.cell_samples, smem_split=t.smem_split, ms=t.ms)


def rift_ile_set_tune(h, cell_samples, smem_split):
    t = Tune(int(cell_samples), int(smem_split), 0.0)
    _check(h, _lib.rift_ile_set_tune(h.ptr, C.byref(t)))


def rift_ile_autotune(h, reps=2, **kw):
    """Time the candidate launch shapes on this workload, keep the fastest (see the C header)."""
    keep = []
    o = _opts(keep=keep, **kw)
    t = Tune()
    _check(h, _lib.rift_ile_autotune(h.ptr, C.byref(o), int(reps), C.byref(t)))
    return dict(cell_samples=t.cell_samples, smem_split=t.smem_split, ms=t.ms)


def autotune_cached(h, key, reps=2, **kw):
    """rift_ile_autotune with a JSON cache (next to the built library) keyed by `key`: a string
    naming the device and workload shape.  A cached choice is applied without re-timing."""
    import json
    path = _PKG / "_lib" / "tune_cache.json"
    try:
        cache = json.loads(path.read_text())
    except (OSError, ValueError):
        cache = {}
    c = cache.get(key)
    if isinstance(c, dict) and "cell_samples" in c and "smem_split" in c:
        rift_ile_set_tune(h, c["cell_samples"], c["smem_split"])
        return dict(c, cached=True)
    best = rift_ile_autotune(h, reps=reps, **kw)
    cache[key] = best
    try:
        path.write_text(json.dumps(cache, indent=1, sort_keys=True))
    except OSError:
        pass
    return dict(best, cached=False)


def rift_ile_draw(h, rnd, n, tables=None, **kw):
    """Samples of one round on the device: theta (7, n), ln p - ln q (n,), bins (3, n)."""
    import torch
    keep = []
    o = _opts(keep=keep, **kw)
    dev = torch.device("cuda")
    theta = torch.empty((7, n), dtype=torch.float32, device=dev)
    lpq = torch.empty(n, dtype=torch.float32, device=dev)
    bins = torch.empty((3, n), dtype=torch.int32, device=dev)
    tptr = None
    if tables is not None:
        tt = torch.as_tensor(np.asarray(tables, dtype=np.float32), device=dev).contiguous()
        keep.append(tt)
        tptr = tt.data_ptr()
    _check(h, _lib.rift_ile_draw(h.ptr, C.byref(o), int(rnd), tptr, n, theta.data_ptr(), lpq.data_ptr(),
                                 bins.data_ptr()))
    return theta, lpq, bins
