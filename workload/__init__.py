"""Seeded synthetic inputs shaped like the paper's ILE workloads.

The paper analyses zero-noise SEOBNRv4/TaylorT4 injections in two-detector
LIGO data (Sec. III.A, Table I, Table II); none of that data, nor the waveform
families, is available here.  This module builds stand-ins of the same shape:

* an analytic advanced-LIGO noise curve (Sathyaprakash & Schutz 2009 fit),
* chirp-like frequency-domain mode waveforms h_lm(f) with amplitude f^(-7/6)
  and a seeded post-Newtonian-style phase series,
* Gaussian noise, a signal built from detector-frame injection coefficients,
* the precomputed inner products Q_{k,lm}(tau), U_{k,lm,l'm'}, V_{k,lm,l'm'}
  of Eq. (QUV) on a uniform time grid (FFT), which are the inputs of the
  likelihood path (Sec. II.A, "Accelerated evaluation").

It holds no step of the likelihood or Monte Carlo method itself: no antenna
response, no time-of-flight formula, no spin-weighted harmonic.  The injected
signal is specified in the detector frame, d_k(t) = Re sum_lm c_{k,lm}
h_lm(t - t_k), so callers that want a physical injection pass c and t_k in
(the tests compute them with the oracle); otherwise c and t_k are drawn from a
seeded distribution.  Both the CUDA path and the oracle consume what this
module returns; neither is imported here.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

C_LIGHT = 299792458.0          # m/s
MSUN_S = 4.925490947641267e-6  # G Msun / c^3 in seconds
T_REF_GPS = 1187008882.4       # synthetic trigger epoch (GPS s), after the 2017 leap second

# ---------------------------------------------------------------------------
# Detector geometry (inputs).  Approximate geodetic vertex and arm azimuths
# (degrees clockwise from local north, arms in the local horizontal plane).
# Geometry is shared input data: it sets realism, not parity.
# ---------------------------------------------------------------------------
_SITES = {
    "H1": (46.45514, -119.40766, 142.554, 324.0006, 234.0006),
    "L1": (30.56289, -90.77424, -6.574, 252.2835, 162.2835),
    "V1": (43.63146, 10.50450, 51.884, 19.4326, 289.4326),
}
_WGS84_A = 6378137.0
_WGS84_E2 = 6.69437999014e-3


def detector(name: str):
    """Return (response tensor d (3,3), vertex position x (3,) in metres), Earth-fixed.

    d = (u u^T - v v^T)/2 for unit arm vectors u (x arm) and v (y arm)."""
    lat, lon, h, xaz, yaz = _SITES[name]
    la, lo = math.radians(lat), math.radians(lon)
    n = _WGS84_A / math.sqrt(1.0 - _WGS84_E2 * math.sin(la) ** 2)
    pos = np.array([(n + h) * math.cos(la) * math.cos(lo),
                    (n + h) * math.cos(la) * math.sin(lo),
                    (n * (1.0 - _WGS84_E2) + h) * math.sin(la)])
    east = np.array([-math.sin(lo), math.cos(lo), 0.0])
    north = np.array([-math.sin(la) * math.cos(lo), -math.sin(la) * math.sin(lo), math.cos(la)])

    def arm(az):
        a = math.radians(az)
        return math.cos(a) * north + math.sin(a) * east

    u, v = arm(xaz), arm(yaz)
    return 0.5 * (np.outer(u, u) - np.outer(v, v)), pos


def max_light_delay(pos) -> float:
    """Largest |x . n| / c over unit vectors n: the time-of-flight bound |x|/c."""
    return float(np.linalg.norm(pos)) / C_LIGHT


# ---------------------------------------------------------------------------
# Noise curve and waveform
# ---------------------------------------------------------------------------
def psd_aligo(f):
    """Analytic zero-detuned high-power aLIGO fit (Sathyaprakash & Schutz 2009)."""
    x = np.asarray(f, dtype=np.float64) / 215.0
    with np.errstate(divide="ignore", invalid="ignore"):
        s = 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))
    return s


ALL_MODES = [(l, m) for l in (2, 3, 4) for m in range(-l, l + 1)]
L2_MODES = [(2, m) for m in range(-2, 3)]


@dataclass
class PointSpec:
    """Shape of one intrinsic point's inputs (one ILE 'lambda')."""
    dets: tuple = ("H1", "L1")
    modes: list = field(default_factory=lambda: list(L2_MODES))
    fs: float = 4096.0            # Q sampling rate (Hz)
    n_t: int | None = None        # Q samples per (k, lm); None -> from t_half
    t_half: float = 0.05          # geocentre time prior is U[-t_half, t_half] around t_ref
    seg_len: float = 8.0          # data segment length (s); df = 1/seg_len
    f_lo: float = 20.0
    f_hi: float = 1024.0
    snr: float = 15.0
    noise: bool = True
    d_ref: float = 100.0          # Mpc
    d_inj: float = 400.0          # Mpc (scale of the drawn injection coefficients)
    t_ref_gps: float = T_REF_GPS
    psd_scale: tuple | None = None  # per-detector multiplier of the PSD
    taps_pad: int = 3             # extra Q samples beyond the time-of-flight bound


def cfg_small() -> PointSpec:
    """Plain ILE, small: H1/L1, l=2 (5 modes), 4096 Hz, t in +-0.05 s, SNR 15."""
    return PointSpec()


def cfg_full() -> PointSpec:
    """Plain ILE, full size: H1/L1/V1, 2<=l<=4 (21 modes), Q over +-0.1 s at 16384 Hz
    (3277 samples), SNR 30, time prior U[-0.05, 0.05] s (the small configuration's priors)."""
    return PointSpec(dets=("H1", "L1", "V1"), modes=list(ALL_MODES), fs=16384.0,
                     n_t=2 * 1638 + 1, t_half=0.05, snr=30.0)


def _window(spec: PointSpec, positions):
    """Q grid: n_t samples centred on t_ref; returns (n_t, J) with tau_j = (j - J)/fs."""
    if spec.n_t is None:
        dmax = max(max_light_delay(p) for p in positions)
        J = int(math.ceil((spec.t_half + dmax) * spec.fs)) + spec.taps_pad
        n_t = 2 * J + 1
    else:
        n_t = int(spec.n_t)
        J = (n_t - 1) // 2
    return n_t, J


def _phase_series(fgw, mc_s, coeffs):
    """Chirp phase at GW frequency fgw (>0): sum_j a_j (pi Mc f)^((j-5)/3)."""
    v = np.pi * mc_s * fgw
    out = np.zeros_like(fgw)
    for j, a in enumerate(coeffs):
        if a != 0.0:
            out += a * v ** ((j - 5.0) / 3.0)
    return out


def _taper(F, lo, hi):
    w = np.zeros_like(F)
    ramp_lo, ramp_hi = 5.0, 64.0
    inb = (F >= lo) & (F <= hi)
    w[inb] = 1.0
    a = inb & (F < lo + ramp_lo)
    w[a] = 0.5 * (1.0 - np.cos(np.pi * (F[a] - lo) / ramp_lo))
    b = inb & (F > hi - ramp_hi)
    w[b] = 0.5 * (1.0 - np.cos(np.pi * (hi - F[b]) / ramp_hi))
    return w


def mode_waveforms(freqs, modes, rng, spec: PointSpec):
    """h_lm(f) at D_ref on the FFT frequency grid, unit overall amplitude.

    m > 0 modes sit at negative frequency (h_lm ~ exp(-i m Phi(t))), m < 0 follow
    the reflection h_{l,-m}(f) = (-1)^l conj(h_{lm}(-f)), m = 0 modes are real
    time series of small amplitude."""
    F = np.abs(freqs)
    amp = np.zeros_like(F)
    nz = F > 0
    amp[nz] = F[nz] ** (-7.0 / 6.0)
    amp *= _taper(F, spec.f_lo, spec.f_hi)
    mc = rng.uniform(8.0, 40.0) * MSUN_S
    coeffs = [3.0 / 128.0, 0.0, 3.0 / 128.0 * rng.uniform(2.0, 5.0),
              -3.0 / 128.0 * 16.0 * np.pi * rng.uniform(0.8, 1.2), 3.0 / 128.0 * rng.uniform(5.0, 15.0)]
    ratio = {}
    chi = {}
    for l in (2, 3, 4):
        for m in range(0, l + 1):
            ratio[(l, m)] = 1.0 if (l, m) == (2, 2) else rng.uniform(0.05, 0.5) * (0.3 if m == 0 else 1.0)
            chi[(l, m)] = rng.uniform(0.0, 2.0 * np.pi)

    def positive_m(l, m):
        # support on f < 0; phase of the m-th harmonic of the orbital phase
        h = np.zeros(freqs.shape, dtype=np.complex128)
        neg = freqs < 0
        Fm = F[neg]
        psi_m = 0.5 * m * _phase_series(2.0 * Fm / m, mc, coeffs)
        h[neg] = ratio[(l, m)] * amp[neg] * np.exp(1j * (psi_m + chi[(l, m)]))
        return h

    n = freqs.shape[0]
    mirror = (-np.arange(n)) % n  # index of -f on the FFT grid
    out = np.zeros((len(modes), n), dtype=np.complex128)
    for i, (l, m) in enumerate(modes):
        if m > 0:
            out[i] = positive_m(l, m)
        elif m < 0:
            hp = positive_m(l, -m)
            out[i] = (-1) ** l * np.conj(hp[mirror])
        else:
            pos = freqs > 0
            h = np.zeros(n, dtype=np.complex128)
            psi0 = _phase_series(F[pos], mc, coeffs)
            h[pos] = ratio[(l, 0)] * amp[pos] * np.exp(-1j * (psi0 + chi[(l, 0)]))
            h = h + np.conj(h[mirror])
            out[i] = h
    return out, mirror


def draw_injection(spec: PointSpec, rng):
    """Detector-frame injection coefficients c_{k,lm} and arrival offsets t_k.

    c_{k,lm} = (D_ref/D_inj) a_k y_lm with a seeded complex per-detector factor a_k
    and per-mode weight y_lm = r_lm exp(i m phi0); t_k = t0 + small offset."""
    K, M = len(spec.dets), len(spec.modes)
    a = rng.uniform(-0.7, 0.7, K) + 1j * rng.uniform(-0.7, 0.7, K)
    phi0 = rng.uniform(0.0, 2.0 * np.pi)
    y = np.empty(M, dtype=np.complex128)
    for i, (l, m) in enumerate(spec.modes):
        r = rng.uniform(0.05, 0.6) if abs(m) == 2 and l == 2 else rng.uniform(0.0, 0.25)
        y[i] = r * np.exp(1j * m * phi0)
    coef = (spec.d_ref / spec.d_inj) * np.outer(a, y)
    t0 = rng.uniform(-0.3, 0.3) * spec.t_half
    tk = t0 + rng.uniform(-0.008, 0.008, K)
    return coef, tk


def _inner(a, b, w, df):
    """2 df sum_f conj(a) b / S over the band (w = mask / S)."""
    return 2.0 * df * np.sum(np.conj(a) * b * w, axis=-1)


def make_point(spec: PointSpec, seed: int, injection=None):
    """Build one point's inputs.

    injection: None (draw detector-frame coefficients) or a pair (coef (K,M), t_k (K,)).
    Returns a dict with the create() inputs (det_tensor, det_pos, lm, Q, q_t0_gps, fs, U, V,
    t_ref_gps, d_ref_mpc, t_lo, t_hi) and the frequency-domain arrays the oracle's
    brute-force checks need (freqs, df, hlm, data, weight = band/S, mirror)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x52494654, int(seed) & 0xFFFFFFFFFFFF]))
    K, M = len(spec.dets), len(spec.modes)
    geo = [detector(d) for d in spec.dets]
    tens = np.stack([g[0] for g in geo])
    pos = np.stack([g[1] for g in geo])

    n = int(round(spec.fs * spec.seg_len))
    df = 1.0 / spec.seg_len
    freqs = np.fft.fftfreq(n, 1.0 / spec.fs)
    F = np.abs(freqs)
    band = (F >= spec.f_lo) & (F <= spec.f_hi)
    psd = np.ones((K, n))
    with np.errstate(divide="ignore", invalid="ignore"):
        base = psd_aligo(np.where(F > 0, F, 1.0))
    scales = spec.psd_scale or tuple(1.0 for _ in range(K))
    weight = np.zeros((K, n))
    for k in range(K):
        psd[k] = base * scales[k]
        weight[k, band] = 1.0 / psd[k, band]

    hlm, mirror = mode_waveforms(freqs, spec.modes, rng, spec)
    if injection is None:
        coef, tk = draw_injection(spec, rng)
    else:
        coef, tk = (np.asarray(injection[0], dtype=np.complex128), np.asarray(injection[1], dtype=np.float64))

    def signal(scale):
        s = np.zeros((K, n), dtype=np.complex128)
        for k in range(K):
            acc = np.zeros(n, dtype=np.complex128)
            for i in range(M):
                acc += 0.5 * (coef[k, i] * hlm[i] + np.conj(coef[k, i]) * np.conj(hlm[i][mirror]))
            s[k] = scale * acc * np.exp(-2j * np.pi * freqs * tk[k])
        return s

    s = signal(1.0)
    rho2 = sum(float(np.real(_inner(s[k], s[k], weight[k], df))) for k in range(K))
    amp = spec.snr / math.sqrt(rho2) if (spec.snr and rho2 > 0) else 1.0
    hlm = hlm * amp
    s = s * amp

    data = s.copy()
    if spec.noise:
        pos_f = (freqs > 0) & band
        for k in range(K):
            sig = np.sqrt(0.25 * psd[k][pos_f] * spec.seg_len)
            nz = np.zeros(n, dtype=np.complex128)
            nz[pos_f] = rng.normal(0.0, 1.0, pos_f.sum()) * sig + 1j * rng.normal(0.0, 1.0, pos_f.sum()) * sig
            nz = nz + np.conj(nz[mirror]) * (~pos_f)  # real noise: n(-f) = conj(n(f))
            data[k] += nz

    n_t, J = _window(spec, pos)
    Q = np.empty((K, M, n_t), dtype=np.complex128)
    idx = (np.arange(n_t) - J) % n
    for k in range(K):
        for i in range(M):
            X = np.conj(hlm[i]) * data[k] * weight[k]
            q = 2.0 * df * n * np.fft.ifft(X)
            Q[k, i] = q[idx]
    U = np.empty((K, M, M), dtype=np.complex128)
    V = np.empty((K, M, M), dtype=np.complex128)
    for k in range(K):
        w = weight[k]
        U[k] = 2.0 * df * (np.conj(hlm) * w) @ hlm.T
        V[k] = 2.0 * df * (hlm[:, mirror] * w) @ hlm.T
    # symmetrise away rounding (U Hermitian, V symmetric by construction)
    U = 0.5 * (U + np.conj(np.transpose(U, (0, 2, 1))))
    V = 0.5 * (V + np.transpose(V, (0, 2, 1)))

    dmax = max(max_light_delay(p) for p in pos)
    t_half = spec.t_half
    return dict(
        det_tensor=tens, det_pos=pos, lm=np.array(spec.modes, dtype=np.int32).reshape(M, 2),
        Q=Q, q_t0_gps=np.full(K, spec.t_ref_gps - J / spec.fs), fs=float(spec.fs), U=U, V=V,
        t_ref_gps=float(spec.t_ref_gps), d_ref_mpc=float(spec.d_ref), t_lo=-t_half, t_hi=t_half,
        # frequency-domain arrays (oracle brute force only)
        freqs=freqs, df=df, hlm=hlm, data=data, weight=weight, mirror=mirror.astype(np.int32),
        nu=np.rint(freqs / df).astype(np.int32),   # the grid's integer bins, freqs = nu df
        coef=coef * amp, tk=tk, snr=spec.snr, dmax=dmax, n_t=n_t, J=J,
    )


def batch_specs(n_points: int, seed: int, snr_range=(8.0, 30.0), fs=16384.0,
                t_range=(800, 3300), m_range=(5, 21)):
    """Per-point specs for the batched workloads: 3 detectors, a mode subset of
    2<=l<=4 of size U{m_range} that always holds (2,+-2), Q length U[t_range],
    SNR U[snr_range].  The time prior of each point is the widest symmetric
    range its Q window covers (window minus time-of-flight bound minus taps)."""
    rng = np.random.default_rng(np.random.SeedSequence([0x42415443, seed]))
    dmax = max(max_light_delay(detector(d)[1]) for d in ("H1", "L1", "V1"))
    specs = []
    others = [lm for lm in ALL_MODES if lm not in ((2, 2), (2, -2))]
    for _ in range(n_points):
        M = int(rng.integers(m_range[0], m_range[1] + 1))
        pick = rng.choice(len(others), size=M - 2, replace=False)
        modes = [(2, -2), (2, 2)] + [others[j] for j in sorted(pick)]
        modes.sort()
        n_t = int(rng.integers(t_range[0], t_range[1] + 1)) | 1
        J = (n_t - 1) // 2
        t_half = J / fs - dmax - 4.0 / fs
        specs.append(PointSpec(dets=("H1", "L1", "V1"), modes=modes, fs=fs, n_t=n_t,
                               t_half=float(t_half), snr=float(rng.uniform(*snr_range))))
    return specs


def create_args(pt):
    """The subset of a make_point() dict that the library's create() consumes."""
    keys = ("det_tensor", "det_pos", "lm", "Q", "q_t0_gps", "fs", "U", "V",
            "t_ref_gps", "d_ref_mpc", "t_lo", "t_hi")
    return {k: pt[k] for k in keys}
