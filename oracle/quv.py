"""Mode inner products Q, U, V of Eq. (QUV), FP64 oracle (test infrastructure: only tests, the
smoke check and the benchmark's CPU leg use this package).

With the inner product of Eq. (overlap), <a|b>_k = 2 sum_f df conj(a(f)) b(f) / S_k(|f|) over the
band (`weight` = band / S_k):

  Q_{k,lm}(tau) = 2 df sum_f exp(2 pi i f tau) conj(h_lm(f)) d_k(f) / S_k      (tau on the Q grid),
  U_{k,lm,l'm'} = <h_lm | h_l'm'>_k       = 2 df sum_f conj(h_lm(f)) h_l'm'(f) / S_k,
  V_{k,lm,l'm'} = <h_lm^* | h_l'm'>_k     = 2 df sum_f h_lm(-f) h_l'm'(f) / S_k,

the last because the transform of the conjugate series conj(h_lm(t)) at f is conj(h_lm(-f)).
Every sum runs over the bins of the frequency grid directly (no FFT), in FP64.
"""
from __future__ import annotations

import numpy as np


def q_grid(fd, k):
    """Q_{k,lm} at the grid times tau_j = q_t0_k - t_ref + j / fs, j < n_t; returns (M, n_t)."""
    f = np.asarray(fd["freqs"], dtype=np.float64)
    band = fd["weight"][k] != 0.0
    tau = (fd["q_t0_gps"][k] - fd["t_ref_gps"]) + np.arange(fd["n_t"]) / float(fd["fs"])
    X = np.conj(fd["hlm"][:, band]) * (fd["data"][k][band] * fd["weight"][k][band])[None, :]   # (M, Nb)
    out = np.empty((X.shape[0], tau.size), dtype=np.complex128)
    for a in range(0, tau.size, 256):
        ph = np.exp(2j * np.pi * np.outer(f[band], tau[a:a + 256]))                           # (Nb, n)
        out[:, a:a + 256] = 2.0 * fd["df"] * (X @ ph)
    return out


def quv(fd):
    """(Q [K][M][n_t], U [K][M][M], V [K][M][M]) of a frequency-domain point."""
    K = fd["data"].shape[0]
    hlm, w, df, mirror = fd["hlm"], fd["weight"], fd["df"], np.asarray(fd["mirror"])
    Q = np.stack([q_grid(fd, k) for k in range(K)])
    U = np.stack([2.0 * df * (np.conj(hlm) * w[k]) @ hlm.T for k in range(K)])
    V = np.stack([2.0 * df * (hlm[:, mirror] * w[k]) @ hlm.T for k in range(K)])
    return Q, U, V
