"""Spin-weighted spherical harmonics -2Y_lm (FP64 oracle).

Eq. (strain_mode) expands h = h_+ - i h_x over -2Y_lm(theta, phi).  The paper
fixes no phase convention; this follows Goldberg et al. (1967), J. Math. Phys.
8, 2155, with the Condon-Shortley phase:

  sY_lm = (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)] sin^{2l}(theta/2)
          sum_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} e^{i m phi} cot^{2r+s-m}(theta/2)

evaluated at s = -2 and (theta, phi) = (inclination, reference phase).  The
product sin^{2l} cot^k is written c^k s^{2l-k} with c = cos(theta/2), s = sin(theta/2)
so it is finite at theta = 0 and pi.
"""
from __future__ import annotations

from math import comb, factorial, pi, sqrt

import numpy as np


def swsh(s: int, l: int, m: int, theta, phi):
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    c = np.cos(theta / 2.0)
    sn = np.sin(theta / 2.0)
    pref = (-1) ** m * sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1)
                            / (4.0 * pi * factorial(l + s) * factorial(l - s)))
    total = np.zeros_like(theta)
    for r in range(0, l - s + 1):
        j = r + s - m
        if j < 0 or j > l + s:
            continue
        k = 2 * r + s - m
        term = comb(l - s, r) * comb(l + s, j) * (-1) ** (l - r - s)
        total = total + term * c ** k * sn ** (2 * l - k)
    return pref * total * np.exp(1j * m * phi)


def ylm_m2(modes, incl, phi):
    """(N, M) array of -2Y_lm(incl, phi) for the point's mode list."""
    incl = np.atleast_1d(incl)
    phi = np.atleast_1d(phi)
    return np.stack([swsh(-2, l, m, incl, phi) for (l, m) in modes], axis=-1)
