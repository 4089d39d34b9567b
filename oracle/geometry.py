"""Sidereal time, detector response and arrival-time delays (FP64 oracle).

Sec. II.A: the detector output is h_k = F_+ h_+(t_k) + F_x h_x(t_k) with arrival
time t_k at the k-th vertex, and F_k = F_+ - i F_x; F is taken time independent
over the coincidence window, so one sidereal angle per intrinsic point is used.

Conventions (the paper gives none; readings recorded in the design notes):
* GMST from the IAU-1982 polynomial in UT1, UT1 ~ UTC = GPS - 18 s.
* Source direction n = (cos dec cos a, cos dec sin a, sin dec) in the Earth-fixed
  frame, a = ra - GMST.  Arrival time t_k = t + delay_k, delay_k = -(x_k . n)/c
  (a vertex displaced toward the source is reached first).
* Polarisation axes: with e_ra = (-sin a, cos a, 0) and
  e_dec = (-sin dec cos a, -sin dec sin a, cos dec),
  X = -cos(psi) e_ra + sin(psi) e_dec,  Y = sin(psi) e_ra + cos(psi) e_dec,
  F_+ = X.d.X - Y.d.Y, F_x = X.d.Y + Y.d.X  (Anderson et al. 2001, PRD 63 042003).
"""
from __future__ import annotations

import numpy as np

C_LIGHT = 299792458.0
GPS_EPOCH_JD = 2444244.5      # 1980-01-06 00:00 UTC
LEAP_SECONDS = 18.0           # GPS - UTC after 2017-01-01


def gmst_from_days(d):
    """IAU-1982 Greenwich mean sidereal time (radians) at d = JD(UT1) - 2451545.0 days.

    GMST[s] = 67310.54841 + (876600 h + 8640184.812866 s) T + 0.093104 T^2 - 6.2e-6 T^3,
    T = d / 36525.  The 876600 h per century term is exactly 86400 s per day, so modulo
    one day it reduces to 86400 * frac(d); keeping it separate keeps FP64 precision."""
    d = np.asarray(d, dtype=np.float64)
    T = d / 36525.0
    sec = 67310.54841 + 8640184.812866 * T + 0.093104 * T * T - 6.2e-6 * T ** 3
    sec = sec + 86400.0 * (d - np.floor(d))
    sec = np.mod(sec, 86400.0)
    return sec / 86400.0 * 2.0 * np.pi


def gmst_from_gps(gps):
    d = (np.asarray(gps, dtype=np.float64) - LEAP_SECONDS) / 86400.0 + (GPS_EPOCH_JD - 2451545.0)
    return gmst_from_days(d)


def source_direction(ra, dec, gmst):
    a = np.asarray(ra) - gmst
    return np.stack([np.cos(dec) * np.cos(a), np.cos(dec) * np.sin(a), np.sin(dec) * np.ones_like(a)], axis=-1)


def polarisation_axes(ra, dec, psi, gmst):
    a = np.asarray(ra, dtype=np.float64) - gmst
    dec = np.asarray(dec, dtype=np.float64)
    psi = np.asarray(psi, dtype=np.float64)
    e_ra = np.stack([-np.sin(a), np.cos(a), np.zeros_like(a)], axis=-1)
    e_dec = np.stack([-np.sin(dec) * np.cos(a), -np.sin(dec) * np.sin(a), np.cos(dec)], axis=-1)
    c, s = np.cos(psi)[..., None], np.sin(psi)[..., None]
    X = -c * e_ra + s * e_dec
    Y = s * e_ra + c * e_dec
    return X, Y


def antenna(d, ra, dec, psi, gmst):
    """(F_+, F_x) for response tensor d (3,3) at sample arrays."""
    X, Y = polarisation_axes(ra, dec, psi, gmst)
    Fp = np.einsum("...i,ij,...j->...", X, d, X) - np.einsum("...i,ij,...j->...", Y, d, Y)
    Fx = np.einsum("...i,ij,...j->...", X, d, Y) + np.einsum("...i,ij,...j->...", Y, d, X)
    return Fp, Fx


def complex_antenna(d, ra, dec, psi, gmst):
    """F = F_+ - i F_x (Sec. II.A)."""
    Fp, Fx = antenna(d, ra, dec, psi, gmst)
    return Fp - 1j * Fx


def delay(pos, ra, dec, gmst):
    """delay = -(x . n)/c, seconds; arrival time at the vertex is t + delay."""
    n = source_direction(ra, dec, gmst)
    return -(n @ np.asarray(pos, dtype=np.float64)) / C_LIGHT
