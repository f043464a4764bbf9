"""Post-processing of VP-LBM results (host side, numpy).

- Drag and lift coefficients, C = F / (rho U^2 D / 2) (Section 3.3).
- Strouhal number St = f D / U from the lift signal (Section 3.3): the peak of
  its spectrum, refined by a parabola through the three highest bins, and,
  as a cross-check, the mean spacing of its upward zero crossings.
- Mean drag C_Dave and RMS lift C_Lrms over the second half of a run.
- Relative L2 error over fluid nodes, Eq. err (Section 3.1).
"""
from __future__ import annotations

import math

import numpy as np


def coefficients(fx, fy, u_ref: float, d: float, rho_ref: float = 1.0):
    q = 0.5 * rho_ref * u_ref * u_ref * d
    return np.asarray(fx) / q, np.asarray(fy) / q


def strouhal_fft(cl, u_ref: float, d: float, dt: float = 1.0) -> float:
    """Shedding frequency from the spectral peak of C_L (mean removed,
    Hann window), refined by parabolic interpolation of the log-magnitude."""
    x = np.asarray(cl, dtype=np.float64)
    x = x - x.mean()
    n = len(x)
    if n < 8:
        return float("nan")
    spec = np.abs(np.fft.rfft(x * np.hanning(n)))
    spec[0] = 0.0
    k = int(np.argmax(spec))
    if 0 < k < len(spec) - 1:
        a, b, c = np.log(spec[k - 1] + 1e-300), np.log(spec[k] + 1e-300), np.log(spec[k + 1] + 1e-300)
        den = a - 2 * b + c
        delta = 0.5 * (a - c) / den if den != 0 else 0.0
    else:
        delta = 0.0
    f = (k + delta) / (n * dt)
    return f * d / u_ref


def strouhal_crossings(cl, u_ref: float, d: float, dt: float = 1.0, smooth: int = 1) -> float:
    """Shedding frequency from the mean spacing of upward zero crossings of
    C_L, after a moving average over `smooth` samples (noise rejection)."""
    x = np.asarray(cl, dtype=np.float64)
    if smooth > 1:
        x = np.convolve(x, np.ones(smooth) / smooth, mode="valid")
    x = x - x.mean()
    up = np.nonzero((x[:-1] < 0) & (x[1:] >= 0))[0]
    if len(up) < 3:
        return float("nan")
    # linear interpolation of each crossing time
    tc = up + (-x[up]) / (x[up + 1] - x[up])
    period = np.mean(np.diff(tc)) * dt
    return d / (period * u_ref)


def wake_statistics(fx, fy, u_ref: float, d: float, discard: float = 0.5, dt: float = 1.0):
    """C_Dave, C_Lrms and St over the part of the run after `discard` of it."""
    cd, cl = coefficients(fx, fy, u_ref, d)
    s = int(len(cd) * discard)
    cd, cl = cd[s:], cl[s:]
    return {
        "C_D_ave": float(np.mean(cd)),
        "C_L_rms": float(np.sqrt(np.mean((cl - np.mean(cl)) ** 2))),
        "St": float(strouhal_fft(cl, u_ref, d, dt)),
        "St_crossings": float(strouhal_crossings(cl, u_ref, d, dt, smooth=max(1, len(cl) // 400) | 1)),
        "samples": int(len(cd)),
    }


def l2_error(u, u_exact, fluid) -> float:
    """Relative L2 error over the fluid nodes (Eq. err)."""
    u = np.asarray(u)
    ue = np.asarray(u_exact)
    m = np.asarray(fluid, dtype=bool)
    return math.sqrt(float(((u - ue)[m] ** 2).sum()) / float((ue[m] ** 2).sum()))


def couette_azimuthal(r, r1: float, r2: float, wall_speed: float):
    """Analytic azimuthal velocity between a rotating inner cylinder (radius
    r1, wall speed wall_speed) and a fixed outer one (radius r2), Eq. Sltan."""
    r = np.asarray(r, dtype=np.float64)
    a = wall_speed * r1 / (r2 * r2 - r1 * r1)
    return -a * r + a * r2 * r2 / r
