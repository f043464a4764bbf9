"""Wake statistics of a force record, for the oracle's reference values.

TEST INFRASTRUCTURE ONLY (like the rest of this package): it turns the
oracle's own per-step force series into the quantities Section 3.3 reports,
so that stored expected values come from the oracle alone. It shares no code
with the library's post-processing; the tests check the two against each
other and against closed forms.

Definitions (Section 3.3, with the readings that the paper leaves open):
  C_D = F_x / (rho_ref U^2 D / 2), C_L = F_y / (rho_ref U^2 D / 2), rho_ref = 1
  C_Dave  the mean of C_D over the record
  C_Lrms  the root mean square of C_L about its mean over the record
  St      f D / U, f the frequency of the largest peak of the lift spectrum:
          C_L minus its mean, times a Hann window, its discrete Fourier
          magnitude |X_k|, the bin k of the largest |X_k| (k >= 1), refined by
          the vertex of the parabola through ln|X_{k-1}|, ln|X_k|, ln|X_{k+1}|
  St_x    the same frequency from the mean spacing of the upward zero
          crossings of C_L about its mean (each crossing placed by linear
          interpolation between its two samples)
One sample per time step (Delta t = 1).
"""
from __future__ import annotations

import math

import numpy as np


def force_coefficients(fx, fy, u_ref: float, d: float):
    """C_D and C_L series: force over the dynamic pressure times the diameter."""
    q = 0.5 * 1.0 * u_ref * u_ref * d
    return np.asarray(fx, dtype=np.float64) / q, np.asarray(fy, dtype=np.float64) / q


def hann(n: int) -> np.ndarray:
    """Symmetric Hann window of n points: 0.5 - 0.5 cos(2 pi j / (n - 1))."""
    j = np.arange(n, dtype=np.float64)
    return 0.5 - 0.5 * np.cos(2.0 * math.pi * j / (n - 1))


def peak_frequency(x) -> float:
    """Frequency (cycles per sample) of the largest spectral peak of x about
    its mean, Hann-windowed, refined by a parabola through the logarithms of
    the peak bin and its two neighbours."""
    x = np.asarray(x, dtype=np.float64)
    n = x.size
    y = (x - x.mean()) * hann(n)
    mag = np.abs(np.fft.rfft(y))  # |X_k|, k = 0 .. n/2
    k = 1 + int(np.argmax(mag[1:]))
    shift = 0.0
    if k + 1 < mag.size:
        lm, l0, lp = math.log(mag[k - 1]), math.log(mag[k]), math.log(mag[k + 1])
        curv = lm - 2.0 * l0 + lp
        if curv != 0.0:
            shift = 0.5 * (lm - lp) / curv
    return (k + shift) / n


def crossing_frequency(x) -> float:
    """Frequency (cycles per sample) from the mean spacing of the upward zero
    crossings of x about its mean."""
    x = np.asarray(x, dtype=np.float64)
    x = x - x.mean()
    times = []
    for i in range(x.size - 1):
        if x[i] < 0.0 <= x[i + 1]:
            times.append(i + x[i] / (x[i] - x[i + 1]))
    if len(times) < 3:
        return float("nan")
    return (len(times) - 1) / (times[-1] - times[0])


def wake_statistics(fx, fy, u_ref: float, d: float) -> dict:
    """C_Dave, C_Lrms, St (spectral peak) and St_x (zero crossings) of a
    force record, every sample included."""
    cd, cl = force_coefficients(fx, fy, u_ref, d)
    return {
        "C_D_ave": float(cd.mean()),
        "C_L_rms": float(np.sqrt(((cl - cl.mean()) ** 2).mean())),
        "St": float(peak_frequency(cl) * d / u_ref),
        "St_crossings": float(crossing_frequency(cl) * d / u_ref),
        "samples": int(cd.size),
    }
