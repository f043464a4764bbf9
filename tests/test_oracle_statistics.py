"""The oracle's wake statistics (oracle/statistics.py) against closed forms,
and the library's post-processing (diag.py) against the oracle's on the same
records: both state the Section 3.3 quantities with the same readings (mean
drag, RMS lift about its mean, Strouhal number from the lift's spectral peak
and from its zero crossings)."""
import math

import numpy as np
import pytest

from oracle import statistics as OS
from paper_1812_05401_gb300 import diag

U, D = 0.05, 40.0
Q = 0.5 * U * U * D  # dynamic pressure times diameter (rho_ref = 1)


def test_coefficients_are_force_over_dynamic_pressure():
    cd, cl = OS.force_coefficients([Q * 1.5, Q * 2.0], [Q * -0.25, 0.0], U, D)
    assert np.array_equal(cd, [1.5, 2.0]) and np.array_equal(cl, [-0.25, 0.0])


@pytest.mark.parametrize("cycles", [7, 14, 31])
def test_integer_cycles_give_exact_statistics(cycles):
    """A lift of whole sine cycles and a drag with a whole number of double-
    frequency cycles: mean drag exact, RMS lift A / sqrt(2), and the spectral
    peak falls on a bin with (nearly: the symmetric Hann window is not exactly
    periodic) equal neighbours, so St is exact to 1e-7."""
    n = 60_000
    t = np.arange(n)
    f0 = cycles / n
    cl = 0.3 * np.sin(2 * math.pi * f0 * t + 0.4)
    cd = 1.4 + 0.02 * np.sin(4 * math.pi * f0 * t)
    s = OS.wake_statistics(cd * Q, cl * Q, U, D)
    assert s["C_D_ave"] == pytest.approx(1.4, abs=1e-12)
    assert s["C_L_rms"] == pytest.approx(0.3 / math.sqrt(2), rel=1e-9)
    assert s["St"] == pytest.approx(f0 * D / U, rel=1e-7)
    assert s["St_crossings"] == pytest.approx(f0 * D / U, rel=1e-6)


def test_off_bin_frequency_within_interpolation_error():
    """Between bins the parabola through the log-magnitudes recovers the
    frequency to a small fraction of a bin (here 14.37 cycles: within 2% of a
    bin); the crossings estimate to round-off of the crossing times."""
    n = 60_000
    f0 = 14.37 / n
    t = np.arange(n)
    cl = 0.25 * np.cos(2 * math.pi * f0 * t)
    s = OS.wake_statistics(np.full(n, Q), cl * Q, U, D)
    assert abs(s["St"] / (D / U) - f0) < 0.02 / n
    assert s["St_crossings"] == pytest.approx(f0 * D / U, rel=1e-6)


def test_library_post_processing_agrees_with_oracle():
    """diag.wake_statistics (discard = 0) on a shedding-like record: mean,
    RMS and spectral St identical to round-off; the crossings estimate agrees
    to the smoothing diag applies against noise."""
    rng = np.random.default_rng(3)
    n = 60_000
    t = np.arange(n)
    f0 = 1 / 4237.3
    cl = 0.28 * np.sin(2 * math.pi * f0 * t) + 0.01 * np.sin(6 * math.pi * f0 * t + 1)
    cd = 1.57 + 0.015 * np.cos(4 * math.pi * f0 * t) + 1e-5 * rng.standard_normal(n)
    a = OS.wake_statistics(cd * Q, cl * Q, U, D)
    b = diag.wake_statistics(cd * Q, cl * Q, U, D, discard=0.0)
    for k in ("C_D_ave", "C_L_rms", "St"):
        assert a[k] == pytest.approx(b[k], rel=1e-12), k
    assert a["St_crossings"] == pytest.approx(b["St_crossings"], rel=1e-4)
