"""CPU checks of the post-processing (diag.py) against closed forms."""
import math

import numpy as np
import pytest

from paper_1812_05401_gb300 import diag


def test_coefficients_definition():
    cd, cl = diag.coefficients([2.0], [-1.0], u_ref=0.05, d=40.0)
    q = 0.5 * 0.05 ** 2 * 40.0
    assert cd[0] == pytest.approx(2.0 / q) and cl[0] == pytest.approx(-1.0 / q)


@pytest.mark.parametrize("period", [377.3, 1000.0, 2513.7])
def test_strouhal_of_a_sinusoid(period):
    t = np.arange(40000)
    cl = 0.3 + 0.8 * np.sin(2 * np.pi * t / period + 0.4)
    u, d = 0.05, 40.0
    st = d / (period * u)
    assert diag.strouhal_fft(cl, u, d) == pytest.approx(st, rel=2e-3)
    assert diag.strouhal_crossings(cl, u, d) == pytest.approx(st, rel=1e-4)


def test_wake_statistics_of_a_synthetic_signal():
    t = np.arange(20000)
    q = 0.5 * 0.04 ** 2 * 128
    fx = q * (1.5 + 0.01 * np.sin(4 * np.pi * t / 800.0))
    fy = q * 0.7 * math.sqrt(2) * np.sin(2 * np.pi * t / 800.0)
    s = diag.wake_statistics(fx, fy, 0.04, 128.0)
    assert s["C_D_ave"] == pytest.approx(1.5, abs=1e-4)
    assert s["C_L_rms"] == pytest.approx(0.7, rel=1e-3)
    assert s["St"] == pytest.approx(128.0 / (800.0 * 0.04), rel=3e-3)


def test_l2_error_and_couette_profile():
    r = np.linspace(24, 56, 50)
    u = diag.couette_azimuthal(r, 24.0, 56.0, 0.01)
    assert u[0] == pytest.approx(0.01) and abs(u[-1]) < 1e-15
    assert diag.l2_error(u, u, np.ones_like(u, bool)) == 0.0
    assert diag.l2_error(1.01 * u, u, np.ones_like(u, bool)) == pytest.approx(0.01)
