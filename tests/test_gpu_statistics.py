"""Wake statistics of every storage form against the FP64 oracle.

Cylinder of D = 40 in a 1024 x 256 free-slip channel at Re = 100 (u = 0.05,
MRT, Lambda = 3/16). Over tens of thousands of steps of an unsteady flow a
pointwise comparison is meaningless, so the runs are compared through their
statistics (Section 3.3): mean drag C_Dave, RMS lift C_Lrms and Strouhal
number St.

The reference is the FP64 oracle's own run (tests/golden/c2_wake_statistics.json,
written by tests/golden/c2_wake_statistics.py, which calls only the oracle):
60,000 steps from the seeded initial state develop the wake, the next 60,000
(about 14 shedding periods) are recorded. The FP64 GPU path repeats that run
from the same initial state. Every other storage starts from the FP64 GPU
path's state at step 60,000 and records the same window, so that the
statistics compare the stationary shedding and not the precision-dependent
time at which shedding starts.

Bars (relative, against the oracle):
  FP64 storage                       1e-8 on C_Dave, C_Lrms and St
  FP32 storage                       1e-3 on C_Dave and St
  FP16 offsets, stochastic rounding  1e-3 on C_Dave and St, for each of four
      realizations of the rounding (rounding_seed 0..3) and their mean
  BF16 offsets, stochastic rounding  misses 1e-3 (8 significant bits): the
      errors of the four realizations are printed and held only to 1e-2, so
      that a change that makes them worse is seen; the test's name says it
      misses the bar.
With round-to-nearest-even the 16-bit forms do not reach 1e-3 on this flow:
the rounding step of an element (~0.01) at 11 significant bits is about ten
times the viscous change of a population per step, and a deterministic
rounding acts as a small systematic forcing. Those tests document the effect
with the FP64 GPU run as the reference and bounds that are the measured
errors with margin (FP16: C_Dave +0.3%, St +0.1%; BF16: C_Dave +1.6%, St
-7.0%, and the RMS lift halved).
"""
import json
import os

import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c2_wake_statistics.json")))
DEVELOP, MEASURE = GOLDEN["develop_steps"], GOLDEN["measure_steps"]
_cache = {}


def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import diag
    from paper_1812_05401_gb300 import vplbm as V
    return V, diag


def _fp64():
    """The FP64 GPU run of the oracle's protocol: statistics of the window
    and the state at its start."""
    if "f64" not in _cache:
        V, diag = _lib()
        w = I.c2_cylinder_re100()
        w.storage = "f64"
        with V.Solver.from_workload(w, ring_len=MEASURE, reduce_mass=False) as s:
            s.step(DEVELOP)
            s.synchronize()
            _cache["developed"] = s.populations()
            s.forces()  # the window's records only
            s.step(MEASURE)
            s.synchronize()
            fx, fy, _ = s.forces()
        _cache["f64"] = diag.wake_statistics(fx, fy, w.u_ref, w.l_ref, discard=0.0)
    return _cache["f64"]


def _run(storage, rounding="stochastic", seed=0):
    if (storage, rounding, seed) in _cache:
        return _cache[(storage, rounding, seed)]
    _fp64()
    V, diag = _lib()
    w = I.c2_cylinder_re100()
    w.storage = storage
    with V.Solver.from_workload(w, ring_len=MEASURE, reduce_mass=False,
                                with_initial_velocity=False, rounding=rounding,
                                rounding_seed=seed) as s:
        s.set_populations(_cache["developed"])
        s.step(MEASURE)
        s.synchronize()
        fx, fy, _ = s.forces()
    st = diag.wake_statistics(fx, fy, w.u_ref, w.l_ref, discard=0.0)
    _cache[(storage, rounding, seed)] = st
    return st


def _rel(a, b):
    return abs(a - b) / abs(b)


def test_golden_is_periodic_shedding():
    """The oracle's reference window is developed shedding (Re = 100)."""
    assert 1.0 < GOLDEN["C_D_ave"] < 3.0
    assert 0.12 < GOLDEN["St"] < 0.3
    assert GOLDEN["C_L_rms"] > 0.05
    assert GOLDEN["St"] == pytest.approx(GOLDEN["St_crossings"], rel=1e-2)


def test_fp64_path_reproduces_oracle_statistics():
    """The FP64 GPU path over the oracle's 120,000 steps: the same statistics
    to 1e-8 (the two differ only in rounding order)."""
    s = _fp64()
    print("f64", s, "oracle", {k: GOLDEN[k] for k in ("C_D_ave", "C_L_rms", "St")})
    for k in ("C_D_ave", "C_L_rms", "St"):
        assert _rel(s[k], GOLDEN[k]) < 1e-8, k


SEEDS = (0, 1, 2, 3)


def _errors(storage, seeds):
    """Signed relative errors against the oracle, per realization and of the
    realizations' mean statistics."""
    runs = [_run(storage, seed=sd) for sd in seeds]
    out = {"runs": [{k: (r[k] - GOLDEN[k]) / GOLDEN[k] for k in ("C_D_ave", "C_L_rms", "St")}
                    for r in runs]}
    out["mean"] = {k: (np.mean([r[k] for r in runs]) - GOLDEN[k]) / GOLDEN[k]
                   for k in ("C_D_ave", "C_L_rms", "St")}
    return out


def test_fp32_statistics_within_1e3_of_oracle():
    s = _run("f32")
    err = {k: _rel(s[k], GOLDEN[k]) for k in ("C_D_ave", "C_L_rms", "St")}
    print("f32 relative error against the oracle", err)
    assert err["C_D_ave"] < 1e-3
    assert err["St"] < 1e-3


def test_fp16_statistics_within_1e3_of_oracle():
    e = _errors("f16", SEEDS)
    print("f16 relative errors against the oracle, per rounding seed", e["runs"], "mean", e["mean"])
    for r in e["runs"] + [e["mean"]]:
        assert abs(r["C_D_ave"]) < 1e-3 and abs(r["St"]) < 1e-3


def test_bf16_stochastic_misses_1e3_bar_reported():
    e = _errors("bf16", SEEDS)
    print("bf16 relative errors against the oracle (bar 1e-3, not met), per rounding seed",
          e["runs"], "mean", e["mean"])
    for r in e["runs"]:
        assert abs(r["C_D_ave"]) < 1e-2 and abs(r["St"]) < 1e-2


@pytest.mark.parametrize("storage,tol_cd,tol_st", [("f32", 1e-3, 1e-3), ("f16", 0.02, 0.015),
                                                   ("bf16", 0.02, 0.08)])
def test_nearest_rounding_statistics(storage, tol_cd, tol_st):
    ref = _fp64()
    s = _run(storage, "nearest")
    print(storage, "nearest", s, "ref", ref)
    assert s["C_D_ave"] == pytest.approx(ref["C_D_ave"], rel=tol_cd)
    assert s["St"] == pytest.approx(ref["St"], rel=tol_st)
