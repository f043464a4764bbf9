"""Reduced-precision storage on the higher-Re cylinder wake (4096 x 1024,
D = 128, u = 0.04, Re = 1000): FP32 populations against FP16 and BF16
offsets (f - w, stochastic rounding) with FP32 collision and an FP64 force
reduction, as errors of the wake statistics (Section 3.3: C_Dave, St)
against the FP64 path's.

Reading (measured): with the printed MRT rates (Lambda = 3/16, so s_q =
0.079 at tau = 0.51536) this flow diverges within 40,000 steps on the GPU,
and a same-tau analog (1024 x 256, D = 32) diverges by step 30,000 in the
FP64 oracle too; Lambda = 1/32 still diverges by 140,000 steps, Lambda =
1/128 (s_q = 0.99) runs stable. The test uses Lambda = 1/128; the even
moments keep s_n = 1/tau.

The paper prints no numbers for this flow, so the reference is the FP64 GPU
path (pinned to the oracle to 1e-12 over 1000 steps and, on the Re = 100
wake, to the oracle's statistics). FP32 develops the wake (100,000 steps from
the seeded state); every storage then records the same 150,000 steps (about
nine shedding periods) from that state.

The 16-bit stores round stochastically, and one realization's statistics
carry its own rounding noise (measured spread of the FP16 C_Dave error over
realizations: several 1e-4). FP16 runs four realizations (rounding_seed
0..3): the mean of their statistics is held to 1e-3 (the systematic error of
the storage), each realization to 2e-3.
"""
import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

LAMBDA = 1.0 / 128.0
DEVELOP, MEASURE = 100_000, 150_000
_cache = {}


def _workload(storage):
    w = I.c3_cylinder_re1000(storage)
    w.lam = LAMBDA
    return w


def _stats(storage, seed=0):
    if (storage, seed) in _cache:
        return _cache[(storage, seed)]
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import diag
    from paper_1812_05401_gb300 import vplbm as V
    if "developed" not in _cache:
        with V.Solver.from_workload(_workload("f32"), ring_len=16, reduce_mass=False) as s:
            s.step(DEVELOP)
            s.synchronize()
            _cache["developed"] = s.populations()
    w = _workload(storage)
    with V.Solver.from_workload(w, ring_len=MEASURE, reduce_mass=False,
                                with_initial_velocity=False, rounding_seed=seed) as s:
        s.set_populations(_cache["developed"])
        s.step(MEASURE)
        s.synchronize()
        fx, fy, _ = s.forces()
    _cache[(storage, seed)] = diag.wake_statistics(fx, fy, w.u_ref, w.l_ref, discard=0.0)
    return _cache[(storage, seed)]


KEYS = ("C_D_ave", "C_L_rms", "St")


def _err(storage, seeds=(0,)):
    """Signed relative errors against FP64: per realization and of the mean."""
    ref = _stats("f64")
    runs = [_stats(storage, sd) for sd in seeds]
    e = {"runs": [{k: (r[k] - ref[k]) / ref[k] for k in KEYS} for r in runs],
         "mean": {k: (np.mean([r[k] for r in runs]) - ref[k]) / ref[k] for k in KEYS}}
    print(storage, "relative errors against FP64, per rounding seed", e["runs"], "mean", e["mean"])
    return e


def test_fp64_wake_is_developed_shedding():
    s = _stats("f64")
    assert 1.0 < s["C_D_ave"] < 3.0 and 0.15 < s["St"] < 0.35 and s["C_L_rms"] > 0.1


def test_fp32_statistics_within_1e3_of_fp64():
    e = _err("f32")["mean"]
    assert abs(e["C_D_ave"]) < 1e-3 and abs(e["St"]) < 1e-3


def test_fp16_statistics_within_1e3_of_fp64():
    e = _err("f16", (0, 1, 2, 3))
    assert abs(e["mean"]["C_D_ave"]) < 1e-3 and abs(e["mean"]["St"]) < 1e-3
    for r in e["runs"]:
        assert abs(r["C_D_ave"]) < 2e-3 and abs(r["St"]) < 2e-3


def test_bf16_statistics_reported_against_1e3_bar():
    """BF16 offsets keep 8 significant bits; the measured errors of four
    realizations are printed against the 1e-3 bar and held to 1e-2, so that a
    change that makes them worse is seen."""
    e = _err("bf16", (0, 1, 2, 3))
    m = e["mean"]
    print("bf16 mean within the 1e-3 bar:", abs(m["C_D_ave"]) < 1e-3 and abs(m["St"]) < 1e-3)
    for r in e["runs"]:
        assert abs(r["C_D_ave"]) < 1e-2 and abs(r["St"]) < 1e-2
