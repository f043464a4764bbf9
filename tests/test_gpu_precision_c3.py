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


def _stats(storage):
    if storage in _cache:
        return _cache[storage]
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
                                with_initial_velocity=False) as s:
        s.set_populations(_cache["developed"])
        s.step(MEASURE)
        s.synchronize()
        fx, fy, _ = s.forces()
    _cache[storage] = diag.wake_statistics(fx, fy, w.u_ref, w.l_ref, discard=0.0)
    return _cache[storage]


def _err(storage):
    ref, s = _stats("f64"), _stats(storage)
    e = {k: abs(s[k] - ref[k]) / abs(ref[k]) for k in ("C_D_ave", "C_L_rms", "St")}
    print(storage, s, "relative error against FP64", e)
    return e


def test_fp64_wake_is_developed_shedding():
    s = _stats("f64")
    assert 1.0 < s["C_D_ave"] < 3.0 and 0.15 < s["St"] < 0.35 and s["C_L_rms"] > 0.1


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_storage_statistics_within_1e3_of_fp64(storage):
    e = _err(storage)
    assert e["C_D_ave"] < 1e-3 and e["St"] < 1e-3


def test_bf16_statistics_reported_against_1e3_bar():
    """BF16 offsets keep 8 significant bits; the measured error is printed
    against the 1e-3 bar and held to 1e-2, so that a change that makes it
    worse is seen."""
    e = _err("bf16")
    print("bf16 within the 1e-3 bar:", e["C_D_ave"] < 1e-3 and e["St"] < 1e-3)
    assert e["C_D_ave"] < 1e-2 and e["St"] < 1e-2
