"""The paper's one printed physics result, reproduced on the GPU path.

Section 3.3 and Table 2: flow past a circular cylinder at Re = 500; domain
30D x 10D discretised with 6048 x 2016 nodes, D = 201 nodes, inlet velocity
0.05, SRT with tau = 0.56 (Re = U D / nu = 502.5), symmetry (free-slip)
top and bottom, constant-velocity inlet, cylinder 25D from the outlet.
Table 2 (VP-LBM column): C_Dave = 1.45, C_Lrms = 0.84, St = 0.22.

Readings: cylinder centre 5D from the inlet (x = 1005) and on the centre line
(y = 1007.5); the outlet is run both as the paper's convective condition
(U_c = the inlet speed) and as a zero-gradient copy; the force is measured both ways -- the penalization volume integral and the
paper's momentum exchange over the mask's fluid-to-solid links; statistics over steps 200,000-400,000 (~11 shedding periods; the
force record shows the shedding saturated by step 200,000), St from the lift
spectrum.

Reproduced (FP32, 400,000 steps, window 200k-400k): convective outlet
C_Dave = 1.553, C_Lrms = 0.935, St = 0.2356; zero-gradient outlet 1.541,
0.970, 0.2342. Against the paper: +7.1%, +11%, +7.1% (convective). Controlled
runs, one change at a time (same steps and window), bound the cause:
  another perturbation seed        C_Dave -0.2%, C_Lrms -0.8%, St  0.0%
  channel height 20D (5% blockage) C_Dave -0.7%, C_Lrms -1.0%, St -0.5%
  half resolution (D = 100)        C_Dave +0.7%, C_Lrms  0.0%, St -0.2%
  MRT, Lambda = 3/16               C_Dave -0.4%, C_Lrms -0.5%, St +0.2%
  centre on a node row             C_Dave +0.1%, C_Lrms -0.7%, St -0.1%
  eta = 1e-5                       C_Dave  0.0%, C_Lrms  0.0%, St  0.0%
  window 400k-800k                 C_Dave +0.15%, C_Lrms -0.3%, St +0.3%
  FP64 vs FP32 over 100k steps     C_Dave 2.6e-4, C_Lrms 2e-4, St 1.3e-4
  inlet ghost at the first
    column's density (not rho = 1) C_Dave +0.29%, C_Lrms +0.14%, St +0.21%
  symmetry planes on the node rows C_Dave +0.01%, C_Lrms +0.03%, St  0.0%
None moves the statistics by more than 1%, so neither blockage, resolution,
the collision operator, the mask position, eta, the window, precision, the
inlet's density nor the position of the symmetry planes explains the 7-11%
gap; the paper's own numbers come from the same 30D x 10D domain. The gap is
stated as open.
Bounds: the reproduced values within 1% (C_Dave, St) and 3% (C_Lrms), which
covers the seed-to-seed spread; both force measures; 1% between the two
measures' C_Dave and St.
"""
import json
import os

import pytest

from paper_1812_05401_gb300 import inputs as I

PAPER = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                    "paper_constants.json")))["cylinder_re500"]

pytestmark = pytest.mark.gpu


REPRODUCED = {"convective": {"C_D_ave": 1.553, "C_L_rms": 0.935, "St": 0.2356},
              "zero-gradient": {"C_D_ave": 1.541, "C_L_rms": 0.970, "St": 0.2342}}


@pytest.mark.parametrize("outlet", ["convective", "zero-gradient"])
def test_table2_cylinder_re500(outlet):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import diag
    from paper_1812_05401_gb300 import vplbm as V
    D, U, steps = float(PAPER["D"]), PAPER["U"], 400_000
    w = I.cylinder_channel(PAPER["nx"], PAPER["ny"], D, U, 500.0, steps, xc=5 * D, collision="srt",
                           storage="f32", perturbation=1e-4, seed=1, outlet=outlet)
    cfg, bodies = V.config_from_workload(w, ring_len=steps, reduce_mass=False)
    cfg.tau = PAPER["tau"]  # as printed
    with V.Solver(cfg, bodies, w.initial_velocity()) as s:
        s.record_momentum_exchange(True)
        s.step(steps)
        s.synchronize()
        fx, fy, _ = s.forces()
        mx, my = s.momentum_exchange_forces()
    st = diag.wake_statistics(fx, fy, U, D, discard=0.5)
    me = diag.wake_statistics(mx, my, U, D, discard=0.5)
    print(f"Table 2 reproduction ({outlet} outlet), penalization integral:", st)
    print(f"Table 2 reproduction ({outlet} outlet), momentum exchange:", me)
    rep = REPRODUCED[outlet]
    print("against the paper:", {k: st[k] / PAPER[k] - 1.0 for k in ("C_D_ave", "C_L_rms", "St")})
    for r in (st, me):
        assert r["C_D_ave"] == pytest.approx(rep["C_D_ave"], rel=0.01)
        assert r["St"] == pytest.approx(rep["St"], rel=0.01)
        assert r["C_L_rms"] == pytest.approx(rep["C_L_rms"], rel=0.03)
    assert me["C_D_ave"] == pytest.approx(st["C_D_ave"], rel=0.01)
    assert me["St"] == pytest.approx(st["St"], rel=0.01)
