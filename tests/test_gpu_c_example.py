"""The C usage example (tests/c/example_cylinder.c) built and run on the GPU:
its mean drag coefficient against the FP64 oracle on the same case.

Case: 256 x 64 channel, cylinder of D = 16 at (64, 31.5), Re = 100 (tau =
0.53), MRT with FP32 storage, seeded 1e-4 perturbation (seed 1, generated on
the device by the example and on the host for the oracle: the same numbers),
3000 steps; mean C_D over the second half. FP32 storage against FP64 over
3000 steps of a steady start: 1e-4 relative.
"""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_example_mean_drag_matches_oracle(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    from paper_1812_05401_gb300 import build as B
    B.build()
    pkg = os.path.join(ROOT, "paper_1812_05401_gb300")
    exe = str(tmp_path / "cylinder")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "example_cylinder.c"), "-o", exe,
                    "-L", pkg, "-lvplbm", "-Wl,-rpath," + pkg], check=True)
    nx, ny, d, steps = 256, 64, 16.0, 3000
    out = subprocess.run([exe, str(nx), str(ny), str(d), str(steps)], check=True,
                         capture_output=True, text=True, timeout=300).stdout
    cd_gpu = float(re.search(r"mean C_D over steps \d+\.\.\d+: (\S+)", out).group(1))

    w = I.cylinder_channel(nx, ny, d, 0.05, 100.0, steps, xc=nx / 4.0, collision="mrt",
                           perturbation=1e-4, seed=1)
    cfg = O.Config(nx=nx, ny=ny, collision=O.MRT, tau=O.tau_from_reynolds(0.05, d, 100.0),
                   lam=3 / 16, bc_x=O.BC_INLET_OUTLET, bc_y=O.BC_FREE_SLIP, u_in=(0.05, 0.0),
                   bodies=[O.Body(b.cx, b.cy, b.radius) for b in w.bodies])
    f = O.init_equilibrium(cfg, 1.0, w.initial_velocity())
    fx, _, _ = O.run(cfg, f, steps)
    cd_ref = float(np.mean(fx[steps // 2:])) / (0.5 * 0.05 ** 2 * d)
    print("C example", cd_gpu, "oracle", cd_ref)
    assert cd_gpu == pytest.approx(cd_ref, rel=1e-4)
