"""Writes tests/golden/c2_wake_statistics.json: the FP64 oracle's wake
statistics of the Re = 100 cylinder channel.

Configuration: 1024 x 256 nodes, cylinder of D = 40 centred at (256, 127.5),
uniform inlet u = 0.05 at x = 0, zero-gradient outlet, free-slip walls, MRT
with Lambda = 3/16, tau from Re = U D / nu = 100, initial state the
equilibrium of the inlet velocity plus a seeded 1e-4 perturbation (seed 1).
The oracle develops the wake for 60,000 steps and records the force on the
solid over the next 60,000 (about 14 shedding periods); the statistics are
those of Section 3.3 (C_Dave, C_Lrms, St), computed by oracle.statistics over
the recorded window.

The paper has no Re = 100 case, so these values are not the paper's: they are
the oracle's, the reference the GPU path's storage forms are held to.

    python tests/golden/c2_wake_statistics.py      # rewrites the JSON (oracle only)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
GOLDEN = os.path.join(HERE, "c2_wake_statistics.json")
DEVELOP, MEASURE = 60_000, 60_000
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def oracle_c2_config():
    import oracle as O
    from paper_1812_05401_gb300 import inputs as I
    w = I.c2_cylinder_re100()
    cfg = O.Config(nx=w.nx, ny=w.ny, collision=O.MRT,
                   tau=O.tau_from_reynolds(w.u_ref, w.l_ref, w.re), lam=w.lam,
                   bc_x=O.BC_INLET_OUTLET, bc_y=O.BC_FREE_SLIP, u_in=(w.u_ref, 0.0),
                   bodies=[O.Body(b.cx, b.cy, b.radius) for b in w.bodies])
    return w, cfg


def main():
    import oracle as O
    from oracle import statistics as OS
    w, cfg = oracle_c2_config()
    f = O.init_equilibrium(cfg, 1.0, w.initial_velocity())
    t0 = time.time()
    chunk = 5000
    for t in range(0, DEVELOP, chunk):
        O.run(cfg, f, chunk, t0=t)
        print(f"develop {t + chunk} steps, {time.time() - t0:.0f} s", flush=True)
    fx, fy = np.zeros(MEASURE), np.zeros(MEASURE)
    for t in range(0, MEASURE, chunk):
        a, b, _ = O.run(cfg, f, chunk, t0=DEVELOP + t)
        fx[t:t + chunk], fy[t:t + chunk] = a, b
        print(f"measure {t + chunk} steps, {time.time() - t0:.0f} s", flush=True)
    st = OS.wake_statistics(fx, fy, w.u_ref, w.l_ref)
    with open(GOLDEN, "w") as fh:
        json.dump({**st, "develop_steps": DEVELOP, "measure_steps": MEASURE,
                   "workload": w.name, "collision": "mrt", "lambda": w.lam,
                   "perturbation": w.perturbation, "seed": w.seed,
                   "first_record": [float(fx[0]), float(fy[0])],
                   "cite": "Section 3.3 (C_D, C_L and St definitions); the paper has no Re = 100 "
                           "case: the values are the FP64 oracle's",
                   "source": "FP64 oracle, written by tests/golden/c2_wake_statistics.py"}, fh, indent=1)
        fh.write("\n")
    print(json.dumps(st))


if __name__ == "__main__":
    main()
