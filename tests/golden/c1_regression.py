"""Writes tests/golden/c1_circular_couette.json: the FP64 oracle's error on
the circular Couette configuration (128 x 128, inner disc R1 = 24 rotating at
wall speed 0.01, fixed outer wall R2 = 56, centre 63.5, SRT tau = 0.8, from
rest, 10^4 steps).

The paper prints this error only in figures (Section 3.2, Fig. 11), so the
value is not the paper's: it is the oracle's, locked as a regression. The
tests hold the oracle (CPU) and the FP64 GPU path to it.

Error: relative L2 norm of the velocity against the analytic azimuthal
profile (Eq. Sltan) over the fluid nodes (Eq. err), from the velocity the
next step computes (the pulled populations of step 10^4).

    python tests/golden/c1_regression.py      # rewrites the JSON (oracle only)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
GOLDEN = os.path.join(HERE, "c1_circular_couette.json")


def c1_error(ux, uy, chi, n=128, r1=24.0, r2=56.0, wall_speed=0.01) -> float:
    """Relative L2 error (Eq. err) over chi == 0 of (ux, uy) against the
    circular Couette field u_theta(r) = a (r2^2 / r - r),
    a = U r1 / (r2^2 - r1^2) (Eq. Sltan), centred at ((n-1)/2, (n-1)/2)."""
    c = (n - 1) / 2.0
    yy, xx = np.mgrid[0:n, 0:n]
    dx, dy = xx - c, yy - c
    r = np.hypot(dx, dy)
    r = np.where(r > 0, r, 1.0)  # the centre is solid; keep the division finite
    a = wall_speed * r1 / (r2 * r2 - r1 * r1)
    ut = a * (r2 * r2 / r - r)
    ex, ey = -ut * dy / r, ut * dx / r
    fl = np.asarray(chi) == 0
    num = ((ux - ex)[fl] ** 2 + (uy - ey)[fl] ** 2).sum()
    den = (ex[fl] ** 2 + ey[fl] ** 2).sum()
    return float(np.sqrt(num / den))


def oracle_c1_error(steps: int = 10_000) -> float:
    sys.path.insert(0, ROOT)
    import oracle as O
    from paper_1812_05401_gb300 import inputs as I
    w = I.c1_circular_couette()
    cfg = O.Config(nx=w.nx, ny=w.ny, collision=O.SRT, tau=w.tau, lam=w.lam,
                   bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                                  b.outside) for b in w.bodies])
    f = O.init_equilibrium(cfg)
    O.run(cfg, f, steps)
    _, ux, uy = O.moments(cfg, f, steps)
    chi, _ = O.mask(cfg, steps)
    return c1_error(ux, uy, chi, w.nx, w.bodies[0].radius, w.bodies[1].radius,
                    w.bodies[0].omega * w.bodies[0].radius)


def main():
    e = oracle_c1_error()
    with open(GOLDEN, "w") as fh:
        json.dump({"l2_error": e, "steps": 10_000,
                   "cite": "Section 3.2, Eq. Sltan (analytic profile), Eq. err (L2 norm); the "
                           "paper plots this error (Fig. 11) without printing it",
                   "source": "FP64 oracle, written by tests/golden/c1_regression.py"}, fh, indent=1)
        fh.write("\n")
    print(e)


if __name__ == "__main__":
    main()
