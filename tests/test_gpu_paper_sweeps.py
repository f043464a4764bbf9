"""The paper's parameter sweeps at the paper's grid sizes, on the GPU.

Each sweep runs as one batch of independent solves through vplbm_group_step
(one grouped launch per step for all members), to steady state. The plate
sweeps use FP64 storage: their optimum is exact up to rounding, and in FP32 a
steady state carries the rounding step times the diffusion time (the FP32 error
at tau* is 4e-5 against the FP64 oracle's 4e-10 at this size). The cylinder
sweeps use FP32 storage (their staircase errors are ~1e-3).

- Section 3.1, symmetric shear (L = 200, H = 100, e = 50, u^d = 0.01, periodic):
  SRT error near zero at tau* = 1/2 + sqrt(6)/4 and clearly larger at other tau
  (Fig. 3a); MRT error near zero at Lambda = 3/8 for any tau (Figs. 3b, 4).
- Section 3.2, flow between two cylinders (L = 200, R1 = 45, R2 = 70,
  u^d = 0.01): the staircase wall gives a nonzero error for every tau
  (Fig. 11); SRT at tau = 10 gives "unrealistic results" while MRT at tau = 10
  does not (Fig. 10); for MRT "the discrepancy between tau = 0.7 and tau = 10
  is not high" (Section 3.2, with the best Lambda of each). Not reproduced:
  the paper's optimum Lambda = 0.0016 at tau = 10 (Fig. 12b) -- with this
  staircase the error at tau = 10 keeps falling as Lambda grows to 0.1
  (measured 9.2e-3 at 0.0016, 6.2e-3 at 0.1).
- Table 1 / Fig. 17: MRT, tau = 0.7, L = 200..800 with R2 - R1 = 25..100:
  the error decreases with the grid.

The error is the relative L2 error over the fluid nodes (Eq. err), of u for
the plates and of the velocity against the azimuthal profile of Eq. Sltan for
the cylinders. Plate walls sit on the outermost solid rows (y <= e and
y >= e + H), the reading that reproduces the near-zero error at tau*.
"""
import math

import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TAU_STAR = 0.5 + math.sqrt(6.0) / 4.0


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import diag, vplbm
    return vplbm, diag, torch.cuda.Stream()


def _run_batch(V, stream, members):
    """members: list of (cfg, bodies, chi, us, steps); returns the moments."""
    solvers = []
    for cfg, bodies, chi, us, steps in members:
        cfg.stream = stream.cuda_stream
        s = V.Solver(cfg, bodies)
        if chi is not None:
            s.set_mask(chi, us)
        solvers.append(s)
    try:
        V.vplbm_group_step([s.h for s in solvers], [m[4] for m in members])
        return [s.moments() for s in solvers]
    finally:
        for s in solvers:
            s.close()


def _plates(V, tau, coll="srt", lam=3 / 16, L=200, H=100, e=50, ud=0.01, storage="f64"):
    ny = H + 2 * e
    y = np.arange(ny)
    lower, upper = y <= e, y >= e + H
    chi = np.zeros((ny, L), np.uint8)
    chi[lower | upper, :] = 1
    us = np.zeros((2, ny, L))
    us[0][lower, :] = -ud
    us[0][upper, :] = ud
    nu = (tau - 0.5) / 3.0
    steps = int(3 * H * H / nu)  # ~30 decay times of the slowest mode
    cfg = V.make_config(L, ny, coll, storage, tau, lam, ring_len=16)
    exact = 2 * ud / H * (y - e) - ud
    return (cfg, [], chi, us, steps), exact, chi[:, 0] == 0


def _plate_error(diag, mom, exact, fluid):
    ux = mom[1][:, 100]
    return diag.l2_error(ux, exact, fluid)


def test_symmetric_shear_tau_sweep_srt(mods):
    V, diag, stream = mods
    taus = [0.7, 1.0, TAU_STAR, 1.5, 2.0]
    cases = [_plates(V, t) for t in taus]
    moms = _run_batch(V, stream, [c[0] for c in cases])
    err = {t: _plate_error(diag, m, c[1], c[2]) for t, m, c in zip(taus, moms, cases)}
    print("symmetric shear SRT", err)
    assert err[TAU_STAR] < 1e-8
    assert min(v for t, v in err.items() if t != TAU_STAR) > 1e4 * err[TAU_STAR]


def test_symmetric_shear_lambda_sweep_mrt(mods):
    V, diag, stream = mods
    lams = [1 / 16, 3 / 16, 3 / 8, 3 / 4]
    cases = [_plates(V, 0.7, "mrt", lam) for lam in lams] + [_plates(V, 1.5, "mrt", 3 / 8)]
    moms = _run_batch(V, stream, [c[0] for c in cases])
    err = [_plate_error(diag, m, c[1], c[2]) for m, c in zip(moms, cases)]
    print("symmetric shear MRT lambda", dict(zip(lams + ["3/8 at tau 1.5"], err)))
    assert err[2] < 1e-8 and err[4] < 1e-8  # Lambda = 3/8, tau = 0.7 and 1.5
    assert min(err[0], err[1], err[3]) > 1e4 * err[2]


def _couette(V, tau, coll="srt", lam=3 / 16, L=200, r1=45.0, r2=70.0, ud=0.01, steps=None):
    c = (L - 1) / 2.0
    bodies = [I.BodySpec(c, c, r1, omega=ud / r1), I.BodySpec(c, c, r2, outside=True)]
    nu = (tau - 0.5) / 3.0
    steps = steps or max(20_000, int(8 * (r2 - r1) ** 2 / nu))
    cfg = V.make_config(L, L, coll, "f32", tau, lam, ring_len=16)
    return (cfg, bodies, None, None, steps), (L, c, r1, r2, ud)


def _couette_error(diag, mom, geo):
    L, c, r1, r2, ud = geo
    yy, xx = np.mgrid[0:L, 0:L]
    dx, dy = xx - c, yy - c
    r = np.hypot(dx, dy)
    fluid = ((dx ** 2 + dy ** 2) > r1 ** 2) & ((dx ** 2 + dy ** 2) < r2 ** 2)
    ut = diag.couette_azimuthal(np.where(fluid, r, r1), r1, r2, ud)
    ux_e, uy_e = -ut * dy / np.where(r > 0, r, 1), ut * dx / np.where(r > 0, r, 1)
    num = ((mom[1] - ux_e) ** 2 + (mom[2] - uy_e) ** 2)[fluid].sum()
    den = (ux_e ** 2 + uy_e ** 2)[fluid].sum()
    return math.sqrt(num / den)


def test_two_cylinders_tau_and_lambda(mods):
    V, diag, stream = mods
    specs = [("srt", 0.7, 3 / 16), ("srt", 1.0, 3 / 16), ("srt", 10.0, 3 / 16)]
    specs += [("mrt", 0.7, lam) for lam in (0.05, 0.1, 3 / 16, 0.3, 0.6)]
    specs += [("mrt", 10.0, lam) for lam in (0.0004, 0.0016, 0.005, 0.02, 0.1)]
    cases = [_couette(V, t, c, lam) for c, t, lam in specs]
    moms = _run_batch(V, stream, [c[0] for c in cases])
    err = {s: _couette_error(diag, m, c[1]) for s, m, c in zip(specs, moms, cases)}
    print("two cylinders", err)
    assert all(v > 1e-4 for v in err.values())  # staircase: never exact
    best = {}
    for tau in (0.7, 10.0):
        lam, e = min(((k[2], v) for k, v in err.items() if k[0] == "mrt" and k[1] == tau),
                     key=lambda kv: kv[1])
        best[tau] = (lam, e)
    print("best Lambda", best)
    assert best[10.0][1] < 2.0 * best[0.7][1]            # MRT: tau = 10 close to tau = 0.7
    assert err[("srt", 10.0, 3 / 16)] > 10 * best[10.0][1]  # SRT at tau = 10 is unrealistic


def test_two_cylinders_grid_refinement_table1(mods):
    V, diag, stream = mods
    grids = [(200, 25), (400, 50), (600, 75), (800, 100)]  # Table 1: L, Ngrid = R2 - R1
    cases = []
    for L, ng in grids:
        s = L / 200.0
        cases.append(_couette(V, 0.7, "mrt", 3 / 16, L=L, r1=45.0 * s, r2=45.0 * s + ng))
    moms = _run_batch(V, stream, [c[0] for c in cases])
    err = [_couette_error(diag, m, c[1]) for m, c in zip(moms, cases)]
    print("Table 1 grids", dict(zip(grids, err)))
    assert all(a > b for a, b in zip(err, err[1:]))
