"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances (stated per test):
  FP64 storage: populations within 1e-12 relative (max abs difference over
  max |f|) after up to 1000 steps; forces within 1e-10 relative.
  FP32 storage: velocity within 1e-5 of the reference speed U (max abs).
  FP16/BF16 offset storage: one step from a known state within the storage
  rounding (half an ulp of the stored offset, plus FP32 arithmetic).
Integer work (masks) is compared bit for bit.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

V = None


@pytest.fixture(scope="module", autouse=True)
def _lib():
    global V
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import vplbm
    V = vplbm
    yield


COLL = {"srt": O.SRT, "mrt": O.MRT}
BC = {"periodic": (O.BC_PERIODIC, O.BC_PERIODIC), "channel": (O.BC_INLET_OUTLET, O.BC_FREE_SLIP),
      "inlet-periodic": (O.BC_INLET_OUTLET, O.BC_PERIODIC), "periodic-slip": (O.BC_PERIODIC, O.BC_FREE_SLIP)}
VBC = {"periodic": (0, 0), "channel": (1, 2), "inlet-periodic": (1, 0), "periodic-slip": (0, 2)}


def _pair(nx, ny, coll="srt", storage="f64", bc="periodic", tau=0.7, lam=3 / 16, u_in=(0.04, 0.0),
          g=(0.0, 0.0), bodies=(), chi=None, us=None, rates=None):
    """An oracle config and a GPU solver with the same parameters."""
    bx, by = BC[bc]
    ocfg = O.Config(nx=nx, ny=ny, collision=COLL[coll], tau=tau, lam=lam, bc_x=bx, bc_y=by,
                    u_in=u_in, g=g, chi=chi, us=us, rates=rates,
                    bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega, b.outside)
                            for b in bodies])
    vb = VBC[bc]
    cfg = V.make_config(nx, ny, coll, storage, tau, lam, bc=vb, u_in=u_in,
                        body_force=g, rates=rates)
    s = V.Solver(cfg, list(bodies))
    if chi is not None:
        s.set_mask(chi, us)
    return ocfg, s


def _rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# -----------------------------------------------------------------------------
# One step from a random state: every storage, collision and boundary mix, on
# ragged grids that span several tiles (128 x 2 nodes) with partial edge tiles.
# -----------------------------------------------------------------------------

@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("coll", ["srt", "mrt"])
@pytest.mark.parametrize("bc", ["periodic", "channel", "inlet-periodic", "periodic-slip"])
def test_one_step_random_state(storage, coll, bc):
    nx, ny = 300, 37
    chi = I.random_mask(nx, ny, 11, 0.15)
    us = I.random_solid_velocity(nx, ny, 12, 0.03)
    bodies = [I.BodySpec(200.5, 18.0, 7.0, omega=0.002)]
    ocfg, s = _pair(nx, ny, coll, storage, bc, tau=0.62, g=(1e-6, -2e-6), bodies=bodies,
                    chi=chi, us=us)
    with s:
        f0 = I.random_populations(nx, ny, 13, 0.05)
        s.set_populations(f0)
        fs = s.populations()  # the state as stored (rounded to the storage type)
        f_ref = fs.copy()
        fx_ref, fy_ref, m_ref = O.run(ocfg, f_ref, 1)
        s.step(1)
        s.synchronize()
        f = s.populations()
        fx, fy, ms = s.forces()
    if storage == "f64":
        assert _rel(f, f_ref) < 1e-14
        assert fx[0] == pytest.approx(fx_ref[0], rel=1e-11)
        assert fy[0] == pytest.approx(fy_ref[0], rel=1e-11)
        assert ms[0] == pytest.approx(m_ref[0], rel=1e-14)
    elif storage == "f32":
        assert np.abs(f - f_ref).max() < 4e-7  # FP32 arithmetic on values <= 0.5
        assert fx[0] == pytest.approx(fx_ref[0], rel=1e-5, abs=1e-6)
        assert ms[0] == pytest.approx(m_ref[0], rel=1e-7)
    else:
        # stored offsets h = f - w, stochastically rounded: one ulp of
        # |h| <= 0.06 plus FP32 arithmetic
        ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
        assert np.abs(f - f_ref).max() < 0.06 * ulp + 1e-6
        assert fx[0] == pytest.approx(fx_ref[0], rel=1e-5, abs=1e-6)


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_one_step_16bit_nearest_rounding(storage):
    """Round-to-nearest-even 16-bit stores: within half an ulp of |h|."""
    nx, ny = 300, 37
    ocfg, _ = _pair(nx, ny, "mrt", "f64", "channel", tau=0.62)
    cfg = V.make_config(nx, ny, "mrt", storage, 0.62, bc=VBC["channel"], u_in=(0.04, 0.0),
                        rounding="nearest")
    with V.Solver(cfg) as s:
        s.set_populations(I.random_populations(nx, ny, 13, 0.05))
        f_ref = s.populations()
        O.run(ocfg, f_ref, 1)
        s.step(1)
        f = s.populations()
    ulp = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    assert np.abs(f - f_ref).max() < 0.06 * ulp + 1e-6


def test_stochastic_rounding_is_unbiased():
    """Stochastic 16-bit rounding: the mean rounding error over many nodes is
    far below the rounding step (nearest rounding of the same values is not
    required to be; both stay within their per-value bounds)."""
    nx, ny = 512, 256
    ocfg, _ = _pair(nx, ny, "srt", "f64", "periodic", tau=0.9)
    with V.Solver(V.make_config(nx, ny, "srt", "f16", 0.9, rounding="stochastic")) as s:
        s.set_populations(I.random_populations(nx, ny, 17, 0.05))
        f_ref = s.populations()
        O.run(ocfg, f_ref, 1)
        s.step(1)
        err = s.populations() - f_ref
    ulp = 2.0 ** -10 * 0.06
    assert np.abs(err).max() < ulp + 1e-6
    # per direction, the mean error of 131072 independent roundings is ~0
    assert np.abs(err.reshape(9, -1).mean(axis=1)).max() < 2e-2 * 2.0 ** -11 * 0.02


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 5), (7, 1), (2, 2), (128, 2), (129, 3), (256, 4), (3, 130)])
@pytest.mark.parametrize("bc", ["periodic", "channel"])
def test_edge_sizes(nx, ny, bc):
    """Degenerate and tile-boundary sizes: single rows or columns, one node,
    exact tile multiples and one-past."""
    ocfg, s = _pair(nx, ny, "mrt", "f64", bc, tau=0.8, u_in=(0.03, 0.0))
    with s:
        f0 = I.random_populations(nx, ny, 21, 0.05)
        s.set_populations(f0)
        f_ref = s.populations()
        O.run(ocfg, f_ref, 5)
        s.step(5)
        assert _rel(s.populations(), f_ref) < 1e-14


def test_empty_and_invalid_inputs():
    with pytest.raises(V.VplbmError):
        V.Solver(V.make_config(0, 16))
    s = V.Solver(V.make_config(16, 16))
    with s:
        s.step(0)
        assert s.t == 0
        with pytest.raises(V.VplbmError):
            s.step(-1)
        fx, fy, ms = s.forces()
        assert len(fx) == 0


# -----------------------------------------------------------------------------
# Long runs
# -----------------------------------------------------------------------------

def test_c1_circular_couette_fp64_1000_steps():
    """Circular Couette (128 x 128, R1 = 24 rotating at 0.01, R2 = 56, SRT,
    tau = 0.8): FP64 GPU within 1e-12 relative of the oracle after 1000 steps."""
    w = I.c1_circular_couette()
    ocfg, s = _pair(w.nx, w.ny, "srt", "f64", "periodic", tau=w.tau, bodies=w.bodies)
    with s:
        f_ref = O.init_equilibrium(ocfg)
        fx_ref, fy_ref, m_ref = O.run(ocfg, f_ref, 1000)
        s.step(1000)
        s.synchronize()
        assert _rel(s.populations(), f_ref) < 1e-12
        fx, fy, ms = s.forces()
        # the net force is zero by symmetry up to round-off of the ~1e-3
        # per-node forces, so the comparison is absolute
        np.testing.assert_allclose(fx, fx_ref, rtol=0, atol=1e-12)
        np.testing.assert_allclose(fy, fy_ref, rtol=0, atol=1e-12)
        np.testing.assert_allclose(ms, m_ref, rtol=1e-12)  # summation order differs
        rho, ux, uy = s.moments()
    r2, ux2, uy2 = O.moments(ocfg, f_ref, 1000)
    assert np.abs(ux - ux2).max() < 1e-14 and np.abs(uy - uy2).max() < 1e-14


def test_c1_error_equals_the_locked_oracle_value():
    """C1 on the GPU in FP64 for 10^4 steps: its circular Couette error
    (Eq. err against Eq. Sltan) equals the oracle's locked value
    (tests/golden/c1_circular_couette.json) to FP64 parity (seven digits)."""
    import importlib.util
    import json
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("c1_regression", os.path.join(here, "c1_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "c1_circular_couette.json")) as fh:
        stored = json.load(fh)["l2_error"]
    w = I.c1_circular_couette()
    assert w.storage == "f64" and w.steps == 10_000
    with V.Solver.from_workload(w) as s:
        s.step(w.steps)
        _, ux, uy = s.moments()
        chi = s.mask()
    r1, r2 = w.bodies[0].radius, w.bodies[1].radius
    e = mod.c1_error(ux, uy, chi, w.nx, r1, r2, w.bodies[0].omega * r1)
    # the error is a small difference (about 5.6e-5 per node against speeds
    # of 5e-3): a 1e-13 velocity discrepancy between GPU (FMA contraction) and
    # oracle moves it by up to ~2e-9 relative
    assert e == pytest.approx(stored, rel=1e-7)


@pytest.mark.parametrize("coll", ["srt", "mrt"])
def test_fp32_velocity_within_1e5_of_U(coll):
    """FP32 storage and arithmetic: velocity within 1e-5 U of the FP64 oracle
    after 1000 steps of circular Couette (U = wall speed)."""
    w = I.c1_circular_couette()
    ocfg, s = _pair(w.nx, w.ny, coll, "f32", "periodic", tau=w.tau, bodies=w.bodies)
    with s:
        f_ref = O.init_equilibrium(ocfg)
        O.run(ocfg, f_ref, 1000)
        s.step(1000)
        rho, ux, uy = s.moments()
    _, ux2, uy2 = O.moments(ocfg, f_ref, 1000)
    err = max(np.abs(ux - ux2).max(), np.abs(uy - uy2).max()) / w.u_ref
    assert err < 1e-5, err


def test_mrt_cylinder_channel_fp64():
    """Cylinder in a free-slip channel with uniform inlet and zero-gradient
    outlet (the C2 geometry scaled to 256 x 64, D = 10), MRT, 500 steps."""
    w = I.cylinder_channel(256, 64, 10.0, 0.05, 100.0, 500, xc=64.0, collision="mrt",
                           storage="f64", perturbation=1e-4, seed=5)
    tau = V.vplbm_tau_from_reynolds(w.u_ref, w.l_ref, w.re)
    ocfg, s = _pair(w.nx, w.ny, "mrt", "f64", "channel", tau=tau, u_in=(w.u_ref, 0.0), bodies=w.bodies)
    u0 = w.initial_velocity()
    with s:
        s.set_initial_velocity(u0)
        f_ref = O.init_equilibrium(ocfg, 1.0, u0)
        fx_ref, fy_ref, _ = O.run(ocfg, f_ref, w.steps)
        s.step(w.steps)
        assert _rel(s.populations(), f_ref) < 1e-12
        fx, fy, _ = s.forces()
    np.testing.assert_allclose(fx, fx_ref, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(fy, fy_ref, rtol=1e-7, atol=1e-13)


def test_moving_cylinder_mask_and_flow_fp64():
    """A cylinder translating as y(t) = y0 + A sin(2 pi t / T): the staircase
    mask rebuilt before every step matches the oracle bit for bit, and the
    flow matches in FP64."""
    # body speed up to 2 pi A / T = 0.019: the mask changes by a few nodes
    w = I.moving_cylinder_channel(192, 64, 12.0, 0.05, 60.0, 120, period=2000.0, amp_fraction=0.5,
                                  storage="f64", seed=2)
    tau = V.vplbm_tau_from_reynolds(w.u_ref, w.l_ref, w.re)
    ocfg, s = _pair(w.nx, w.ny, "mrt", "f64", "channel", tau=tau, u_in=(w.u_ref, 0.0), bodies=w.bodies)
    u0 = w.initial_velocity()
    with s:
        s.set_initial_velocity(u0)
        f_ref = O.init_equilibrium(ocfg, 1.0, u0)
        t = 0
        for chunk in (1, 9, 30, 40, 40):
            chi_ref, _ = O.mask(ocfg, t)
            assert np.array_equal(s.mask(), chi_ref), t
            O.run(ocfg, f_ref, chunk, t0=t)
            s.step(chunk)
            t += chunk
        assert _rel(s.populations(), f_ref) < 1e-12


def test_mrt_with_equal_rates_matches_srt_on_gpu():
    nx, ny = 140, 33
    bodies = [I.BodySpec(70.0, 16.0, 6.0, omega=0.003)]
    _, a = _pair(nx, ny, "srt", "f64", "periodic", tau=0.9, bodies=bodies)
    _, b = _pair(nx, ny, "mrt", "f64", "periodic", tau=0.9, bodies=bodies, rates=(1 / 0.9,) * 9)
    with a, b:
        f0 = I.random_populations(nx, ny, 5, 0.05)
        a.set_populations(f0)
        b.set_populations(f0)
        a.step(100)
        b.step(100)
        assert _rel(a.populations(), b.populations()) < 1e-13


def test_poiseuille_at_optimal_tau_on_gpu():
    """The closed-form Poiseuille profile at tau* = 1/2 + sqrt(6)/4 (Section 3.1)
    reproduced by the FP64 GPU path, plates given as a static mask."""
    H, e, gx = 20, 4, 1e-6
    ny, nx = H + 2 * e, 4
    y = np.arange(ny)
    chi = np.zeros((ny, nx), np.uint8)
    chi[(y <= e) | (y >= e + H), :] = 1
    tau = 0.5 + math.sqrt(6) / 4
    nu = (tau - 0.5) / 3
    s = V.Solver(V.make_config(nx, ny, "srt", "f64", tau, body_force=(gx, 0.0)))
    with s:
        s.set_mask(chi)
        s.step(int(8 * H * H / nu))
        _, ux, _ = s.moments()
    ua = gx / (2 * nu) * (y - e) * (e + H - y)
    fl = chi[:, 0] == 0
    err = math.sqrt(((ux[:, 0] - ua)[fl] ** 2).sum() / (ua[fl] ** 2).sum())
    assert err < 1e-6


# -----------------------------------------------------------------------------
# Grouped launches (serving): identical alone and in the mix
# -----------------------------------------------------------------------------

def test_group_step_bitwise_equal_to_alone():
    specs = [
        ("srt", "f32", I.c1_circular_couette(), 37),
        ("mrt", "f32", I.cylinder_channel(300, 75, 12.0, 0.05, 150.0, 0, storage="f32"), 50),
        ("mrt", "f16", I.cylinder_channel(200, 50, 8.0, 0.05, 100.0, 0, storage="f16"), 23),
        ("srt", "f16", I.circular_couette(64, 12.0, 28.0, 0.01, 0.7, 0, "srt", "f16"), 50),
        ("mrt", "f64", I.circular_couette(40, 7.0, 17.0, 0.01, 0.9, 0, "mrt", "f64"), 11),
    ]
    import torch
    shared = torch.cuda.Stream()  # grouped solvers share one stream
    alone, mixed = [], []
    for coll, storage, w, n in specs:
        w.collision, w.storage = coll, storage
        alone.append(V.Solver.from_workload(w))
        mixed.append(V.Solver.from_workload(w, stream=shared))
    try:
        for s, (_, _, _, n) in zip(alone, specs):
            s.step(n)
        V.vplbm_group_step([s.h for s in mixed], [n for *_, n in specs])
        for a, b in zip(alone, mixed):
            assert a.t == b.t
            assert np.array_equal(a.populations(), b.populations())
            fa, fb = a.forces(), b.forces()
            for x, y in zip(fa, fb):
                assert np.array_equal(x, y)
    finally:
        for s in alone + mixed:
            s.close()


def test_launch_count_is_one_kernel_per_step():
    w = I.cylinder_channel(256, 64, 10.0, 0.05, 100.0, 0)
    with V.Solver.from_workload(w) as s:
        n0 = s.launches
        s.step(17)
        assert s.launches - n0 == 17
    w = I.moving_cylinder_channel(256, 64, 10.0, 0.05, 100.0, 0, period=100.0)
    with V.Solver.from_workload(w) as s:
        s.step(1)
        n0 = s.launches
        s.step(17)
        assert s.launches - n0 == 34  # mask update + fused step per step


def test_divergence_is_reported():
    """A non-finite population is flagged at the next synchronisation (a
    host-written input; no device fault involved)."""
    with V.Solver(V.make_config(32, 8, "srt", "f32")) as s:
        f = I.random_populations(32, 8, 3, 0.05)
        f[0, 3, 5] = np.nan
        s.set_populations(f)
        s.step(1)
        with pytest.raises(V.VplbmError) as e:
            s.synchronize()
        assert e.value.status == V.VPLBM_ERR_DIVERGED


@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
def test_device_seeded_initial_field_matches_host_generator(storage):
    """vplbm_set_initial_perturbation draws the same SplitMix64 field on the
    device as inputs.velocity_field on the host, bit for bit."""
    w = I.cylinder_channel(300, 70, 10.0, 0.05, 100.0, 0, storage=storage, perturbation=1e-4, seed=9)
    with V.Solver.from_workload(w) as a, V.Solver.from_workload(w, device_init=True) as b:
        assert np.array_equal(a.populations(), b.populations())
        a.step(20)
        b.step(20)
        assert np.array_equal(a.populations(), b.populations())


def test_forces_async_matches_forces():
    import torch
    w = I.cylinder_channel(256, 64, 10.0, 0.05, 100.0, 0)
    with V.Solver.from_workload(w) as a, V.Solver.from_workload(w) as b:
        a.step(37)
        b.step(37)
        fx, fy, ms = a.forces()
        rec = torch.empty((64, 3), dtype=torch.float64, pin_memory=True)
        n = V.vplbm_forces_async(b.h, rec.numpy())
        b.synchronize()
        r = rec.numpy()[:n]
        assert n == 37
        assert np.array_equal(r[:, 0], fx) and np.array_equal(r[:, 1], fy) and np.array_equal(r[:, 2], ms)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
def test_checkpoint_restart_is_bitwise(storage):
    """Save after n steps, run n more; a new solver loaded from the saved state
    and run n steps gives the same store and force records bit for bit
    (moving body: its motion and the rounding bits depend on the step index)."""
    w = I.moving_cylinder_channel(256, 64, 10.0, 0.05, 100.0, 0, period=500.0, storage=storage)
    chi = I.random_mask(256, 64, 3, 0.02)
    us = I.random_solid_velocity(256, 64, 4, 0.01)
    n = 40
    with V.Solver.from_workload(w) as a:
        a.set_mask(chi, us)
        a.step(n)
        a.forces()
        state = V.vplbm_save_state(a.h)
        a.step(n)
        fa = a.populations()
        ra = a.forces()
    with V.Solver.from_workload(w, with_initial_velocity=False) as b:
        V.vplbm_load_state(b.h, state)
        assert b.t == n
        b.step(n)
        assert np.array_equal(b.populations(), fa)
        for x, y in zip(b.forces(), ra):
            assert np.array_equal(x, y)
    with V.Solver(V.make_config(128, 64, "mrt", storage)) as c:
        with pytest.raises(V.VplbmError):
            V.vplbm_load_state(c.h, state)
