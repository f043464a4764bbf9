"""GPU parity of the convective outlet (Section 3.3, after Yang) against the
oracle, and its state handling (grouped steps, checkpoint, refusal by the
allocation-free step).

Tolerances as in the other parity tests: FP64 storage 1e-12 relative over
long runs; FP32 a few 1e-7 per step on values <= 0.5; 16-bit offsets one
rounding step of |h| <= 0.06 plus FP32 arithmetic, for one step.
"""
import ctypes as C

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


def _pair(nx, ny, coll, storage, bc_y, uc, chi=None, us=None, bodies=(), tau=0.62):
    ocfg = O.Config(nx=nx, ny=ny, collision=O.MRT if coll == "mrt" else O.SRT, tau=tau,
                    bc_x=O.BC_INLET_CONVECTIVE, bc_y=bc_y, u_in=(0.04, 0.0), u_conv=uc,
                    chi=chi, us=us,
                    bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                                   b.outside) for b in bodies])
    vby = 2 if bc_y == O.BC_FREE_SLIP else 0
    cfg = V.make_config(nx, ny, coll, storage, tau, bc=(V.VPLBM_BC_INLET_CONVECTIVE, vby),
                        u_in=(0.04, 0.0), u_conv=uc, body_force=(1e-6, -2e-6))
    ocfg.g = (1e-6, -2e-6)
    s = V.Solver(cfg, list(bodies))
    if chi is not None:
        s.set_mask(chi, us)
    return ocfg, s


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("coll", ["srt", "mrt"])
@pytest.mark.parametrize("bc_y", [O.BC_FREE_SLIP, O.BC_PERIODIC])
def test_convective_outlet_random_state(storage, coll, bc_y):
    """Random state on a ragged grid (partial edge tiles, solids on the last
    column): several steps for FP64/FP32 (the state carries across steps and
    buffers), one for the 16-bit stores; the moments of the next step too."""
    nx, ny = 301, 37
    chi = I.random_mask(nx, ny, 51, 0.15)
    us = I.random_solid_velocity(nx, ny, 52, 0.03)
    bodies = [I.BodySpec(290.0, 18.0, 7.0, omega=0.002)]
    ocfg, s = _pair(nx, ny, coll, storage, bc_y, 0.05, chi, us, bodies)
    n = 1 if storage in ("f16", "bf16") else 3
    with s:
        s.set_populations(I.random_populations(nx, ny, 53, 0.05))
        f_ref = s.populations()
        ocfg.outlet = O.outlet_from_store(f_ref)
        fx_ref, _, m_ref = O.run(ocfg, f_ref, n)
        s.step(n)
        f = s.populations()
        fx, _, ms = s.forces()
        rho, _, _ = s.moments()
    # moments the next step computes, from the device's own store (this
    # compares the read-only outlet pull of the moments kernel)
    rho2, _, _ = O.moments(ocfg, f, n)
    if storage == "f64":
        assert np.abs(f - f_ref).max() / np.abs(f_ref).max() < 1e-14
        np.testing.assert_allclose(fx, fx_ref, rtol=1e-11)
        np.testing.assert_allclose(ms, m_ref, rtol=1e-14)
        assert np.abs(rho - rho2).max() < 1e-14
    elif storage == "f32":
        assert np.abs(f - f_ref).max() < 4e-7 * n
        assert np.abs(rho - rho2).max() < 2e-6
    else:
        ulp = 2.0 ** -10 if storage == "f16" else 2.0 ** -7
        assert np.abs(f - f_ref).max() < 0.06 * ulp + 1e-6
        assert np.abs(rho - rho2).max() < 2e-6


def test_convective_outlet_cylinder_fp64_long_run():
    """FP64, MRT cylinder channel with the convective outlet, 400 steps from
    a perturbed uniform flow: populations within 1e-12 of the oracle."""
    w = I.cylinder_channel(160, 48, 10.0, 0.05, 100.0, 400, xc=50.0, collision="mrt",
                           storage="f64", outlet="convective", seed=5)
    with V.Solver.from_workload(w) as s:
        s.step(w.steps)
        f = s.populations()
        fx, fy, _ = s.forces()
    cfg, bodies = V.config_from_workload(w)
    ocfg = O.Config(nx=w.nx, ny=w.ny, collision=O.MRT, tau=cfg.tau, lam=w.lam,
                    bc_x=O.BC_INLET_CONVECTIVE, bc_y=O.BC_FREE_SLIP, u_in=(0.05, 0.0),
                    u_conv=0.05, bodies=[O.Body(b.cx, b.cy, b.radius) for b in bodies])
    f_ref = O.init_equilibrium(ocfg, 1.0, w.initial_velocity())
    ocfg.outlet = O.outlet_from_store(f_ref)
    fx_ref, fy_ref, _ = O.run(ocfg, f_ref, w.steps)
    assert np.abs(f - f_ref).max() / np.abs(f_ref).max() < 1e-12
    assert np.abs(fx - fx_ref).max() < 1e-10 * np.abs(fx_ref).max()


def test_convective_outlet_differs_from_zero_gradient():
    """The two outlets are different conditions: with a wake reaching the
    outlet the stores differ, and the convective one matches its oracle."""
    base = dict(nx=96, ny=32, diameter=8.0, u_in=0.05, re=80.0, steps=300, xc=70.0,
                collision="srt", storage="f64", seed=6)
    out = []
    for outlet in ("zero-gradient", "convective"):
        w = I.cylinder_channel(outlet=outlet, **base)
        with V.Solver.from_workload(w) as s:
            s.step(w.steps)
            out.append(s.populations())
    assert np.abs(out[0] - out[1]).max() > 1e-6


def test_convective_outlet_group_and_checkpoint_bitwise():
    """Grouped steps use the outlet state of the right buffer (bitwise equal
    to stepping alone), and a checkpoint carries the state (restart is
    bitwise)."""
    import torch
    shared = torch.cuda.Stream()
    w = I.cylinder_channel(300, 75, 12.0, 0.05, 150.0, 0, xc=240.0, storage="f32",
                           outlet="convective", seed=7)
    w2 = I.cylinder_channel(200, 50, 8.0, 0.05, 100.0, 0, xc=160.0, storage="f32", seed=8)
    with V.Solver.from_workload(w) as a, V.Solver.from_workload(w, stream=shared) as b, \
            V.Solver.from_workload(w2, stream=shared) as c:
        a.step(37)
        V.vplbm_group_step([b.h, c.h], [37, 20])
        assert np.array_equal(a.populations(), b.populations())
        state = V.vplbm_save_state(a.h)
        a.step(25)
        fa = a.populations()
    with V.Solver.from_workload(w, with_initial_velocity=False) as d:
        V.vplbm_load_state(d.h, state)
        d.step(25)
        assert np.array_equal(d.populations(), fa)
    # a state saved with the convective outlet does not load into a solver without it
    w.outlet = "zero-gradient"
    with V.Solver.from_workload(w, with_initial_velocity=False) as e:
        with pytest.raises(V.VplbmError):
            V.vplbm_load_state(e.h, state)


def test_convective_outlet_rejected_by_noalloc_and_validation():
    """The allocation-free step has nowhere to keep the outlet state and
    refuses the convective outlet (before any launch; the buffers are real and
    sized for the grid all the same); a negative U_c is refused at creation."""
    import torch
    nx, ny, pitch = 64, 32, 64
    cfg = V.make_config(nx, ny, "srt", "f32", 0.7, bc="channel-convective", u_in=(0.05, 0.0))
    cfg.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = V.lib()
    L.vplbm_step_noalloc.argtypes = [C.POINTER(V.vplbm_config), C.POINTER(V.vplbm_body),
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
    L.vplbm_step_noalloc.restype = C.c_int
    dev = torch.device("cuda")
    src = torch.zeros((9, ny, pitch), dtype=torch.float32, device=dev)
    dst = torch.zeros_like(src)
    mask = torch.zeros((ny, pitch), dtype=torch.uint8, device=dev)
    record = torch.zeros(3, dtype=torch.float64, device=dev)
    st = L.vplbm_step_noalloc(C.byref(cfg), None, 0, src.data_ptr(), dst.data_ptr(),
                              mask.data_ptr(), None, pitch, 0, record.data_ptr(), None)
    assert st == V.VPLBM_ERR_INVALID
    bad = V.make_config(nx, ny, "srt", "f32", 0.7, bc="channel-convective", u_in=(0.05, 0.0),
                        u_conv=-1.0)
    with pytest.raises(V.VplbmError):
        V.Solver(bad)
