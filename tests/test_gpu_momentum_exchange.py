"""GPU parity of the momentum-exchange force (Section 3.3) against the oracle.

The GPU reduction and the oracle read the same stored values (the oracle gets
the store as exported, so the 16-bit and FP32 offsets enter both exactly); the
two differ only in summation order, so every storage is held to 1e-12
relative to the sum of the link magnitudes. Per-step records of an FP64 run
are held to the FP64 trajectory tolerance (1e-10 relative to the force scale).
"""
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


BC = {"periodic": ((O.BC_PERIODIC, O.BC_PERIODIC), (0, 0)),
      "channel": ((O.BC_INLET_OUTLET, O.BC_FREE_SLIP), (1, 2)),
      "periodic-slip": ((O.BC_PERIODIC, O.BC_FREE_SLIP), (0, 2))}


def _pair(nx, ny, storage, bc, bodies=(), chi=None, us=None, coll="mrt", tau=0.62):
    (obx, oby), vbc = BC[bc]
    ocfg = O.Config(nx=nx, ny=ny, collision=O.MRT if coll == "mrt" else O.SRT, tau=tau,
                    bc_x=obx, bc_y=oby, u_in=(0.04, 0.0), chi=chi, us=us,
                    bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                                   b.outside) for b in bodies])
    cfg = V.make_config(nx, ny, coll, storage, tau, bc=vbc, u_in=(0.04, 0.0), ring_len=64)
    s = V.Solver(cfg, list(bodies))
    if chi is not None:
        s.set_mask(chi, us)
    return ocfg, s


def _link_scale(f, chi):
    """Sum of |f| over the populations that can enter a link (an upper bound
    of the sum of the terms' magnitudes)."""
    return float(np.abs(f).sum())


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("bc", ["periodic", "channel", "periodic-slip"])
def test_momentum_exchange_random_state(storage, bc):
    """Random static mask (solids on every edge and across the periodic
    seams), a rotating body, random populations: one on-demand evaluation."""
    nx, ny = 300, 37
    chi = I.random_mask(nx, ny, 21, 0.15)
    us = I.random_solid_velocity(nx, ny, 22, 0.03)
    bodies = [I.BodySpec(200.5, 18.0, 7.0, omega=0.002)]
    ocfg, s = _pair(nx, ny, storage, bc, bodies, chi, us)
    with s:
        s.set_populations(I.random_populations(nx, ny, 23, 0.05))
        f = s.populations()  # as stored
        fx, fy = s.momentum_exchange()
    ex, ey = O.momentum_exchange(ocfg, f, 0)
    tol = 1e-12 * _link_scale(f, chi)
    assert abs(fx - ex) < tol and abs(fy - ey) < tol, (fx, ex, fy, ey)
    assert abs(ex) + abs(ey) > 1e-3  # a nontrivial sum


def test_momentum_exchange_body_only_box():
    """A body without a static layer: the reduction covers only its box; a
    small body far from the origin on a large grid still gets every link."""
    nx, ny = 1000, 300
    bodies = [I.BodySpec(701.3, 150.2, 9.4, omega=0.001)]
    ocfg, s = _pair(nx, ny, "f32", "channel", bodies)
    with s:
        s.set_populations(I.random_populations(nx, ny, 31, 0.05))
        f = s.populations()
        fx, fy = s.momentum_exchange()
    ex, ey = O.momentum_exchange(ocfg, f, 0)
    assert abs(fx - ex) < 1e-12 * _link_scale(f, None)
    assert abs(fy - ey) < 1e-12 * _link_scale(f, None)
    assert abs(ex) > 1e-3


def test_momentum_exchange_no_solids_is_zero():
    ocfg, s = _pair(64, 40, "f32", "periodic")
    with s:
        s.set_populations(I.random_populations(64, 40, 5, 0.05))
        assert s.momentum_exchange() == (0.0, 0.0)


def test_momentum_exchange_records_follow_oracle_trajectory():
    """FP64, a moving cylinder in a channel: the per-step records (taken from
    f*(t) with the mask of step t) against the oracle along its own run."""
    nx, ny = 160, 64
    bodies = [I.BodySpec(60.0, 31.5, 8.0, amp_y=6.0, period=400.0)]
    ocfg, s = _pair(nx, ny, "f64", "channel", bodies)
    u = I.velocity_field(nx, ny, (0.04, 0.0), 5e-3, seed=4)
    n = 60
    with s:
        s.set_initial_velocity(u)
        f = O.init_equilibrium(ocfg, 1.0, u)
        s.record_momentum_exchange(True)
        s.step(n)
        fx, fy = s.momentum_exchange_forces()
        ref = []
        for t in range(n):
            ref.append(O.momentum_exchange(ocfg, f, t))
            O.run(ocfg, f, 1, t0=t)
    ref = np.array(ref)
    assert len(fx) == n
    scale = np.abs(ref).max()
    assert np.abs(fx - ref[:, 0]).max() < 1e-10 * scale
    assert np.abs(fy - ref[:, 1]).max() < 1e-10 * scale


def test_momentum_exchange_records_bitwise_and_grouped():
    """Two identical runs give bitwise equal records; a recording solver in
    vplbm_group_step (stepped alone inside the group) gives the same records
    as vplbm_step, and the solvers grouped with it are unaffected."""
    import torch
    nx, ny = 257, 70
    bodies = [I.BodySpec(90.0, 35.0, 10.0, amp_y=5.0, period=300.0, omega=0.001)]
    stream = torch.cuda.Stream()

    def make(record):
        cfg = V.make_config(nx, ny, "mrt", "f32", 0.6, bc=(1, 2), u_in=(0.05, 0.0), ring_len=64)
        cfg.stream = stream.cuda_stream
        s = V.Solver(cfg, list(bodies))
        s.set_initial_velocity(I.velocity_field(nx, ny, (0.05, 0.0), 5e-3, seed=9))
        if record:
            s.record_momentum_exchange(True)
        return s

    with make(True) as a, make(True) as b, make(True) as c, make(False) as d, make(False) as e:
        a.step(40)
        b.step(40)
        V.vplbm_group_step([c.h, d.h], [40, 40])
        e.step(40)
        ra, rb, rc = a.momentum_exchange_forces(), b.momentum_exchange_forces(), \
            c.momentum_exchange_forces()
        assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])
        assert np.array_equal(ra[0], rc[0]) and np.array_equal(ra[1], rc[1])
        assert np.array_equal(d.populations(), e.populations())
        assert np.array_equal(a.populations(), c.populations())


def test_momentum_exchange_recording_window_and_state_errors():
    """Records start at the step recording is enabled; reading without ever
    enabling is a state error; a ring shorter than the unread steps keeps the
    newest records."""
    nx, ny = 96, 40
    bodies = [I.BodySpec(30.0, 19.5, 6.0)]
    cfg = V.make_config(nx, ny, "srt", "f64", 0.7, bc=(1, 2), u_in=(0.04, 0.0), ring_len=8)
    with V.Solver(cfg, bodies) as s:
        with pytest.raises(RuntimeError):
            s.momentum_exchange_forces()
        s.step(5)
        s.record_momentum_exchange(True)
        s.step(3)
        fx, _ = s.momentum_exchange_forces()
        assert len(fx) == 3
        s.step(20)  # more than the ring holds
        fx2, _ = s.momentum_exchange_forces()
        assert len(fx2) == 8
        f_now = s.populations()
        # the newest record is the one of step 27, computed from f*(27) --
        # step once more and compare it with an on-demand value at step 28
        on_demand = s.momentum_exchange()
        s.step(1)
        fx3, fy3 = s.momentum_exchange_forces()
        assert (fx3[0], fy3[0]) == on_demand
        assert f_now.shape == (9, ny, nx)
        s.record_momentum_exchange(False)
        s.step(2)
        assert len(s.momentum_exchange_forces()[0]) == 0
