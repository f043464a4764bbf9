"""In-place (AA-pattern) streaming against the A/B scheme and the oracle.

The in-place scheme stores every value rounded with the same bits as the A/B
scheme (node, direction, step), so the bar is bitwise equality with A/B for
every storage: exported populations f*(t) after odd and even step counts (a
push step or a local step last), force and mass records, moments,
momentum-exchange forces, grouped stepping, checkpoints. FP64 runs are also
compared with the oracle directly (1e-12 relative).
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


BCS = {"periodic": (0, 0), "channel": (1, 2), "channel-convective": (3, 2),
       "inlet-periodic": (1, 0), "convective-periodic": (3, 0), "periodic-slip": (0, 2)}


def _solver(nx, ny, coll, storage, bc, streaming, bodies=(), chi=None, us=None, stream=None):
    cfg = V.make_config(nx, ny, coll, storage, 0.62, bc=BCS[bc], u_in=(0.04, 0.0),
                        body_force=(1e-6, -2e-6), streaming=streaming, ring_len=64, stream=stream)
    s = V.Solver(cfg, list(bodies))
    if chi is not None:
        s.set_mask(chi, us)
    return s


def _run_pair(nx, ny, coll, storage, bc, n, bodies, chi, us, seed, record_me=False):
    out = []
    for streaming in ("ab", "aa"):
        with _solver(nx, ny, coll, storage, bc, streaming, bodies, chi, us) as s:
            s.set_populations(I.random_populations(nx, ny, seed, 0.05))
            if record_me:
                s.record_momentum_exchange(True)
            s.step(n)
            r = {"f": s.populations(), "forces": s.forces(), "mom": s.moments(),
                 "me": s.momentum_exchange()}
            if record_me:
                r["me_rec"] = s.momentum_exchange_forces()
            out.append(r)
    return out


def _assert_same(a, b):
    assert np.array_equal(a["f"], b["f"])
    for x, y in zip(a["forces"], b["forces"]):
        assert np.array_equal(x, y)
    for x, y in zip(a["mom"], b["mom"]):
        assert np.array_equal(x, y)
    assert a["me"] == b["me"]
    if "me_rec" in a:
        for x, y in zip(a["me_rec"], b["me_rec"]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("coll", ["srt", "mrt"])
@pytest.mark.parametrize("bc", list(BCS))
@pytest.mark.parametrize("n", [1, 4])
def test_aa_bitwise_equal_to_ab(storage, coll, bc, n):
    """Ragged grid spanning interior and boundary tiles, random static mask,
    a rotating and a moving body, random populations."""
    nx, ny = 301, 70
    chi = I.random_mask(nx, ny, 61, 0.1)
    us = I.random_solid_velocity(nx, ny, 62, 0.03)
    bodies = [I.BodySpec(150.5, 35.0, 9.0, omega=0.002),
              I.BodySpec(60.0, 30.0, 6.0, amp_y=4.0, period=200.0)]
    ab, aa = _run_pair(nx, ny, coll, storage, bc, n, bodies, chi, us, 63, record_me=(n == 4))
    _assert_same(ab, aa)


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 5), (2, 3), (3, 130), (129, 2), (257, 33)])
@pytest.mark.parametrize("bc", ["periodic", "channel", "convective-periodic"])
def test_aa_edge_sizes_bitwise(nx, ny, bc):
    ab, aa = _run_pair(nx, ny, "mrt", "f32", bc, 3, [], None, None, 64)
    _assert_same(ab, aa)


def test_aa_fp64_against_oracle():
    """FP64 MRT channel with a cylinder, 301 steps in place (a push step
    last): populations within 1e-12 of the oracle."""
    w = I.cylinder_channel(160, 48, 10.0, 0.05, 100.0, 301, xc=50.0, collision="mrt",
                           storage="f64", seed=5)
    cfg, bodies = V.config_from_workload(w)
    cfg.streaming = V.VPLBM_STREAM_AA
    with V.Solver(cfg, bodies, w.initial_velocity()) as s:
        s.step(w.steps)
        f = s.populations()
    ocfg = O.Config(nx=w.nx, ny=w.ny, collision=O.MRT, tau=cfg.tau, lam=w.lam,
                    bc_x=O.BC_INLET_OUTLET, bc_y=O.BC_FREE_SLIP, u_in=(0.05, 0.0),
                    bodies=[O.Body(b.cx, b.cy, b.radius) for b in bodies])
    f_ref = O.init_equilibrium(ocfg, 1.0, w.initial_velocity())
    O.run(ocfg, f_ref, w.steps)
    assert np.abs(f - f_ref).max() / np.abs(f_ref).max() < 1e-12


def test_aa_grouped_and_checkpoint_bitwise():
    """In-place solvers at both phases grouped with A/B solvers of the same
    storage give the same stores as stepping alone; a checkpoint taken after
    a push step restarts bitwise; an in-place state does not load into an A/B
    solver."""
    import torch
    shared = torch.cuda.Stream()
    w = I.cylinder_channel(300, 75, 12.0, 0.05, 150.0, 0, xc=200.0, storage="f16",
                           outlet="convective", seed=7)

    def make(streaming, stream=None, pre=0):
        cfg, bodies = V.config_from_workload(w, stream=stream)
        cfg.streaming = {"ab": 0, "aa": 1}[streaming]
        s = V.Solver(cfg, bodies, w.initial_velocity())
        s.step(pre)
        return s

    with make("ab") as a0, make("ab", pre=1) as a1, make("aa", shared) as b0, \
            make("aa", shared, pre=1) as b1, make("ab", shared) as c:
        a0.step(23)
        a1.step(16)
        V.vplbm_group_step([b0.h, b1.h, c.h], [23, 16, 9])
        assert np.array_equal(a0.populations(), b0.populations())
        assert np.array_equal(a1.populations(), b1.populations())
        for x, y in zip(a0.forces(), b0.forces()):
            assert np.array_equal(x, y)
        state = V.vplbm_save_state(b0.h)  # after 23 steps: a push step last
        b0.step(12)
        fb = b0.populations()
    with make("aa") as d:
        V.vplbm_load_state(d.h, state)
        assert d.t == 23
        d.step(12)
        assert np.array_equal(d.populations(), fb)
    with make("ab") as e:
        with pytest.raises(V.VplbmError):
            V.vplbm_load_state(e.h, state)
