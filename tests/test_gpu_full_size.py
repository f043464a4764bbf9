"""Parity at the benchmark's full size, in the configuration the benchmark
times: the 16384 x 4096 moving-cylinder channel (67.1M nodes, MRT), built and
stepped exactly as bench.py builds and steps it.

The oracle cannot run this grid, so it checks sampled outputs node by node
(orc_step_nodes: the oracle's pull with every boundary rule, mask and
collision for the listed nodes, from the GPU's own stored f*(t)): random
nodes, every kind of boundary node, tile-border nodes, the ring around the
moving body, and every solid node for the force record of the step.
Tolerances: FP32 storage 4e-7 on one step's populations (FP32 arithmetic on
values <= 0.5); FP16 and BF16 offsets (stochastically rounded) one rounding
step of each offset's own binade plus FP32 arithmetic; the force within 2e-5 relative
(FP32 node forces summed in FP64).
The in-place scheme is bitwise the A/B scheme at this size as well.
"""
import numpy as np
import pytest

import oracle as O
from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

V = None
WARMUP = 5  # bench.py's default warm-up steps: the checked step is step index 5


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


def _oracle_config(w, cfg):
    return O.Config(nx=w.nx, ny=w.ny, collision=O.MRT if w.collision == "mrt" else O.SRT,
                    tau=cfg.tau, lam=cfg.lam, eta=cfg.eta, bc_x=O.BC_INLET_OUTLET,
                    bc_y=O.BC_FREE_SLIP, u_in=(cfg.u_in[0], cfg.u_in[1]),
                    bodies=[O.Body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                                   b.outside) for b in w.bodies])


def _element_offset(f, u_in, axis):
    """|f - r| of each population: the magnitude a 16-bit element of a
    channel holds (r = w + (3/2) w xi_x u_in,x, the reference of the 16-bit
    stores when the flow has an inlet, before its rounding to a 2^-28 grid);
    its binade sets the rounding step."""
    xi = O.velocity_set().astype(float)
    w = O.weights()
    r = w + 1.5 * w * xi[:, 0] * float(u_in[0])
    shape = [1, 1, 1]
    shape[axis] = 9
    return np.abs(f - r.reshape(shape[:f.ndim]))


def _export(torch, s, nx, ny):
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    V.vplbm_populations(s.h, f, on_device=True)
    s.synchronize()
    return f


def _sample(w, t):
    """Sampled nodes: random, boundary, tile borders, ring around the body."""
    nx, ny = w.nx, w.ny
    rng = np.random.default_rng(20240)
    xs = [rng.integers(0, nx, 4096)]
    ys = [rng.integers(0, ny, 4096)]
    edge = rng.integers(0, max(nx, ny), 512)
    xs += [np.zeros(256, int), np.full(256, nx - 1), edge[:256] % nx, edge[256:] % nx]
    ys += [edge[:256] % ny, edge[256:] % ny, np.zeros(256, int), np.full(256, ny - 1)]
    xs.append(np.array([0, 0, nx - 1, nx - 1]))
    ys.append(np.array([0, ny - 1, 0, ny - 1]))
    tb = rng.integers(1, nx // 128, 512) * 128 + rng.integers(-1, 1, 512)  # tile borders
    xs.append(tb)
    ys.append(rng.integers(0, ny, 512))
    b = w.bodies[0]
    cy = b.cy + b.amp_y * np.sin(2 * np.pi * t / b.period)
    th = np.linspace(0.0, 2 * np.pi, 2400, endpoint=False)
    for dr in (-1.5, -0.5, 0.5, 1.5):
        xs.append(np.rint(b.cx + (b.radius + dr) * np.cos(th)).astype(int))
        ys.append(np.rint(cy + (b.radius + dr) * np.sin(th)).astype(int))
    x, y = np.concatenate(xs), np.concatenate(ys)
    ok = (x >= 0) & (x < nx) & (y >= 0) & (y < ny)
    return x[ok], y[ok]


def _solid_nodes(w, t):
    b = w.bodies[0]
    cy = b.cy + b.amp_y * np.sin(2 * np.pi * t / b.period)
    r = int(np.ceil(b.radius)) + 2
    yy, xx = np.mgrid[int(cy) - r:int(cy) + r + 2, int(b.cx) - r:int(b.cx) + r + 2]
    return xx.ravel(), yy.ravel()


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_bench_workload_sampled_against_oracle(storage):
    import torch
    w = I.c5_moving_cylinder(storage)
    nx, ny = w.nx, w.ny
    with V.Solver.from_workload(w, ring_len=4096) as s:
        cfg, _ = V.config_from_workload(w)
        s.step(WARMUP)
        f_t = _export(torch, s, nx, ny)
        s.step(1)
        fx, fy, _ = s.forces()
        f_t1 = _export(torch, s, nx, ny)
    t = WARMUP
    ocfg = _oracle_config(w, cfg)
    f_host = f_t.cpu().numpy()
    del f_t
    x, y = _sample(w, t)
    ref, _, _, _ = O.step_nodes(ocfg, f_host, t, x, y)
    xi = torch.as_tensor(x, device="cuda")
    yi = torch.as_tensor(y, device="cuda")
    got = f_t1[:, yi, xi].T.cpu().numpy()
    err = np.abs(got - ref)
    if storage == "f32":
        assert err.max() < 4e-7, err.max()
    else:
        # stochastic 16-bit rounding of the stored element f - r: less than
        # one rounding step of its binade (10 stored bits for FP16, 7 for
        # BF16), plus FP32 arithmetic
        h = _element_offset(ref, (w.u_ref, 0.0), 1)
        drop = 10 if storage == "f16" else 7
        step = 2.0 ** (np.floor(np.log2(np.maximum(h, 2.0 ** -14))) - drop)
        assert (err < step + 2e-6).all(), (err.max(), (err - step).max())
        assert h.max() < 0.5
    # the step's force record against the oracle's node forces over every solid node
    sx, sy = _solid_nodes(w, t)
    _, fpx, fpy, chi = O.step_nodes(ocfg, f_host, t, sx, sy)
    solid = chi.astype(bool)
    assert solid.sum() > 50_000
    ex, ey = -fpx[solid].sum(), -fpy[solid].sum()
    assert fx[-1] == pytest.approx(ex, rel=2e-5)
    assert fy[-1] == pytest.approx(ey, rel=2e-5, abs=2e-5 * abs(ex))


def test_bench_workload_in_place_bitwise():
    """The in-place side measurement's solver against the A/B one after an
    odd and an even number of steps (a push step and a local step last)."""
    import torch
    w = I.c5_moving_cylinder("f32")
    with V.Solver.from_workload(w, ring_len=64) as a, \
            V.Solver.from_workload(w, ring_len=64, streaming="aa") as b:
        for n in (WARMUP, 1):
            a.step(n)
            b.step(n)
            assert torch.equal(_export(torch, a, w.nx, w.ny), _export(torch, b, w.nx, w.ny))
            fa, fb = a.forces(), b.forces()
            for u, v in zip(fa, fb):
                assert np.array_equal(u, v)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
def test_cylinder_re1000_whole_grid_one_step(storage):
    """The bench's 4096 x 1024 cylinder workload is small enough for the
    oracle to step whole: every node of one step against the oracle, from the
    GPU's own stored state after the bench's warm-up."""
    import torch
    w = I.c3_cylinder_re1000(storage)
    cfg, _ = V.config_from_workload(w)
    with V.Solver.from_workload(w, ring_len=64) as s:
        s.step(WARMUP)
        f_t = _export(torch, s, w.nx, w.ny).cpu().numpy()
        s.step(1)
        f_gpu = _export(torch, s, w.nx, w.ny).cpu().numpy()
        fx, _, mass = s.forces()
    ocfg = _oracle_config(w, cfg)
    fx_ref, _, m_ref = O.run(ocfg, f_t, 1, t0=WARMUP)
    err = np.abs(f_gpu - f_t)
    if storage == "f32":
        assert err.max() < 4e-7
    else:
        h = _element_offset(f_t, (w.u_ref, 0.0), 0)
        drop = 10 if storage == "f16" else 7
        step = 2.0 ** (np.floor(np.log2(np.maximum(h, 2.0 ** -14))) - drop)
        assert (err < step + 2e-6).all()
    assert fx[-1] == pytest.approx(fx_ref[0], rel=2e-5)
    assert mass[-1] == pytest.approx(m_ref[0], rel=1e-7)


def test_grid_beyond_2_31_population_elements():
    """A 32768 x 8192 periodic grid (9 planes of 2^28 nodes: offsets past
    2^31 elements) started from a transverse plane shear wave
    u = U e sin(k.x), e perpendicular to k (its advective term vanishes, so it
    decays as exp(-nu |k|^2 t) exactly in the incompressible limit): every
    sampled velocity follows that decay and the total mass stays N. An index
    that wrapped at 32 bits would scramble whole population planes. The
    in-place scheme on the same grid gives bitwise the same moments after a
    local step and after a push step."""
    import torch
    nx, ny, U, n, tau = 32768, 8192, 0.01, 200, 0.8
    cfg = V.make_config(nx, ny, "mrt", "f32", tau, bc="periodic", ring_len=n + 8)
    kx, ky = 2 * np.pi * 8 / nx, 2 * np.pi * 4 / ny
    kk = np.hypot(kx, ky)
    ex, ey = ky / kk, -kx / kk
    phase = kx * np.arange(nx)[None, :] + ky * np.arange(ny)[:, None]
    u = np.empty((2, ny, nx))
    np.sin(phase, out=u[0])
    u[1] = u[0] * (U * ey)
    u[0] *= U * ex
    del phase

    def moments(s):
        m = torch.empty((3, ny, nx), dtype=torch.float64, device="cuda")
        V.vplbm_moments(s.h, m[0], m[1], m[2], on_device=True)
        s.synchronize()
        return m

    with V.Solver(cfg, [], u) as s:
        s.step(n)
        _, _, mass = s.forces()
        mom = moments(s)
        s.step(1)
        mom1 = moments(s)
    cfg.streaming = V.VPLBM_STREAM_AA
    with V.Solver(cfg, [], u) as s:
        del u
        s.step(n)
        assert torch.equal(moments(s), mom)
        s.step(1)
        assert torch.equal(moments(s), mom1)
    del mom1
    nu = (tau - 0.5) / 3.0
    rng = np.random.default_rng(7)
    xs, ys = rng.integers(0, nx, 20000), rng.integers(0, ny, 20000)
    xs[:4], ys[:4] = [0, nx - 1, 0, nx - 1], [0, 0, ny - 1, ny - 1]
    xi, yi = torch.as_tensor(xs, device="cuda"), torch.as_tensor(ys, device="cuda")
    ux = mom[1][yi, xi].cpu().numpy()
    uy = mom[2][yi, xi].cpu().numpy()
    amp = U * np.sin(kx * xs + ky * ys) * np.exp(-nu * kk * kk * n)
    assert np.abs(ux - ex * amp).max() < 2e-6, np.abs(ux - ex * amp).max()
    assert np.abs(uy - ey * amp).max() < 2e-6, np.abs(uy - ey * amp).max()
    assert np.abs(mass / (nx * ny) - 1.0).max() < 1e-6
