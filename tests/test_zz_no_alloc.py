"""The allocation-free step (vplbm_step_noalloc) against the regular solver.

vplbm_step_noalloc is for callers that cannot allocate device memory when
they step (graph capture, host callbacks, fixed-budget loops, frameworks that
own all allocations): it runs the same fused kernel on caller-owned buffers,
with its reduction scratch in a fixed array inside the library. Here the
caller's buffers are torch tensors, allocated by the test beforehand.

Two calls in a row (t = 0, then t = 1 on swapped buffers) must reproduce
vplbm_step's populations and per-step record, for every storage type and for
a row pitch that is not the library's own 128-byte rounding. Both paths run
the same kernel on the same arithmetic; the tolerances are the parity
tolerances of the other tests (FP64 1e-12 relative, FP32 4e-7, the 16-bit
forms one rounding step of a stored offset, forces 1e-5 relative); in
practice the results are identical.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
# population tolerance (max abs) per storage
TOL = {"f64": 1e-12, "f32": 4e-7, "f16": 3e-5, "bf16": 2.5e-4}
MAX_TILES = 43_491  # the fixed scratch's capacity, in fused-step tiles


@pytest.fixture(scope="module")
def V():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1812_05401_gb300 import build as B
    B.build()
    from paper_1812_05401_gb300 import vplbm
    L = vplbm.lib()
    L.vplbm_step_noalloc.argtypes = [C.POINTER(vplbm.vplbm_config), C.POINTER(vplbm.vplbm_body),
                                     C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
    L.vplbm_step_noalloc.restype = C.c_int
    return vplbm


def _dtype(storage):
    import torch
    return {"f64": torch.float64, "f32": torch.float32, "f16": torch.float16,
            "bf16": torch.bfloat16}[storage]


U_IN = (0.04, 0.0)  # the channel's inlet velocity in these tests
XI = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]])


def _ref(storage):
    """Per-direction reference of the 16-bit elements of a channel: half the
    inlet equilibrium's momentum term along x, (3/2) w xi_x u_in,x, rounded to
    multiples of 2^-28 (exact in FP32); zero for the other storages."""
    if storage not in ("f16", "bf16"):
        return np.zeros(9)
    r = 1.5 * W * XI[:, 0] * U_IN[0]
    return np.round(r * 2.0 ** 28) / 2.0 ** 28


def _store(f, storage):
    """The storage's elements of the FP64 populations f (those the solver
    holds: FP64 stores f, FP32 the offsets f - w, the 16-bit forms f - w
    minus the reference)."""
    import torch
    h = f if storage == "f64" else f - W[:, None, None] - _ref(storage)[:, None, None]
    return torch.from_numpy(h).to(_dtype(storage))


def _state(V, nx, ny, pitch, coll, storage):
    import torch
    chi = I.random_mask(nx, ny, 41, 0.1)
    us = I.random_solid_velocity(nx, ny, 42, 0.02)
    body = I.BodySpec(nx * 0.6, ny * 0.5, 9.0, omega=0.001)
    cfg = V.make_config(nx, ny, coll, storage, 0.6, bc="channel", u_in=U_IN)
    cfg.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ref = V.Solver(cfg, [body])
    ref.set_mask(chi, us)
    f0 = I.random_populations(nx, ny, 43, 0.05)
    ref.set_populations(f0)
    mask_host = np.zeros((ny, pitch), np.uint8)
    m = ref.mask()  # 0/1 view; rebuild the library's encoding for the caller's buffer
    yy, xx = np.mgrid[0:ny, 0:nx]
    in_body = (xx - body.cx) ** 2 + (yy - body.cy) ** 2 <= body.radius ** 2
    mask_host[:, :nx] = np.where(chi != 0, 255, np.where(in_body, 1, 0))
    assert np.array_equal(mask_host[:, :nx] != 0, m != 0)
    dev = torch.device("cuda")
    src = torch.zeros((9, ny, pitch), dtype=_dtype(storage), device=dev)
    src[:, :, :nx] = _store(ref.populations(), storage).to(dev)
    dst = torch.zeros_like(src)
    mask_d = torch.from_numpy(mask_host).to(dev)
    vt = torch.float64 if storage == "f64" else torch.float32  # double2 / float2 per node
    us_d = torch.zeros((ny, pitch, 2), dtype=vt, device=dev)
    us_d[:, :nx, :] = torch.from_numpy(np.moveaxis(us, 0, -1).copy()).to(vt).to(dev)
    record = torch.zeros(3, dtype=torch.float64, device=dev)
    flag = torch.zeros(1, dtype=torch.int32, device=dev)
    bodies = (V.vplbm_body * 1)(V.vplbm_body(body.cx, body.cy, body.radius, 0, 0, 0, body.omega, 0, 0))
    return cfg, ref, src, dst, mask_d, us_d, record, flag, bodies


def _populations(dst, nx, storage):
    h = dst[:, :, :nx].float().cpu().numpy()
    if storage == "f64":
        return dst[:, :, :nx].double().cpu().numpy()
    # the kernel's FP32 decode: element + reference, then w + that in FP64
    return (h + _ref(storage)[:, None, None].astype(np.float32)).astype(np.float64) + W[:, None, None]


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16"])
@pytest.mark.parametrize("coll", ["mrt", "srt"])
@pytest.mark.parametrize("pitch_rule", ["128-byte rows", "multiple of 8"])
def test_noalloc_step_matches_regular_step_twice(V, storage, coll, pitch_rule):
    import torch
    nx, ny = 300, 70
    esize = {"f64": 8, "f32": 4, "f16": 2, "bf16": 2}[storage]
    pitch = -(-nx * esize // 128) * 128 // esize if pitch_rule == "128-byte rows" else -(-nx // 8) * 8
    cfg, ref, src, dst, mask_d, us_d, record, flag, bodies = _state(V, nx, ny, pitch, coll, storage)
    L = V.lib()
    try:
        for t in range(2):
            st = L.vplbm_step_noalloc(C.byref(cfg), bodies, 1, src.data_ptr(), dst.data_ptr(),
                                      mask_d.data_ptr(), us_d.data_ptr(), pitch, t,
                                      record.data_ptr(), flag.data_ptr())
            assert st == V.VPLBM_OK
            ref.step(1)
            torch.cuda.synchronize()
            f_ref = ref.populations()
            f_new = _populations(dst, nx, storage)
            assert np.abs(f_new - f_ref).max() <= TOL[storage] * (np.abs(f_ref).max() if storage == "f64" else 1.0)
            fx, fy, ms = ref.forces()
            rec = record.cpu().numpy()
            assert rec[0] == pytest.approx(fx[-1], rel=1e-5, abs=1e-9)
            assert rec[1] == pytest.approx(fy[-1], rel=1e-5, abs=1e-9)
            assert rec[2] == pytest.approx(ms[-1], rel=1e-12)
            assert int(flag.item()) == 0
            src, dst = dst, src
    finally:
        ref.close()


def test_noalloc_unknown_labels_are_solids_at_rest(V):
    """A caller-written mask may hold labels the call has no body for (here 9
    and 200 with one body): such nodes are solid with u_s = 0, exactly as
    label 255 without a solid-velocity field."""
    import torch
    nx, ny, pitch = 300, 70, 304
    cfg, ref, src, dst, mask_d, us_d, record, flag, bodies = _state(V, nx, ny, pitch, "mrt", "f32")
    ref.close()
    L = V.lib()
    m = mask_d.clone()
    m[10:20, 40:60] = 9
    m[30:40, 100:130] = 200
    m255 = mask_d.clone()
    m255[10:20, 40:60] = 255
    m255[30:40, 100:130] = 255
    # without a solid-velocity field every 255 node is at rest too, so the two
    # masks describe the same solids
    out = []
    for mk in (m, m255):
        d = torch.zeros_like(dst)
        rec = torch.zeros(3, dtype=torch.float64, device=d.device)
        st = L.vplbm_step_noalloc(C.byref(cfg), bodies, 1, src.data_ptr(), d.data_ptr(), mk.data_ptr(),
                                  None, pitch, 0, rec.data_ptr(), None)
        assert st == V.VPLBM_OK
        torch.cuda.synchronize()
        out.append((d.cpu().numpy(), rec.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])
    assert np.isfinite(out[0][0]).all()


def test_noalloc_capacity_boundary(V):
    """The largest grid the fixed scratch holds (43,491 tiles of 128 x 32
    nodes, FP16) runs; one more tile is refused before anything runs. Both
    calls get buffers of the larger grid's full size, so the second call would
    stay in bounds even if it ran."""
    import torch
    ny = 32
    nx_ok, nx_over = 128 * MAX_TILES, 128 * (MAX_TILES + 1)
    dev = torch.device("cuda")
    src = torch.zeros((9, ny, nx_over), dtype=torch.float16, device=dev)
    dst = torch.zeros_like(src)
    mask = torch.zeros((ny, nx_over), dtype=torch.uint8, device=dev)
    rec = torch.zeros(3, dtype=torch.float64, device=dev)
    L = V.lib()
    try:
        for nx, want in ((nx_ok, V.VPLBM_OK), (nx_over, V.VPLBM_ERR_INVALID)):
            cfg = V.make_config(nx, ny, "mrt", "f16")
            st = L.vplbm_step_noalloc(C.byref(cfg), None, 0, src.data_ptr(), dst.data_ptr(),
                                      mask.data_ptr(), None, nx_over, 0, rec.data_ptr(), None)
            assert st == want, nx
        torch.cuda.synchronize()
        # rest state in, rest state out; the record counts every node's density
        assert float(dst[:, :, :nx_ok].abs().max()) == 0.0
        assert rec[2].item() == pytest.approx(nx_ok * ny, rel=1e-12)
    finally:
        del src, dst, mask
        torch.cuda.empty_cache()


def test_noalloc_config_without_solver_fields(V):
    """rho0 and force_ring_len describe a solver's own state; a config that
    leaves them zero is accepted."""
    import torch
    nx, ny = 64, 16
    cfg = V.make_config(nx, ny, "srt", "f32")
    cfg.rho0 = 0.0
    cfg.force_ring_len = 0
    dev = torch.device("cuda")
    src = torch.zeros((9, ny, nx), dtype=torch.float32, device=dev)
    dst = torch.ones_like(src)
    mask = torch.zeros((ny, nx), dtype=torch.uint8, device=dev)
    rec = torch.zeros(3, dtype=torch.float64, device=dev)
    st = V.lib().vplbm_step_noalloc(C.byref(cfg), None, 0, src.data_ptr(), dst.data_ptr(),
                                    mask.data_ptr(), None, nx, 0, rec.data_ptr(), None)
    assert st == V.VPLBM_OK
    torch.cuda.synchronize()
    assert float(dst.abs().max()) == 0.0
