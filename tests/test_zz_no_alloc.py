"""The allocation-free step (vplbm_step_noalloc) against the regular solver.

vplbm_step_noalloc is for callers that cannot allocate device memory when
they step (graph capture, host callbacks, fixed-budget loops, frameworks that
own all allocations): it runs the same fused kernel on caller-owned buffers,
with its reduction scratch in a fixed array inside the library. Here the
caller's buffers are torch tensors, allocated by the test beforehand.

Two calls in a row (t = 0, then t = 1 on swapped buffers) must reproduce
vplbm_step's populations and per-step record. Both paths run the same kernel
on the same arithmetic, so the tolerance is the FP32 parity tolerance of the
other tests (4e-7 on populations, 1e-5 relative on forces); in practice the
results are identical.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1812_05401_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def _state(V, nx, ny, pitch, coll):
    import torch
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    chi = I.random_mask(nx, ny, 41, 0.1)
    us = I.random_solid_velocity(nx, ny, 42, 0.02)
    body = I.BodySpec(nx * 0.6, ny * 0.5, 9.0, omega=0.001)
    cfg = V.make_config(nx, ny, coll, "f32", 0.6, bc="channel", u_in=(0.04, 0.0))
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
    src = torch.zeros((9, ny, pitch), dtype=torch.float32, device=dev)
    # FP32 storage holds the offsets f - w
    src[:, :, :nx] = torch.from_numpy((ref.populations() - w[:, None, None]).astype(np.float32)).to(dev)
    dst = torch.zeros_like(src)
    mask_d = torch.from_numpy(mask_host).to(dev)
    us_d = torch.zeros((ny, pitch, 2), dtype=torch.float32, device=dev)
    us_d[:, :nx, :] = torch.from_numpy(np.moveaxis(us, 0, -1).astype(np.float32)).to(dev)
    record = torch.zeros(3, dtype=torch.float64, device=dev)
    flag = torch.zeros(1, dtype=torch.int32, device=dev)
    bodies = (V.vplbm_body * 1)(V.vplbm_body(body.cx, body.cy, body.radius, 0, 0, 0, body.omega, 0, 0))
    return cfg, ref, src, dst, mask_d, us_d, record, flag, bodies, w


@pytest.mark.parametrize("coll", ["mrt", "srt"])
def test_noalloc_step_matches_regular_step_twice(V, coll):
    import torch
    nx, ny, pitch = 300, 70, 320
    cfg, ref, src, dst, mask_d, us_d, record, flag, bodies, w = _state(V, nx, ny, pitch, coll)
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
            f_new = dst[:, :, :nx].double().cpu().numpy() + w[:, None, None]
            assert np.abs(f_new - f_ref).max() < 4e-7
            fx, fy, ms = ref.forces()
            rec = record.cpu().numpy()
            assert rec[0] == pytest.approx(fx[-1], rel=1e-5, abs=1e-9)
            assert rec[1] == pytest.approx(fy[-1], rel=1e-5, abs=1e-9)
            assert rec[2] == pytest.approx(ms[-1], rel=1e-12)
            assert int(flag.item()) == 0
            src, dst = dst, src
    finally:
        ref.close()


def test_noalloc_rejects_grids_beyond_its_scratch(V):
    """A grid of 43,776 tiles needs more than the fixed 1 MiB of reduction
    scratch and is refused before anything runs. The buffers passed are real
    and of the full size, so the call would stay in bounds even if it ran."""
    import torch
    nx, ny = 128 * 256, 32 * 171  # FP16 tiles are 128 x 32 nodes
    cfg = V.make_config(nx, ny, "mrt", "f16")
    dev = torch.device("cuda")
    src = torch.zeros((9, ny, nx), dtype=torch.float16, device=dev)
    dst = torch.zeros_like(src)
    mask = torch.zeros((ny, nx), dtype=torch.uint8, device=dev)
    rec = torch.zeros(3, dtype=torch.float64, device=dev)
    st = V.lib().vplbm_step_noalloc(C.byref(cfg), None, 0, src.data_ptr(), dst.data_ptr(),
                                    mask.data_ptr(), None, nx, 0, rec.data_ptr(), None)
    assert st == V.VPLBM_ERR_INVALID
    del src, dst, mask
    torch.cuda.empty_cache()
