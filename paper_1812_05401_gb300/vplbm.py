"""Thin ctypes binding of the vplbm C ABI (include/vplbm.h).

Functions keep the C names and only marshal arguments; every step of the time
step runs in the CUDA library. There is no fallback: if libvplbm.so is missing
or cannot be loaded, loading raises.

`Solver` is a small convenience wrapper over the same calls (numpy arrays in,
numpy arrays out, torch streams accepted). `config_from_workload` turns a
workload description (paper_1812_05401_gb300.inputs.Workload) into a
vplbm_config plus rigid bodies.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libvplbm.so")

VPLBM_OK, VPLBM_ERR_INVALID, VPLBM_ERR_NOMEM, VPLBM_ERR_CUDA = 0, 1, 2, 3
VPLBM_ERR_DIVERGED, VPLBM_ERR_TIMEOUT, VPLBM_ERR_STATE = 4, 5, 6
VPLBM_SRT, VPLBM_MRT = 0, 1
VPLBM_F64, VPLBM_F32, VPLBM_F16_OFFSET, VPLBM_BF16_OFFSET = 0, 1, 2, 3
VPLBM_BC_PERIODIC, VPLBM_BC_INLET_OUTLET, VPLBM_BC_FREE_SLIP, VPLBM_BC_INLET_CONVECTIVE = 0, 1, 2, 3
VPLBM_STREAM_AB, VPLBM_STREAM_AA = 0, 1
VPLBM_MAX_BODIES = 8
VPLBM_ROUND_NEAREST, VPLBM_ROUND_STOCHASTIC = 0, 1

STORAGE = {"f64": VPLBM_F64, "f32": VPLBM_F32, "f16": VPLBM_F16_OFFSET, "bf16": VPLBM_BF16_OFFSET}
COLLISION = {"srt": VPLBM_SRT, "mrt": VPLBM_MRT}
BYTES_PER_VALUE = {VPLBM_F64: 8, VPLBM_F32: 4, VPLBM_F16_OFFSET: 2, VPLBM_BF16_OFFSET: 2}


class vplbm_body(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("radius", C.c_double),
                ("amp_x", C.c_double), ("amp_y", C.c_double), ("period", C.c_double),
                ("omega", C.c_double), ("outside", C.c_int32), ("reserved", C.c_int32)]


# the device memory hook of vplbm_config: void* dev_alloc(size_t, void*), void dev_free(void*, void*)
DEV_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
DEV_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class vplbm_config(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("collision", C.c_int32),
                ("storage", C.c_int32), ("bc_x", C.c_int32), ("bc_y", C.c_int32),
                ("use_rates", C.c_int32), ("reduce_mass", C.c_int32),
                ("tau", C.c_double), ("lam", C.c_double), ("eta", C.c_double),
                ("u_in", C.c_double * 2), ("rho0", C.c_double), ("u0", C.c_double * 2),
                ("body_force", C.c_double * 2), ("rates", C.c_double * 9),
                ("force_ring_len", C.c_int32), ("rounding", C.c_int32), ("stream", C.c_void_p),
                ("u_conv", C.c_double), ("streaming", C.c_int32), ("tile_rows", C.c_int32),
                ("dev_alloc", DEV_ALLOC_FN), ("dev_free", DEV_FREE_FN), ("alloc_ctx", C.c_void_p),
                ("rounding_seed", C.c_uint32), ("reserved", C.c_uint32)]


class VplbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_lock = threading.Lock()


def lib() -> C.CDLL:
    """Loads libvplbm.so; raises if it is not built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_1812_05401_gb300.build.build() "
                              "(the CUDA library has no fallback)")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.vplbm_config_init.argtypes = [C.POINTER(vplbm_config)]
        L.vplbm_config_init.restype = None
        L.vplbm_tau_from_reynolds.argtypes = [C.c_double] * 3
        L.vplbm_tau_from_reynolds.restype = C.c_double
        L.vplbm_footprint_bytes.argtypes = [C.POINTER(vplbm_config)]
        L.vplbm_footprint_bytes.restype = C.c_size_t
        L.vplbm_create.argtypes = [C.POINTER(vplbm_config), C.POINTER(P)]
        L.vplbm_set_initial_velocity.argtypes = [P, dp]
        L.vplbm_set_initial_perturbation.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_uint64]
        L.vplbm_forces_async.argtypes = [P, dp, C.c_int64, C.POINTER(C.c_int64)]
        L.vplbm_state_bytes.argtypes = [P]
        L.vplbm_state_bytes.restype = C.c_size_t
        L.vplbm_save_state.argtypes = [P, P, C.c_size_t]
        L.vplbm_load_state.argtypes = [P, P, C.c_size_t]
        L.vplbm_set_mask_and_solid_velocity.argtypes = [P, P, P, C.c_int32]
        L.vplbm_set_bodies.argtypes = [P, C.POINTER(vplbm_body), C.c_int32]
        L.vplbm_step.argtypes = [P, C.c_int64]
        L.vplbm_synchronize.argtypes = [P]
        L.vplbm_step_count.argtypes = [P]
        L.vplbm_step_count.restype = C.c_int64
        L.vplbm_moments.argtypes = [P, P, P, P, C.c_int32]
        L.vplbm_populations.argtypes = [P, P, C.c_int32]
        L.vplbm_set_populations.argtypes = [P, P, C.c_int32]
        L.vplbm_mask.argtypes = [P, P]
        L.vplbm_forces.argtypes = [P, dp, dp, dp, C.c_int64, C.POINTER(C.c_int64)]
        L.vplbm_momentum_exchange.argtypes = [P, dp, dp]
        L.vplbm_enable_momentum_exchange.argtypes = [P, C.c_int32]
        L.vplbm_momentum_exchange_forces.argtypes = [P, dp, dp, C.c_int64, C.POINTER(C.c_int64)]
        L.vplbm_group_step.argtypes = [C.POINTER(P), C.c_int32, C.POINTER(C.c_int64)]
        L.vplbm_launch_count.argtypes = [P]
        L.vplbm_launch_count.restype = C.c_int64
        L.vplbm_enable_timing.argtypes = [P, C.c_int32]
        L.vplbm_fused_timing.argtypes = [P, dp, C.POINTER(C.c_int64)]
        L.vplbm_last_error.argtypes = [P]
        L.vplbm_last_error.restype = C.c_char_p
        L.vplbm_create_error.argtypes = []
        L.vplbm_create_error.restype = C.c_char_p
        L.vplbm_status_string.argtypes = [C.c_int]
        L.vplbm_status_string.restype = C.c_char_p
        L.vplbm_destroy.argtypes = [P]
        L.vplbm_destroy.restype = None
        for name in ("vplbm_create", "vplbm_set_initial_velocity", "vplbm_set_initial_perturbation",
                     "vplbm_forces_async", "vplbm_save_state", "vplbm_load_state",
                     "vplbm_set_mask_and_solid_velocity",
                     "vplbm_set_bodies", "vplbm_step", "vplbm_synchronize", "vplbm_moments",
                     "vplbm_populations", "vplbm_set_populations", "vplbm_mask", "vplbm_forces",
                     "vplbm_group_step", "vplbm_enable_timing", "vplbm_fused_timing",
                     "vplbm_momentum_exchange", "vplbm_enable_momentum_exchange",
                     "vplbm_momentum_exchange_forces"):
            getattr(L, name).restype = C.c_int
        _lib = L
        return L


# ---------------------------------------------------------------------------
# C-named wrappers (argument marshalling only)
# ---------------------------------------------------------------------------

def vplbm_config_init() -> vplbm_config:
    c = vplbm_config()
    lib().vplbm_config_init(C.byref(c))
    return c


def vplbm_tau_from_reynolds(u_ref: float, l_ref: float, re: float) -> float:
    return lib().vplbm_tau_from_reynolds(u_ref, l_ref, re)


def vplbm_footprint_bytes(cfg: vplbm_config) -> int:
    return int(lib().vplbm_footprint_bytes(C.byref(cfg)))


def _check(handle, st: int, what: str):
    if st != VPLBM_OK:
        msg = lib().vplbm_last_error(handle).decode() if handle else ""
        raise VplbmError(st, f"{what}: {lib().vplbm_status_string(st).decode()} {msg}".strip())


# Grid of each handle made by vplbm_create here, for the buffer checks below.
_grids: dict = {}


def vplbm_create(cfg: vplbm_config) -> int:
    h = C.c_void_p()
    st = lib().vplbm_create(C.byref(cfg), C.byref(h))
    if st != VPLBM_OK:
        why = lib().vplbm_create_error().decode()
        raise VplbmError(st, f"vplbm_create: {lib().vplbm_status_string(st).decode()}: {why}")
    _grids[h.value] = (cfg.nx, cfg.ny)
    return h.value


def _ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _dev(t):
    return C.c_void_p(t.data_ptr())


def _buffer(h, a, per_node: int, dtype, on_device: bool, what: str, write: bool = False):
    """Refuses, before the library sees it, a buffer that it would read or
    write past the end of: the C calls take bare pointers and fill whole
    fields ([per_node][ny][nx] elements). Checks the element type, that the
    memory is contiguous (and writable for an output), that a device buffer
    is a CUDA tensor and a host buffer a numpy array, and the element count
    when the handle's grid is known."""
    if on_device:
        import torch
        tdt = {np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        ok = isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == tdt and a.is_contiguous()
        n = a.numel() if ok else 0
    else:
        ok = (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous
              and (a.flags.writeable or not write))
        n = a.size if ok else 0
    grid = _grids.get(h)
    need = None if grid is None else per_node * grid[0] * grid[1]
    if not ok or (need is not None and n != need):
        kind = "CUDA tensor" if on_device else "numpy array"
        size = "" if need is None else f" of {need} elements"
        raise ValueError(f"{what}: needs a contiguous{' writable' if write else ''} "
                         f"{np.dtype(dtype).name} {kind}{size}")


def vplbm_set_initial_velocity(h, u=None):
    dp = None
    if u is not None:
        u = np.ascontiguousarray(u, dtype=np.float64)
        _buffer(h, u, 2, np.float64, False, "vplbm_set_initial_velocity")
        dp = u.ctypes.data_as(C.POINTER(C.c_double))
    _check(h, lib().vplbm_set_initial_velocity(h, dp), "vplbm_set_initial_velocity")


def vplbm_set_initial_perturbation(h, u0x: float, u0y: float, amp: float, seed: int):
    _check(h, lib().vplbm_set_initial_perturbation(h, u0x, u0y, amp, int(seed) & ((1 << 64) - 1)),
           "vplbm_set_initial_perturbation")


def vplbm_forces_async(h, records) -> int:
    """records: page-locked float64 array [cap][3] (e.g. a pinned torch
    tensor's numpy view); valid once the solver's stream reaches this point."""
    if not (isinstance(records, np.ndarray) and records.dtype == np.float64 and records.ndim == 2
            and records.shape[1] == 3 and records.flags.c_contiguous and records.flags.writeable):
        raise ValueError("vplbm_forces_async: needs a contiguous writable float64 array [cap][3]")
    cnt = C.c_int64()
    _check(h, lib().vplbm_forces_async(h, records.ctypes.data_as(C.POINTER(C.c_double)),
                                       records.shape[0], C.byref(cnt)), "vplbm_forces_async")
    return cnt.value


def vplbm_state_bytes(h) -> int:
    return int(lib().vplbm_state_bytes(h))


def vplbm_save_state(h) -> bytes:
    n = vplbm_state_bytes(h)
    buf = (C.c_char * n)()
    _check(h, lib().vplbm_save_state(h, buf, n), "vplbm_save_state")
    return bytes(buf)


def vplbm_load_state(h, state: bytes):
    buf = (C.c_char * max(1, len(state))).from_buffer_copy(bytes(state) or b"\0")
    _check(h, lib().vplbm_load_state(h, buf, len(state)), "vplbm_load_state")


def vplbm_set_mask_and_solid_velocity(h, chi, us=None, on_device: bool = False):
    what = "vplbm_set_mask_and_solid_velocity"
    if on_device:
        _buffer(h, chi, 1, np.uint8, True, what)
        if us is not None:
            _buffer(h, us, 2, np.float64, True, what)
        _check(h, lib().vplbm_set_mask_and_solid_velocity(
            h, _dev(chi), None if us is None else _dev(us), 1), "vplbm_set_mask_and_solid_velocity")
        return
    chi = np.ascontiguousarray(chi, dtype=np.uint8)
    us = None if us is None else np.ascontiguousarray(us, dtype=np.float64)
    _buffer(h, chi, 1, np.uint8, False, what)
    if us is not None:
        _buffer(h, us, 2, np.float64, False, what)
    _check(h, lib().vplbm_set_mask_and_solid_velocity(h, _ptr(chi), _ptr(us), 0),
           "vplbm_set_mask_and_solid_velocity")


def vplbm_set_bodies(h, bodies):
    arr = (vplbm_body * max(1, len(bodies)))()
    for i, b in enumerate(bodies):
        arr[i] = vplbm_body(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period, b.omega,
                            int(b.outside), 0)
    _check(h, lib().vplbm_set_bodies(h, arr, len(bodies)), "vplbm_set_bodies")


def vplbm_step(h, n: int):
    _check(h, lib().vplbm_step(h, int(n)), "vplbm_step")


def vplbm_synchronize(h):
    _check(h, lib().vplbm_synchronize(h), "vplbm_synchronize")


def vplbm_step_count(h) -> int:
    return int(lib().vplbm_step_count(h))


def vplbm_moments(h, rho, ux, uy, on_device: bool = False):
    for a in (rho, ux, uy):
        _buffer(h, a, 1, np.float64, on_device, "vplbm_moments", write=True)
    if on_device:
        _check(h, lib().vplbm_moments(h, _dev(rho), _dev(ux), _dev(uy), 1), "vplbm_moments")
    else:
        _check(h, lib().vplbm_moments(h, _ptr(rho), _ptr(ux), _ptr(uy), 0), "vplbm_moments")


def vplbm_populations(h, f, on_device: bool = False):
    _buffer(h, f, 9, np.float64, on_device, "vplbm_populations", write=True)
    _check(h, lib().vplbm_populations(h, _dev(f) if on_device else _ptr(f), int(on_device)),
           "vplbm_populations")


def vplbm_set_populations(h, f, on_device: bool = False):
    if not on_device:
        f = np.ascontiguousarray(f, dtype=np.float64)
    _buffer(h, f, 9, np.float64, on_device, "vplbm_set_populations")
    _check(h, lib().vplbm_set_populations(h, _dev(f) if on_device else _ptr(f), int(on_device)),
           "vplbm_set_populations")


def vplbm_mask(h, chi):
    _buffer(h, chi, 1, np.uint8, False, "vplbm_mask", write=True)
    _check(h, lib().vplbm_mask(h, _ptr(chi)), "vplbm_mask")


def vplbm_forces(h, cap: int):
    fx, fy, ms = np.zeros(cap), np.zeros(cap), np.zeros(cap)
    cnt = C.c_int64()
    dp = C.POINTER(C.c_double)
    _check(h, lib().vplbm_forces(h, fx.ctypes.data_as(dp), fy.ctypes.data_as(dp),
                                 ms.ctypes.data_as(dp), cap, C.byref(cnt)), "vplbm_forces")
    k = cnt.value
    return fx[:k], fy[:k], ms[:k]


def vplbm_momentum_exchange(h):
    fx, fy = C.c_double(), C.c_double()
    _check(h, lib().vplbm_momentum_exchange(h, C.byref(fx), C.byref(fy)), "vplbm_momentum_exchange")
    return fx.value, fy.value


def vplbm_enable_momentum_exchange(h, enable: bool = True):
    _check(h, lib().vplbm_enable_momentum_exchange(h, 1 if enable else 0),
           "vplbm_enable_momentum_exchange")


def vplbm_momentum_exchange_forces(h, cap: int):
    fx, fy = np.zeros(cap), np.zeros(cap)
    cnt = C.c_int64()
    dp = C.POINTER(C.c_double)
    _check(h, lib().vplbm_momentum_exchange_forces(h, fx.ctypes.data_as(dp), fy.ctypes.data_as(dp),
                                                   cap, C.byref(cnt)),
           "vplbm_momentum_exchange_forces")
    k = cnt.value
    return fx[:k], fy[:k]


def vplbm_group_step(handles, steps):
    n = len(handles)
    arr = (C.c_void_p * max(1, n))(*handles)
    st = (C.c_int64 * max(1, n))(*[int(s) for s in steps])
    _check(handles[0] if n else None, lib().vplbm_group_step(arr, n, st), "vplbm_group_step")


def vplbm_launch_count(h) -> int:
    return int(lib().vplbm_launch_count(h))


def vplbm_enable_timing(h, enable: bool = True):
    _check(h, lib().vplbm_enable_timing(h, int(enable)), "vplbm_enable_timing")


def vplbm_fused_timing(h):
    ms = C.c_double()
    n = C.c_int64()
    _check(h, lib().vplbm_fused_timing(h, C.byref(ms), C.byref(n)), "vplbm_fused_timing")
    return ms.value, n.value


def vplbm_last_error(h) -> str:
    return lib().vplbm_last_error(h).decode()


def vplbm_destroy(h):
    lib().vplbm_destroy(h)
    _grids.pop(h, None)


# ---------------------------------------------------------------------------
# Convenience wrapper
# ---------------------------------------------------------------------------

class TorchAllocator:
    """The device memory hook of vplbm_config served by PyTorch's caching
    allocator: blocks come from torch.cuda.caching_allocator_alloc and go back
    through caching_allocator_delete, so a solver's buffers count in
    torch.cuda.memory_allocated and share PyTorch's pool. Keeps counts of the
    calls (allocs, frees) and of the bytes it has out (live_bytes).

    The caching allocator reuses a block in stream order only on the stream it
    was allocated for, so the allocator and the solver share one stream:
    `stream` (a torch.cuda.Stream or a raw handle), else the config's stream
    at install(), else a new torch.cuda.Stream (never the legacy NULL stream,
    for which the library would create a private stream of its own).

    A config carrying the hook holds a reference to this object; keep the
    config (a Solver does) or the allocator alive while a solver created with
    it exists."""

    def __init__(self, stream=None, device=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self._stream_obj = stream
        self.stream = None if stream is None else int(getattr(stream, "cuda_stream", stream))
        self.allocs = 0
        self.frees = 0
        self.live_bytes = 0
        self._sizes = {}
        self._alloc = DEV_ALLOC_FN(self._do_alloc)
        self._free = DEV_FREE_FN(self._do_free)

    def _do_alloc(self, nbytes, _ctx):
        try:
            ptr = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except Exception:  # out of memory (or any failure): the library reports NOMEM
            return None
        self.allocs += 1
        self._sizes[ptr] = int(nbytes)
        self.live_bytes += int(nbytes)
        return ptr

    def _do_free(self, ptr, _ctx):
        try:
            self._torch.cuda.caching_allocator_delete(ptr)
        except Exception:  # interpreter shutdown: the process is ending anyway
            return
        self.frees += 1
        self.live_bytes -= self._sizes.pop(ptr, 0)

    def install(self, cfg: vplbm_config) -> vplbm_config:
        if self.stream is None:
            if cfg.stream:
                self.stream = int(cfg.stream)
            else:
                self._stream_obj = self._torch.cuda.Stream(self.device)
                self.stream = self._stream_obj.cuda_stream
        if self.stream == 0:
            raise ValueError("the legacy default stream cannot carry a solver with this allocator")
        if cfg.stream and int(cfg.stream) != self.stream:
            raise ValueError("the allocator's stream must be the solver's stream")
        cfg.stream = C.c_void_p(self.stream)
        cfg.dev_alloc = self._alloc
        cfg.dev_free = self._free
        cfg.alloc_ctx = None
        cfg._allocator = self  # the callbacks live as long as the config
        return cfg


def make_config(nx, ny, collision="srt", storage="f32", tau=0.8, lam=3.0 / 16.0, eta=1e-7,
                bc="periodic", u_in=(0.0, 0.0), u0=(0.0, 0.0), rho0=1.0, body_force=(0.0, 0.0),
                rates=None, reduce_mass=True, ring_len=4096, stream=None,
                rounding="stochastic", u_conv=None, streaming="ab",
                allocator: TorchAllocator | None = None, tile_rows: int = 0,
                rounding_seed: int = 0) -> vplbm_config:
    """bc: "periodic", "channel" (inlet, zero-gradient outlet, free-slip walls),
    "channel-convective" (the same with the convective outlet; U_c = u_conv,
    by default the inlet speed), or a (bc_x, bc_y) pair. allocator: a
    TorchAllocator (or any object with install(cfg)) for the device memory
    hook; None keeps the library's stream-ordered pool. tile_rows: the fused
    step's tile height (8, 16 or 32; 0 lets the library choose).
    rounding_seed: realization of the 16-bit stores' stochastic rounding."""
    c = vplbm_config_init()
    c.nx, c.ny = int(nx), int(ny)
    c.collision = COLLISION[collision] if isinstance(collision, str) else int(collision)
    c.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    if bc == "periodic":
        c.bc_x, c.bc_y = VPLBM_BC_PERIODIC, VPLBM_BC_PERIODIC
    elif bc == "channel":
        c.bc_x, c.bc_y = VPLBM_BC_INLET_OUTLET, VPLBM_BC_FREE_SLIP
    elif bc == "channel-convective":
        c.bc_x, c.bc_y = VPLBM_BC_INLET_CONVECTIVE, VPLBM_BC_FREE_SLIP
    else:
        c.bc_x, c.bc_y = bc
    c.u_conv = float(u_in[0] if u_conv is None else u_conv)
    c.streaming = {"ab": VPLBM_STREAM_AB, "aa": VPLBM_STREAM_AA}[streaming] \
        if isinstance(streaming, str) else int(streaming)
    c.tau, c.lam, c.eta = tau, lam, eta
    c.u_in[0], c.u_in[1] = u_in
    c.u0[0], c.u0[1] = u0
    c.rho0 = rho0
    c.body_force[0], c.body_force[1] = body_force
    if rates is not None:
        c.use_rates = 1
        for k in range(9):
            c.rates[k] = rates[k]
    c.reduce_mass = int(bool(reduce_mass))
    c.tile_rows = int(tile_rows)
    c.rounding_seed = int(rounding_seed)
    c.force_ring_len = int(ring_len)
    c.rounding = {"nearest": VPLBM_ROUND_NEAREST, "stochastic": VPLBM_ROUND_STOCHASTIC}[rounding] \
        if isinstance(rounding, str) else int(rounding)
    if stream is not None:
        c.stream = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    if allocator is not None:
        allocator.install(c)
    return c


def config_from_workload(w, ring_len: int = 4096, stream=None, reduce_mass: bool = True,
                         rounding: str = "stochastic", streaming: str = "ab", allocator=None,
                         tile_rows: int = 0, rounding_seed: int = 0):
    """vplbm_config and body list for an inputs.Workload (tau from its
    Reynolds number when it gives one)."""
    tau = w.tau if w.tau is not None else vplbm_tau_from_reynolds(w.u_ref, w.l_ref, w.re)
    u_in = (w.u_ref, 0.0) if w.bc == "channel" else (0.0, 0.0)
    bc = "channel-convective" if w.bc == "channel" and w.outlet == "convective" else w.bc
    cfg = make_config(w.nx, w.ny, w.collision, w.storage, tau, w.lam, bc=bc, u_in=u_in,
                      ring_len=ring_len, stream=stream, reduce_mass=reduce_mass, rounding=rounding,
                      streaming=streaming, allocator=allocator, tile_rows=tile_rows,
                      rounding_seed=rounding_seed)
    return cfg, list(w.bodies)


class Solver:
    """One vplbm solver; arrays are numpy (host) unless a call says otherwise."""

    def __init__(self, cfg: vplbm_config, bodies=(), u_init=None, perturbation=None):
        """u_init: host [2][ny][nx] initial velocity; or perturbation =
        (u0x, u0y, amp, seed) for the seeded field generated on the device."""
        self.cfg = cfg
        self.nx, self.ny = cfg.nx, cfg.ny
        self.h = vplbm_create(cfg)
        try:
            if u_init is not None:
                vplbm_set_initial_velocity(self.h, u_init)
            elif perturbation is not None:
                vplbm_set_initial_perturbation(self.h, *perturbation)
            if bodies:
                vplbm_set_bodies(self.h, list(bodies))
        except Exception:
            self.close()
            raise

    @classmethod
    def from_workload(cls, w, stream=None, ring_len: int = 4096, reduce_mass: bool = True,
                      with_initial_velocity: bool = True, rounding: str = "stochastic",
                      device_init: bool = False, streaming: str = "ab", allocator=None,
                      tile_rows: int = 0, rounding_seed: int = 0):
        """device_init: generate the workload's seeded initial field on the
        device (bit-identical to w.initial_velocity())."""
        cfg, bodies = config_from_workload(w, ring_len, stream, reduce_mass, rounding, streaming,
                                           allocator, tile_rows, rounding_seed)
        if not with_initial_velocity:
            return cls(cfg, bodies)
        if device_init:
            u0 = (w.u_ref, 0.0) if w.bc == "channel" else (0.0, 0.0)
            return cls(cfg, bodies, perturbation=(u0[0], u0[1], w.perturbation, w.seed))
        return cls(cfg, bodies, w.initial_velocity())

    def close(self):
        if getattr(self, "h", None):
            vplbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def t(self) -> int:
        return vplbm_step_count(self.h)

    def step(self, n: int = 1):
        vplbm_step(self.h, n)
        return self

    def synchronize(self):
        vplbm_synchronize(self.h)

    def set_mask(self, chi, us=None):
        vplbm_set_mask_and_solid_velocity(self.h, chi, us)

    def set_bodies(self, bodies):
        vplbm_set_bodies(self.h, list(bodies))

    def set_initial_velocity(self, u=None):
        vplbm_set_initial_velocity(self.h, u)

    def moments(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        vplbm_moments(self.h, rho, ux, uy)
        return rho, ux, uy

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        vplbm_populations(self.h, f)
        return f

    def set_populations(self, f):
        vplbm_set_populations(self.h, f)

    def mask(self):
        chi = np.empty((self.ny, self.nx), dtype=np.uint8)
        vplbm_mask(self.h, chi)
        return chi

    def forces(self, cap: int | None = None):
        return vplbm_forces(self.h, cap or self.cfg.force_ring_len)

    def momentum_exchange(self):
        """Momentum-exchange force on the solids at the current state."""
        return vplbm_momentum_exchange(self.h)

    def record_momentum_exchange(self, enable: bool = True):
        vplbm_enable_momentum_exchange(self.h, enable)

    def momentum_exchange_forces(self, cap: int | None = None):
        return vplbm_momentum_exchange_forces(self.h, cap or self.cfg.force_ring_len)

    @property
    def launches(self) -> int:
        return vplbm_launch_count(self.h)
