"""ctypes front end of the plain FP64 C oracle (vplbm_oracle.c).

TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
baseline of the benchmark; never by the product path. Arrays are numpy float64
in the layout f[alpha][y][x] (alpha = 0..8), fields [ny][nx], vectors [2][ny][nx].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vplbm_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

SRT, MRT = 0, 1
BC_PERIODIC, BC_INLET_OUTLET, BC_FREE_SLIP, BC_INLET_CONVECTIVE = 0, 1, 2, 3
OUTLET_DIRS = (3, 6, 7)  # directions entering through the outlet, rows of the outlet state


class OrcBody(C.Structure):
    _fields_ = [
        ("cx", C.c_double), ("cy", C.c_double), ("radius", C.c_double),
        ("amp_x", C.c_double), ("amp_y", C.c_double), ("period", C.c_double),
        ("omega", C.c_double), ("outside", C.c_int32), ("pad_", C.c_int32),
    ]


class OrcConfig(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32), ("collision", C.c_int32),
        ("bc_x", C.c_int32), ("bc_y", C.c_int32), ("use_rates", C.c_int32),
        ("tau", C.c_double), ("lam", C.c_double), ("eta", C.c_double),
        ("u_in", C.c_double * 2), ("g", C.c_double * 2), ("rates", C.c_double * 9),
        ("chi", C.POINTER(C.c_uint8)), ("us", C.POINTER(C.c_double)),
        ("bodies", C.POINTER(OrcBody)), ("n_bodies", C.c_int32), ("pad_", C.c_int32),
        ("u_conv", C.c_double), ("outlet", C.POINTER(C.c_double)),
    ]


def build(force: bool = False) -> str:
    """Compile vplbm_oracle.c into liboracle.so next to it (gcc, -O2, OpenMP,
    no floating-point contraction so that x86 and Arm hosts round alike)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vplbm_oracle.h"))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # VPLBM_ORACLE_LIB: load another build of this source instead (the
            # mutation test points it at deliberately broken copies)
            path = os.environ.get("VPLBM_ORACLE_LIB") or build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            cp = C.POINTER(OrcConfig)
            L.orc_velocity_set.argtypes = [C.POINTER(C.c_int32)]
            L.orc_weights.argtypes = [dp]
            L.orc_moment_matrix.argtypes = [dp]
            L.orc_moment_matrix_inverse.argtypes = [dp]
            L.orc_equilibrium.argtypes = [C.c_double] * 3 + [dp]
            L.orc_guo_force_srt.argtypes = [C.c_double] * 5 + [dp]
            L.orc_guo_force_mrt.argtypes = [C.c_double] * 4 + [dp]
            L.orc_mrt_equilibrium_moments.argtypes = [C.c_double] * 3 + [dp]
            L.orc_node_macros.argtypes = [cp, dp, C.c_int32, C.c_double, C.c_double] + [dp] * 5
            L.orc_node_macros_literal.argtypes = L.orc_node_macros.argtypes
            L.orc_collide_node.argtypes = [cp, dp, C.c_int32, C.c_double, C.c_double, dp, dp, dp]
            L.orc_mask.argtypes = [cp, C.c_int64, C.POINTER(C.c_uint8), dp]
            L.orc_init_equilibrium.argtypes = [cp, C.c_double, dp, dp]
            L.orc_run.argtypes = [cp, dp, C.c_int64, C.c_int64, dp, dp, dp]
            L.orc_moments.argtypes = [cp, dp, C.c_int64, dp, dp, dp]
            L.orc_num_threads.restype = C.c_int
            L.orc_set_num_threads.argtypes = [C.c_int]
            L.orc_set_num_threads.restype = None
            L.orc_momentum_exchange.argtypes = [cp, dp, C.c_int64, dp, dp]
            ip = C.POINTER(C.c_int32)
            L.orc_step_nodes.argtypes = [cp, dp, C.c_int64, C.c_int64, ip, ip, dp, dp, dp,
                                         C.POINTER(C.c_uint8)]
            L.orc_step_nodes.restype = C.c_int
            L.orc_momentum_exchange.restype = C.c_int
            for name in ("orc_mask", "orc_init_equilibrium", "orc_run", "orc_moments"):
                getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Body:
    """Rigid circle: centre(t) = c + amp sin(2 pi t / period); rotation omega."""
    cx: float
    cy: float
    radius: float
    amp_x: float = 0.0
    amp_y: float = 0.0
    period: float = 0.0
    omega: float = 0.0
    outside: bool = False


@dataclass
class Config:
    nx: int
    ny: int
    collision: int = SRT
    tau: float = 0.8
    lam: float = 3.0 / 16.0
    eta: float = 1e-7
    bc_x: int = BC_PERIODIC
    bc_y: int = BC_PERIODIC
    u_in: tuple = (0.0, 0.0)
    g: tuple = (0.0, 0.0)
    rates: tuple | None = None
    chi: np.ndarray | None = None     # uint8 [ny][nx]
    us: np.ndarray | None = None      # float64 [2][ny][nx]
    bodies: list = field(default_factory=list)
    u_conv: float = 0.0               # convective outlet velocity U_c
    outlet: np.ndarray | None = None  # convective outlet state [3][ny], updated by run()

    def c_struct(self):
        """Returns (struct, keepalive) — keepalive holds the arrays it points to."""
        s = OrcConfig()
        s.nx, s.ny, s.collision = self.nx, self.ny, self.collision
        s.bc_x, s.bc_y = self.bc_x, self.bc_y
        s.tau, s.lam, s.eta = self.tau, self.lam, self.eta
        s.u_in[0], s.u_in[1] = self.u_in
        s.g[0], s.g[1] = self.g
        keep = []
        if self.rates is not None:
            s.use_rates = 1
            for k in range(9):
                s.rates[k] = self.rates[k]
        if self.chi is not None:
            chi = np.ascontiguousarray(self.chi, dtype=np.uint8)
            assert chi.shape == (self.ny, self.nx)
            keep.append(chi)
            s.chi = chi.ctypes.data_as(C.POINTER(C.c_uint8))
        if self.us is not None:
            us = np.ascontiguousarray(self.us, dtype=np.float64)
            assert us.shape == (2, self.ny, self.nx)
            keep.append(us)
            s.us = _dp(us)
        if self.outlet is not None:
            # the state is updated in place: it must be the caller's own array
            assert self.outlet.dtype == np.float64 and self.outlet.flags.c_contiguous
            assert self.outlet.shape == (3, self.ny)
            s.outlet = _dp(self.outlet)
        s.u_conv = self.u_conv
        if self.bodies:
            arr = (OrcBody * len(self.bodies))()
            for i, b in enumerate(self.bodies):
                arr[i] = OrcBody(b.cx, b.cy, b.radius, b.amp_x, b.amp_y, b.period,
                                 b.omega, int(b.outside), 0)
            keep.append(arr)
            s.bodies = C.cast(arr, C.POINTER(OrcBody))
            s.n_bodies = len(self.bodies)
        return s, keep


# ----------------------------------------------------------------------------
# single-node routines
# ----------------------------------------------------------------------------

def velocity_set() -> np.ndarray:
    xi = np.zeros((9, 2), dtype=np.int32)
    lib().orc_velocity_set(xi.ctypes.data_as(C.POINTER(C.c_int32)))
    return xi


def weights() -> np.ndarray:
    w = np.zeros(9)
    lib().orc_weights(_dp(w))
    return w


def moment_matrix() -> np.ndarray:
    M = np.zeros((9, 9))
    lib().orc_moment_matrix(_dp(M))
    return M


def moment_matrix_inverse() -> np.ndarray:
    M = np.zeros((9, 9))
    lib().orc_moment_matrix_inverse(_dp(M))
    return M


def equilibrium(rho, ux, uy) -> np.ndarray:
    f = np.zeros(9)
    lib().orc_equilibrium(rho, ux, uy, _dp(f))
    return f


def guo_force_srt(tau, ux, uy, fx, fy) -> np.ndarray:
    F = np.zeros(9)
    lib().orc_guo_force_srt(tau, ux, uy, fx, fy, _dp(F))
    return F


def guo_force_mrt(ux, uy, fx, fy) -> np.ndarray:
    F = np.zeros(9)
    lib().orc_guo_force_mrt(ux, uy, fx, fy, _dp(F))
    return F


def mrt_equilibrium_moments(rho, ux, uy) -> np.ndarray:
    m = np.zeros(9)
    lib().orc_mrt_equilibrium_moments(rho, ux, uy, _dp(m))
    return m


def node_macros(cfg: Config, f, chi, usx, usy, literal=False):
    s, keep = cfg.c_struct()
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = [C.c_double() for _ in range(5)]
    fn = lib().orc_node_macros_literal if literal else lib().orc_node_macros
    fn(C.byref(s), _dp(f), int(chi), usx, usy, *[C.byref(o) for o in out])
    return tuple(o.value for o in out)  # rho, ux, uy, fpx, fpy


def collide_node(cfg: Config, f, chi=0, usx=0.0, usy=0.0):
    s, keep = cfg.c_struct()
    f = np.ascontiguousarray(f, dtype=np.float64)
    fo = np.zeros(9)
    px, py = C.c_double(), C.c_double()
    lib().orc_collide_node(C.byref(s), _dp(f), int(chi), usx, usy, _dp(fo),
                           C.byref(px), C.byref(py))
    return fo, (px.value, py.value)


# ----------------------------------------------------------------------------
# grid routines
# ----------------------------------------------------------------------------

def mask(cfg: Config, t: int = 0):
    s, keep = cfg.c_struct()
    chi = np.zeros((cfg.ny, cfg.nx), dtype=np.uint8)
    us = np.zeros((2, cfg.ny, cfg.nx))
    rc = lib().orc_mask(C.byref(s), t, chi.ctypes.data_as(C.POINTER(C.c_uint8)), _dp(us))
    assert rc == 0
    return chi, us


def init_equilibrium(cfg: Config, rho0: float = 1.0, u_init=None) -> np.ndarray:
    s, keep = cfg.c_struct()
    f = np.zeros((9, cfg.ny, cfg.nx))
    up = None
    if u_init is not None:
        u_init = np.ascontiguousarray(u_init, dtype=np.float64)
        assert u_init.shape == (2, cfg.ny, cfg.nx)
        up = _dp(u_init)
    rc = lib().orc_init_equilibrium(C.byref(s), rho0, up, _dp(f))
    assert rc == 0
    return f


def run(cfg: Config, f: np.ndarray, n: int, t0: int = 0):
    """Advances the post-collision store f (modified in place) by n steps.
    Returns (fx, fy, mass) per step."""
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (9, cfg.ny, cfg.nx)
    s, keep = cfg.c_struct()
    fx, fy, ms = np.zeros(n), np.zeros(n), np.zeros(n)
    rc = lib().orc_run(C.byref(s), _dp(f), t0, n, _dp(fx), _dp(fy), _dp(ms))
    assert rc == 0, rc
    return fx, fy, ms


def moments(cfg: Config, f: np.ndarray, t: int = 0):
    s, keep = cfg.c_struct()
    f = np.ascontiguousarray(f, dtype=np.float64)
    rho = np.zeros((cfg.ny, cfg.nx))
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    rc = lib().orc_moments(C.byref(s), _dp(f), t, _dp(rho), _dp(ux), _dp(uy))
    assert rc == 0
    return rho, ux, uy


def momentum_exchange(cfg: Config, f: np.ndarray, t: int = 0):
    """Momentum-exchange force on the solids from the store f*(t)."""
    s, keep = cfg.c_struct()
    f = np.ascontiguousarray(f, dtype=np.float64)
    fx, fy = C.c_double(), C.c_double()
    rc = lib().orc_momentum_exchange(C.byref(s), _dp(f), t, C.byref(fx), C.byref(fy))
    assert rc == 0
    return fx.value, fy.value


def step_nodes(cfg: Config, f: np.ndarray, t: int, xs, ys):
    """One step (index t) of the listed nodes from the store f*(t):
    (f*(t+1) [n][9], fpx [n], fpy [n], chi [n])."""
    s, keep = cfg.c_struct()
    assert f.dtype == np.float64 and f.flags.c_contiguous and f.shape == (9, cfg.ny, cfg.nx)
    xs = np.ascontiguousarray(xs, dtype=np.int32)
    ys = np.ascontiguousarray(ys, dtype=np.int32)
    n = xs.size
    fout = np.zeros((n, 9))
    fpx, fpy, chi = np.zeros(n), np.zeros(n), np.zeros(n, np.uint8)
    ip = C.POINTER(C.c_int32)
    rc = lib().orc_step_nodes(C.byref(s), _dp(f), t, n, xs.ctypes.data_as(ip), ys.ctypes.data_as(ip),
                              _dp(fout), _dp(fpx), _dp(fpy), chi.ctypes.data_as(C.POINTER(C.c_uint8)))
    assert rc == 0, rc
    return fout, fpx, fpy, chi


def outlet_from_store(f: np.ndarray) -> np.ndarray:
    """Convective outlet state that starts as a zero-gradient copy of the last
    column of the store f[9][ny][nx]."""
    return np.ascontiguousarray(f[list(OUTLET_DIRS), :, -1], dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's row loop; n <= 0 restores all processors."""
    lib().orc_set_num_threads(int(n))


def tau_from_reynolds(u_ref: float, l_ref: float, re: float) -> float:
    """nu = U L / Re and nu = c_s^2 (tau - 1/2) (Section 2.1.1): tau = 3 nu + 1/2."""
    nu = u_ref * l_ref / re
    return 3.0 * nu + 0.5


__all__ = [n for n in dir() if not n.startswith("_")]
