"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and the
oracle tests.

This module holds no arithmetic of the method: it states workload geometry
(grid sizes, body positions, inlet speeds, Reynolds numbers, step counts) and
draws the random numbers the workloads need. Relaxation times, masks and
equilibria are computed by each side on its own.

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014): state += 0x9E3779B97F4A7C15,
then the two xor-shift-multiply rounds and a final xor-shift; the top 53 bits
give a double in [0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n successive SplitMix64 outputs (uint64) from the given seed."""
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        idx = np.arange(1, n + 1, dtype=np.uint64)
        z = (np.uint64(seed & _MASK64) + idx * np.uint64(0x9E3779B97F4A7C15))
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        out[:] = z ^ (z >> np.uint64(31))
    return out


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def velocity_field(nx: int, ny: int, u0=(0.0, 0.0), amp: float = 0.0, seed: int = 1) -> np.ndarray:
    """Initial velocity [2][ny][nx]: uniform u0 plus, when amp > 0, independent
    uniform perturbations in [-amp, amp] drawn in the order y, then x, then
    component."""
    u = np.empty((2, ny, nx), dtype=np.float64)
    u[0] = u0[0]
    u[1] = u0[1]
    if amp > 0.0:
        r = uniform01(seed, 2 * nx * ny).reshape(ny, nx, 2)
        u[0] += amp * (2.0 * r[:, :, 0] - 1.0)
        u[1] += amp * (2.0 * r[:, :, 1] - 1.0)
    return u


def random_populations(nx: int, ny: int, seed: int, spread: float = 0.02) -> np.ndarray:
    """Positive populations near the D2Q9 rest state, for unit tests of a
    single step: w_alpha (4/9, 1/9, 1/36 as printed with the model) times
    (1 + spread * (2 r - 1)). Layout [9][ny][nx]."""
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    r = uniform01(seed, 9 * nx * ny).reshape(9, ny, nx)
    return w[:, None, None] * (1.0 + spread * (2.0 * r - 1.0))


def random_mask(nx: int, ny: int, seed: int, solid_fraction: float = 0.2) -> np.ndarray:
    """uint8 [ny][nx] with about solid_fraction of the nodes set to 1."""
    r = uniform01(seed, nx * ny).reshape(ny, nx)
    return (r < solid_fraction).astype(np.uint8)


def random_solid_velocity(nx: int, ny: int, seed: int, amp: float = 0.02) -> np.ndarray:
    r = uniform01(seed, 2 * nx * ny).reshape(2, ny, nx)
    return amp * (2.0 * r - 1.0)


# -----------------------------------------------------------------------------
# Workloads shaped like the paper's cases
# -----------------------------------------------------------------------------

@dataclass
class BodySpec:
    """Rigid circle: centre(t) = (cx, cy) + (amp_x, amp_y) sin(2 pi t / period)
    (period 0: fixed), rigid rotation omega about the centre; outside = True
    makes the solid the region r >= radius (an enclosing cylinder wall)."""
    cx: float
    cy: float
    radius: float
    amp_x: float = 0.0
    amp_y: float = 0.0
    period: float = 0.0
    omega: float = 0.0
    outside: bool = False


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    collision: str            # "srt" | "mrt"
    storage: str              # "f64" | "f32" | "f16" | "bf16"
    bc: str                   # "periodic" | "channel" (inlet/outlet in x, free slip in y)
    steps: int
    u_ref: float              # inlet speed (channel) or wall speed (Couette)
    l_ref: float              # length the Reynolds number is based on
    re: float | None = None   # None: tau given directly
    tau: float | None = None
    lam: float = 3.0 / 16.0
    bodies: list = field(default_factory=list)
    perturbation: float = 0.0
    seed: int = 1
    outlet: str = "zero-gradient"  # channel outlet: "zero-gradient" | "convective"

    def initial_velocity(self) -> np.ndarray:
        u0 = (self.u_ref, 0.0) if self.bc == "channel" else (0.0, 0.0)
        return velocity_field(self.nx, self.ny, u0, self.perturbation, self.seed)


def circular_couette(n: int = 128, r1: float = 24.0, r2: float = 56.0, wall_speed: float = 0.01,
                     tau: float = 0.8, steps: int = 10_000, collision: str = "srt",
                     storage: str = "f64") -> Workload:
    """Rotating inner cylinder (radius r1, wall speed wall_speed) inside a fixed
    outer cylinder (radius r2), both centred in an n x n periodic box."""
    c = (n - 1) / 2.0
    return Workload(
        name=f"circular-couette-{n}x{n}", nx=n, ny=n, collision=collision, storage=storage,
        bc="periodic", steps=steps, u_ref=wall_speed, l_ref=r2 - r1, tau=tau,
        bodies=[BodySpec(c, c, r1, omega=wall_speed / r1), BodySpec(c, c, r2, outside=True)])


def cylinder_channel(nx: int, ny: int, diameter: float, u_in: float, re: float, steps: int,
                     xc: float | None = None, collision: str = "mrt", storage: str = "f32",
                     perturbation: float = 1e-4, seed: int = 1, lam: float = 3.0 / 16.0,
                     outlet: str = "zero-gradient") -> Workload:
    """Fixed cylinder in a channel: uniform inlet at x = 0, outlet at x = nx - 1
    (zero-gradient or convective), free-slip walls at y = 0 and y = ny - 1."""
    xc = nx / 4.0 if xc is None else xc
    return Workload(
        name=f"cylinder-channel-{nx}x{ny}-D{diameter:g}-Re{re:g}", nx=nx, ny=ny,
        collision=collision, storage=storage, bc="channel", steps=steps, u_ref=u_in,
        l_ref=diameter, re=re, lam=lam, bodies=[BodySpec(xc, (ny - 1) / 2.0, diameter / 2.0)],
        perturbation=perturbation, seed=seed, outlet=outlet)


def moving_cylinder_channel(nx: int = 16384, ny: int = 4096, diameter: float = 256.0,
                            u_in: float = 0.05, re: float = 2000.0, steps: int = 50_000,
                            period: float = 20_000.0, amp_fraction: float = 0.5,
                            storage: str = "f32", seed: int = 1) -> Workload:
    """Cylinder translating transversely, y(t) = y0 + A sin(2 pi t / T), A = amp_fraction D."""
    w = cylinder_channel(nx, ny, diameter, u_in, re, steps, xc=nx / 4.0, storage=storage,
                         perturbation=1e-4, seed=seed)
    b = w.bodies[0]
    b.amp_y = amp_fraction * diameter
    b.period = period
    w.name = f"moving-cylinder-{nx}x{ny}-D{diameter:g}-Re{re:g}"
    return w


# The five workloads of the method's evaluation, at full size.
def c1_circular_couette():
    return circular_couette(128, 24.0, 56.0, 0.01, 0.8, 10_000, "srt", "f64")


def c2_cylinder_re100():
    return cylinder_channel(1024, 256, 40.0, 0.05, 100.0, 100_000, xc=256.0, storage="f32")


def c3_cylinder_re1000(storage: str = "f32"):
    return cylinder_channel(4096, 1024, 128.0, 0.04, 1000.0, 200_000, storage=storage)


def c5_moving_cylinder(storage: str = "f32"):
    return moving_cylinder_channel(storage=storage)


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    workload: Workload
    deadline: float | None = None  # seconds after arrival the result is wanted by (None: no limit)


def serving_mix(n_requests: int = 256, rate: float = 4.0, seed: int = 1234,
                side_min: int = 64, side_max: int = 1024, steps_min: int = 2000,
                steps_max: int = 20_000, storage: str | None = None,
                nu_min: float = 0.02 / 3.0) -> list:
    """Seeded serving mix: Poisson arrivals at `rate` per second; circular
    Couette or cylinder channel 50/50; square side log-uniform in
    [side_min, side_max] (channels are 4 side x side); Re uniform in [20, 500];
    SRT or MRT 50/50; steps uniform in [steps_min, steps_max]; storage f32 or
    f16 50/50 unless fixed. Each request runs at the largest lattice speed
    (0.01 for Couette, 0.05 for channels) with its relaxation time from Re, and
    never below tau_min = 1/2 + 3 nu_min: a grid too coarse for the requested
    Re at tau_min runs at the highest Re it resolves (U L / nu_min), which is
    recorded in the workload. tau_min = 0.52 is the smallest relaxation time
    at which MRT with the printed rates (Lambda = 3/16) keeps every channel
    size of the mix stable for the mix's longest run of 20,000 steps; at 0.515
    and below every size diverged (SRT stays stable down to 0.505)."""
    r = uniform01(seed, 8 * n_requests).reshape(n_requests, 8)
    reqs = []
    t = 0.0
    for i in range(n_requests):
        t += -math.log(1.0 - r[i, 0]) / rate
        side = int(round(math.exp(math.log(side_min) + r[i, 1] * (math.log(side_max) - math.log(side_min)))))
        re = 20.0 + 480.0 * r[i, 2]
        coll = "srt" if r[i, 3] < 0.5 else "mrt"
        steps = int(steps_min + math.floor(r[i, 4] * (steps_max - steps_min + 1)))
        st = storage or ("f32" if r[i, 5] < 0.5 else "f16")
        if r[i, 6] < 0.5:
            r1, r2 = 0.1875 * side, 0.4375 * side
            lref = r2 - r1
            u = 0.01
            re = min(re, u * lref / nu_min)
            w = circular_couette(side, r1, r2, u, 0.8, steps, coll, st)
            w.tau = None
            w.re = re
        else:
            d = max(4.0, round(40.0 * side / 256.0))
            u = 0.05
            re = min(re, u * d / nu_min)
            w = cylinder_channel(4 * side, side, d, u, re, steps, collision=coll, storage=st,
                                 perturbation=1e-4, seed=seed + i)
        w.name = f"req{i}-" + w.name
        reqs.append(Request(i, t, w))
    return reqs
