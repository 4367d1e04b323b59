"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only *describes* inputs: lattice sizes, boundary kinds, relaxation
times, marker coordinates on a circle and seeded random population fields.  It
holds none of the method's arithmetic (no equilibrium, no kernel, no forcing)
and imports neither the oracle nor the CUDA library, so both can be fed from it.

The shapes follow the paper's workloads (Sec. 2.9, Table I): a fixed cylinder
in a channel with uniform inflow, zero-gradient outflow and far-field top and
bottom; an in-line oscillating cylinder in quiescent fluid with open sides; a
settling disk in a walled channel; and a stream of mixed requests for serving.
Markers sit at theta_k = 2 pi k / N starting on the +x axis with spacing
ds = pi D / N (Table I, "Lagrangian markers").
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Tuple

import numpy as np

# enum values shared by value (not by code) with the C interfaces
PERIODIC, VELOCITY, NEUMANN = 0, 1, 2
BGK, TRT, CMMRT, STREAM_ONLY = 0, 1, 2, 3
HAT, PESKIN4 = 0, 1
DF, MDF, DFC = 0, 1, 2
FIXED, PRESCRIBED, FREE, FREE_TRANSLATION = 0, 1, 2, 3
F64, F32, F16S = 0, 1, 2

COLLISIONS = {"bgk": BGK, "trt": TRT, "cmmrt": CMMRT}
KERNELS = {"hat": HAT, "p4": PESKIN4}
SCHEMES = {"df": DF, "mdf": MDF, "dfc": DFC}
STORAGES = {"f64": F64, "f32": F32, "f16": F16S}


@dataclasses.dataclass
class BodySpec:
    xy: np.ndarray            # (n, 2) marker coordinates, lattice units
    ds: float
    kernel: int
    scheme: int
    xc: float
    yc: float
    radius: float
    rho_ratio: float = 1.0
    motion: int = FIXED
    gx: float = 0.0
    gy: float = 0.0
    internal_mass: int = 1
    mdf_nmin: int = 5
    mdf_nmax: int = 20
    mdf_tol: float = 1e-4
    mdf_omega: float = 0.0
    osc_amp: float = 0.0
    osc_period: float = 1.0


@dataclasses.dataclass
class CaseSpec:
    name: str
    nx: int
    ny: int
    bc: Tuple[int, int, int, int]
    ubc: Tuple[Tuple[float, float], ...]
    collision: int
    tau: float
    storage: int = F64
    trt_lambda: float = 3.0 / 16.0
    cm_sq: float = 1.2
    cm_se: float = 1.4
    force: Tuple[float, float] = (0.0, 0.0)
    init_u: Tuple[float, float] = (0.0, 0.0)
    bodies: List[BodySpec] = dataclasses.field(default_factory=list)
    steps: int = 1
    wall_closure: int = 0

    @property
    def nodes(self) -> int:
        return self.nx * self.ny


def circle_markers(xc: float, yc: float, diameter: float, n: int) -> Tuple[np.ndarray, float]:
    """n equispaced markers on a circle, first one on the +x axis; returns (xy, ds)."""
    th = 2.0 * math.pi * np.arange(n) / n
    r = 0.5 * diameter
    xy = np.stack([xc + r * np.cos(th), yc + r * np.sin(th)], axis=1)
    return np.ascontiguousarray(xy), math.pi * diameter / n


def tau_for(u_ref: float, diameter: float, re: float) -> float:
    """Relaxation time giving Re = u_ref D / nu with nu = (tau - 1/2)/3 (App. A.1)."""
    return 0.5 + 3.0 * u_ref * diameter / re


def _cylinder_channel(name, nx, ny, xc, yc, diameter, nmark, u_inf, tau, collision, kernel,
                      scheme, storage, steps, mdf_nmin=5, mdf_nmax=20) -> CaseSpec:
    xy, ds = circle_markers(xc, yc, diameter, nmark)
    body = BodySpec(xy=xy, ds=ds, kernel=kernel, scheme=scheme, xc=xc, yc=yc,
                    radius=0.5 * diameter, mdf_nmin=mdf_nmin, mdf_nmax=mdf_nmax)
    ubc = ((u_inf, 0.0), (0.0, 0.0), (u_inf, 0.0), (u_inf, 0.0))
    return CaseSpec(name=name, nx=nx, ny=ny, bc=(VELOCITY, NEUMANN, VELOCITY, VELOCITY), ubc=ubc,
                    collision=collision, tau=tau, storage=storage, init_u=(u_inf, 0.0),
                    bodies=[body], steps=steps)


def fixed_cylinder_re20(storage=F64, steps=2000, collision=BGK, kernel=HAT, scheme=DF) -> CaseSpec:
    """200x100 lattice, D=20 at (50,50), 63 markers, U=0.05, tau=0.65 (Re=20)."""
    return _cylinder_channel("cyl-re20-200x100", 200, 100, 50.0, 50.0, 20.0, 63, 0.05, 0.65,
                             collision, kernel, scheme, storage, steps)


def fixed_cylinder_2048(re=100.0, storage=F32, collision=BGK, kernel=PESKIN4, scheme=DF,
                        steps=200000, nx=2048, ny=1024, diameter=64.0, nmark=201,
                        mdf_iters=5) -> CaseSpec:
    """2048x1024 lattice, D=64 at (0.4 Lx, 0.5 Ly), 201 markers, U=0.1 (Sec. 2.9.1 shape).

    MDF runs with N_min = N_max = ``mdf_iters`` (5 fixed iterations)."""
    tau = tau_for(0.1, diameter, re)
    name = "cyl-re%d-%dx%d" % (int(re), nx, ny)
    return _cylinder_channel(name, nx, ny, 0.4 * nx, 0.5 * ny, diameter, nmark, 0.1, tau,
                             collision, kernel, scheme, storage, steps,
                             mdf_nmin=mdf_iters, mdf_nmax=mdf_iters)


def oscillating_cylinder(storage=F32, kernel=PESKIN4, scheme=DF, nx=1024, ny=512, diameter=40.0,
                         kc=5.0, u_max=0.1, re=100.0, steps=20000) -> CaseSpec:
    """In-line oscillation x_c(t) = x0 - A sin(2 pi t/T) in quiescent fluid, open sides.

    KC = U_max T / D and A = KC D / (2 pi) (Sec. 2.9.2)."""
    nmark = int(round(math.pi * diameter))
    xc, yc = 0.5 * nx, 0.5 * ny
    xy, ds = circle_markers(xc, yc, diameter, nmark)
    period = kc * diameter / u_max
    body = BodySpec(xy=xy, ds=ds, kernel=kernel, scheme=scheme, xc=xc, yc=yc, radius=0.5 * diameter,
                    motion=PRESCRIBED, osc_amp=kc * diameter / (2.0 * math.pi), osc_period=period)
    tau = tau_for(u_max, diameter, re)
    return CaseSpec(name="osc-%dx%d" % (nx, ny), nx=nx, ny=ny, bc=(NEUMANN,) * 4,
                    ubc=((0.0, 0.0),) * 4, collision=BGK, tau=tau, storage=storage,
                    bodies=[body], steps=steps)


def sedimentation(two_particles=False, storage=F64, internal_mass=1, kernel=PESKIN4, scheme=DFC,
                  nx=400, ny=1600, diameter=20.0, tau=0.65, g=8.33e-5, steps=60000) -> CaseSpec:
    """Walled channel, gravity along -y, disk(s) released at rest (Sec. 2.9.3 shape)."""
    nmark = int(round(math.pi * diameter))
    # released 8 D below the top wall; the second (heavy) particle 2 D below the light one
    if two_particles:
        placements = [(0.5 * nx, ny - 10.0 * diameter, 1.5), (0.5 * nx, ny - 8.0 * diameter, 1.01)]
    else:
        placements = [(0.5 * nx, ny - 8.0 * diameter, 1.5)]
    bodies = []
    for xc, yc, rr in placements:
        xy, ds = circle_markers(xc, yc, diameter, nmark)
        bodies.append(BodySpec(xy=xy, ds=ds, kernel=kernel, scheme=scheme, xc=xc, yc=yc,
                               radius=0.5 * diameter, rho_ratio=rr, motion=FREE, gx=0.0, gy=-g,
                               internal_mass=internal_mass))
    return CaseSpec(name="sed-%dx%d" % (nx, ny), nx=nx, ny=ny, bc=(VELOCITY,) * 4,
                    ubc=((0.0, 0.0),) * 4, collision=BGK, tau=tau, storage=storage, bodies=bodies,
                    steps=steps)


def random_populations(seed: int, nx: int, ny: int, amp: float = 0.05) -> np.ndarray:
    """Seeded positive populations near a resting state, shape (9, ny, nx).

    Base levels per direction class (rest 4/9, axial 1/9, diagonal 1/36) times
    (1 + amp * U(-1, 1)): an input recipe, not the method's equilibrium."""
    rng = np.random.default_rng(seed)
    base = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)[:, None, None]
    return np.ascontiguousarray(base * (1.0 + amp * rng.uniform(-1.0, 1.0, size=(9, ny, nx))))


def random_markers(seed: int, n: int, lo: Tuple[float, float], hi: Tuple[float, float]) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(np.stack([rng.uniform(lo[0], hi[0], n), rng.uniform(lo[1], hi[1], n)], 1))


SERVING_GRIDS = [(128, 64), (256, 128), (512, 256), (1024, 512), (2048, 1024)]


def serving_requests(seed: int = 0, n: int = 256, rate: float = 100.0, steps: int = 2000,
                     grids=None, storage=F32):
    """Seeded request stream: Poisson arrivals (rate per second), grids drawn
    log-uniformly from ``grids``, D = ny/8, round(pi D) markers, uniform
    scheme/kernel/collision, Re uniform in [20, 200], U = 0.1, resampled while
    tau is below the operator's floor (0.6 for BGK, whose runs below it went
    unstable on the coarse grids at U = 0.1; 0.55 for TRT and CM-MRT).
    Returns (arrival_times, [CaseSpec]), plus the resample count."""
    grids = grids or SERVING_GRIDS
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    specs, resampled = [], 0
    for r in range(n):
        nx, ny = grids[rng.integers(len(grids))]
        d = ny / 8.0
        scheme = int(rng.integers(3))
        kernel = int(rng.integers(2))
        collision = int(rng.integers(3))
        floor = 0.6 if collision == BGK else 0.55
        while True:
            re = rng.uniform(20.0, 200.0)
            tau = tau_for(0.1, d, re)
            if tau >= floor:
                break
            resampled += 1
        spec = _cylinder_channel("req%d" % r, nx, ny, 0.4 * nx, 0.5 * ny, d,
                                 int(round(math.pi * d)), 0.1, tau, collision, kernel, scheme,
                                 storage, steps)
        specs.append(spec)
    return t, specs, resampled
