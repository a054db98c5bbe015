"""Synthetic shallow-water scenarios (seeded), shared by the oracle tests, the CUDA
tests and the benchmark.

A scenario is pure input description: a mesh recipe, physical constants, the
bathymetry B(x, y) and the initial state as functions of physical coordinates.
Both sides evaluate these functions at their own interpolation nodes, so this
module holds none of the discontinuous Galerkin arithmetic.

The bathymetry function has the signature ``bathymetry(x, y, cx, cy)`` and the
initial-state function ``init(x, y, cx, cy, B)``, where
``x, y`` are node coordinates (any shape), ``cx, cy`` the centroid of each
node's element (same shape) and ``B`` the bathymetry at those nodes; it returns
``(h, hu, hv)``.

Limiter mask bits: 1 = positivity-preserving limiter, 2 = TVB limiter.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable

import numpy as np

from . import meshes

LIM_PP = 1
LIM_TVB = 2


@dataclasses.dataclass
class Scenario:
    name: str
    mesh: Callable[[], tuple]          # () -> (vx, vy, EToV)
    N: int
    g: float
    h0: float
    cfl: float
    nlevels: int
    limiter_mask: int
    tvb_M: float
    bathymetry: Callable
    init: Callable
    steps: int = 1                      # finest substeps for a parity run
    tvb_nu: float = 1.5
    dry_mode: int = 0
    note: str = ""

    def build_mesh(self):
        return self.mesh()


# ----------------------------------------------------------------------------
# bathymetries and initial states


def flat_bed(depth: float):
    return lambda x, y, cx=None, cy=None: np.full(np.shape(x), -float(depth))


def gaussian_hump_init(amp: float, x0: float, y0: float, width: float):
    def init(x, y, cx, cy, B):
        eta = amp * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / width ** 2)
        h = eta - B
        return h, np.zeros_like(h), np.zeros_like(h)
    return init


def tanh_beach(x_mid: float = 380e3, width: float = 5e3, deep: float = -4000.0,
               rise: float = 4010.0):
    """B = deep + rise * (1 + tanh((x - x_mid) / width)) / 2 (metres).

    With the defaults B rises from -4000 m to about +8.6 m at x = 400 km and the
    still-water shoreline (B = 0) sits near x = 395 km, so the last few km are dry.
    """
    return lambda x, y, cx=None, cy=None: deep + rise * 0.5 * (
        1.0 + np.tanh((np.asarray(x) - x_mid) / width))


def bump_on_beach_init(amp: float, x0: float, y0: float, radius: float):
    """Free surface eta = amp * exp(-r^2/radius^2); h = max(0, eta - B); at rest."""
    def init(x, y, cx, cy, B):
        eta = amp * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / radius ** 2)
        h = np.maximum(0.0, eta - B)
        return h, np.zeros_like(h), np.zeros_like(h)
    return init


def dam_init(x_dam: float, h_left: float):
    """h = h_left on elements whose centroid is left of x_dam, else dry."""
    def init(x, y, cx, cy, B):
        h = np.where(np.asarray(cx) < x_dam, h_left, 0.0) + 0.0 * np.asarray(x)
        return h, np.zeros_like(h), np.zeros_like(h)
    return init


def lake_at_rest_init(eta0: float):
    def init(x, y, cx, cy, B):
        h = np.maximum(0.0, eta0 - B)
        return h, np.zeros_like(h), np.zeros_like(h)
    return init


def smooth_bump_bed(depth: float = 2.0, amp: float = 0.8, x0=0.5, y0=0.5, w=0.15):
    return lambda x, y, cx=None, cy=None: -depth + amp * np.exp(
        -((x - x0) ** 2 + (y - y0) ** 2) / w ** 2)


def step_bed_by_centroid(x_step: float, low: float, high: float, slope: float = 0.0):
    """A bed that jumps across element faces: ``low`` left of x_step, ``high`` right
    of it (decided by element centroid), plus an optional linear slope in x, so it
    is discontinuous between elements and smooth inside each one."""
    def bed(x, y, cx, cy=None):
        base = np.where(np.asarray(cx) < x_step, low, high)
        return base + slope * np.asarray(x)
    return bed


# ----------------------------------------------------------------------------
# the benchmark configurations


def hump_square(n: int = 16, N: int = 2, steps: int = 100) -> Scenario:
    """Unit square, n x n x 2 triangles, flat bed of depth 1, Gaussian hump 0.01/0.1."""
    return Scenario(
        name=f"hump_square_{n}x{n}x2_N{N}",
        mesh=lambda: meshes.structured_rect(0.0, 1.0, 0.0, 1.0, n, n),
        N=N, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=0, tvb_M=0.0,
        bathymetry=flat_bed(1.0), init=gaussian_hump_init(0.01, 0.5, 0.5, 0.1),
        steps=steps, note="plain method, single-rate AB3")


def dam_break(nx: int = 320, ny: int = 32, N: int = 3, steps: int = 2000) -> Scenario:
    """[0,20] x [0,2], dam at x = 10 on an element edge, flat dry bed to the right."""
    return Scenario(
        name=f"dam_break_{nx}x{ny}x2_N{N}",
        mesh=lambda: meshes.structured_rect(0.0, 20.0, 0.0, 2.0, nx, ny),
        N=N, g=9.81, h0=1e-5, cfl=0.5, nlevels=1, limiter_mask=LIM_PP | LIM_TVB,
        tvb_M=0.0, bathymetry=flat_bed(0.0), init=dam_init(10.0, 1.0), steps=steps,
        note="wet/dry dam break, PP + TVB (M=0) every stage")


def tsunami(nx: int = 1000, ny: int = 250, N: int = 4, seed: int = 3, nlevels: int = 4,
            steps: int = 200, amp: float = 2.0, src=(200e3, 50e3),
            limiter_mask: int = LIM_PP | LIM_TVB, tvb_M: float = 1e-3) -> Scenario:
    """400 km x 100 km, x-graded 8:1 toward a tanh beach, seeded jitter, MRAB levels."""
    return Scenario(
        name=f"tsunami_{nx}x{ny}x2_N{N}_L{nlevels}",
        mesh=lambda: meshes.graded_jittered_rect(0.0, 400e3, 0.0, 100e3, nx, ny,
                                                 ratio=8.0, jitter=0.15, seed=seed),
        N=N, g=9.81, h0=1e-3, cfl=0.5, nlevels=nlevels, limiter_mask=limiter_mask,
        tvb_M=tvb_M, bathymetry=tanh_beach(),
        init=bump_on_beach_init(amp, src[0], src[1], 10e3), steps=steps,
        note="tsunami-like run-up, MRAB3")


def ensemble(n: int = 64, seed: int = 4, kmin: int = 5000, kmax: int = 200000,
             orders=(3, 4, 5), nlevels: int = 4, steps: int = 500):
    """Uneven scenarios: K log-uniform, aspect 4:1 grids, random source and amplitude."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(n):
        K = float(np.exp(rng.uniform(math.log(kmin), math.log(kmax))))
        ny = max(2, int(round(math.sqrt(K / 8.0))))
        nx = 4 * ny
        N = int(rng.choice(orders))
        sx = float(rng.uniform(20e3, 200e3))
        sy = float(rng.uniform(10e3, 90e3))
        amp = float(rng.uniform(0.5, 5.0))
        sc = tsunami(nx=nx, ny=ny, N=N, seed=seed * 1000 + i, nlevels=nlevels, steps=steps,
                     amp=amp, src=(sx, sy))
        sc.name = f"ens{i:02d}_" + sc.name
        out.append(sc)
    return out


def served_stream(rate: float = 50.0, duration: float = 60.0, seed: int = 5,
                  kmin: int = 2000, kmax: int = 1000000, orders=(2, 3, 4),
                  steps: int = 500, nlevels: int = 4):
    """Poisson arrivals: list of (arrival_time_s, Scenario)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            break
        K = float(np.exp(rng.uniform(math.log(kmin), math.log(kmax))))
        ny = max(2, int(round(math.sqrt(K / 8.0))))
        nx = 4 * ny
        N = int(rng.choice(orders))
        sx = float(rng.uniform(20e3, 200e3))
        sy = float(rng.uniform(10e3, 90e3))
        amp = float(rng.uniform(0.5, 5.0))
        sc = tsunami(nx=nx, ny=ny, N=N, seed=seed * 100000 + len(out), nlevels=nlevels,
                     steps=steps, amp=amp, src=(sx, sy))
        out.append((t, sc))
    return out
