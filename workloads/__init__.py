"""Seeded synthetic inputs shaped like the test problems of the PySPH paper.

This module builds particle lattices, jitter, masses, the closed-form initial
velocity of the Taylor-Green problem (Sec. 4.1) and the run parameters of each
workload. It holds none of the SPH method's arithmetic (no kernel, no equation
of state, no pair sum, no integrator). It is the only code shared by the CUDA
path (tests, bench) and the CPU oracle: both receive exactly the same arrays.

Workloads (sizes follow the five benchmark configurations of the WCSPH hot path):

* ``taylor_green_2d``  periodic unit square, n x n jittered lattice, quintic kernel,
  h = dx, laminar viscosity nu = U L / Re (Sec. 4.1 closed form at t = 0).
* ``dam_break_2d``     1 x 2 m fluid column at dx = 0.01 in a 4 x 4 m tank with three
  layers of wall particles (Sec. 3.2 geometry), Wendland C2 kernel, h = 1.3 dx,
  Monaghan artificial viscosity alpha = 0.1, XSPH eps = 0.5, g = -9.81.
* ``taylor_green_3d``  periodic unit cube, the 2D Taylor-Green field extruded in z.
* ``batch_tg2d``       many independent Taylor-Green instances of uneven size.
* ``dam_break_3d``     1 x 0.5 x 0.5 m block at dx = 0.005 in a 3.2 x 1.0 m tank with
  three wall layers 0.5 m high (906,828 wall particles).
* ``gaussian_blob``    particles with their own smoothing lengths (normally distributed
  positions, h from the local number density) for the variable-support search.

Seeds: numpy PCG64 with seed = 1909_04504 + workload index unless given.
Jitter: independent U[-j dx, +j dx] per coordinate.
Initial density: uniform rho0 for every particle; initial pressure follows from it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 1909_04504

QUINTIC = 0
WENDLAND_C2 = 1
CUBIC_SPLINE = 2
FLUID = 0
WALL = 1
PREC_FP64 = 0
PREC_FP32 = 1


@dataclass
class ParticleSet:
    """One named particle array (fluid or wall), all properties as float64."""
    name: str
    role: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    u: np.ndarray
    v: np.ndarray
    w: np.ndarray
    rho: np.ndarray
    m: np.ndarray
    p: Optional[np.ndarray] = None  # pressure of the EDAC form (a state variable there)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


@dataclass
class Workload:
    """Domain, particle arrays and run parameters of one synthetic problem."""
    name: str
    dim: int
    kernel: int
    h: float
    lo: List[float]
    hi: List[float]
    periodic: List[int]
    precision: int
    arrays: List[ParticleSet]
    rho0: float
    c0: float
    gamma: float = 7.0
    nu: float = 0.0
    eta: float = 0.01
    alpha: float = 0.0
    xsph_eps: float = 0.0
    g: List[float] = field(default_factory=lambda: [0.0, 0.0, 0.0])
    density: int = 0          # 0 continuity, 1 summation density, 2 EDAC pressure equation
    edac_alpha: float = 0.5   # EDAC pressure diffusivity nu_e = edac_alpha h c0 / 8
    wall_bc: int = 0          # 0 wall density from continuity, 1 wall pressure of Adami et al.
    integrator: int = 0       # 0 kick-drift-kick, 1 midpoint predict-evaluate-correct
    dt: float = 0.0
    steps: int = 1

    @property
    def n_total(self) -> int:
        return sum(a.n for a in self.arrays)

    @property
    def n_fluid(self) -> int:
        return sum(a.n for a in self.arrays if a.role == FLUID)

    def concat(self, prop: str) -> np.ndarray:
        """Property concatenated over arrays in the given order (global particle ids); an
        array without a pressure contributes zeros to ``p``."""
        return np.concatenate([
            np.zeros(a.n) if prop == "p" and a.p is None else getattr(a, prop)
            for a in self.arrays])

    def roles(self) -> np.ndarray:
        return np.concatenate([np.full(a.n, a.role, dtype=np.uint8) for a in self.arrays])

    def with_precision(self, precision: int) -> "Workload":
        import copy
        w = copy.deepcopy(self)
        w.precision = precision
        return w

    def with_wall_bc(self, wall_bc: int) -> "Workload":
        import copy
        w = copy.deepcopy(self)
        w.wall_bc = wall_bc
        w.name = self.name + ("_adami" if wall_bc == 1 else "")
        return w

    def with_integrator(self, integrator: int) -> "Workload":
        import copy
        w = copy.deepcopy(self)
        w.integrator = integrator
        w.name = self.name + ("_pec" if integrator == 1 else "")
        return w


def _rng(seed: Optional[int], index: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + index if seed is None else seed))


def _zeros(n: int) -> np.ndarray:
    return np.zeros(n, dtype=np.float64)


def taylor_green_2d(n: int = 50, jitter: float = 0.05, re: float = 100.0, U: float = 1.0,
                    rho0: float = 1.0, c0: float = 10.0, steps: int = 200,
                    precision: int = PREC_FP64, seed: Optional[int] = None,
                    hdx: float = 1.0) -> Workload:
    """2D Taylor-Green vortex on the periodic unit square (Sec. 4.1).

    Velocity at t = 0 from the printed exact solution:
    u = -U cos(2 pi x) sin(2 pi y), v = U sin(2 pi x) cos(2 pi y).
    """
    rng = _rng(seed, 0)
    dx = 1.0 / n
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = (i.ravel() + 0.5) * dx
    y = (j.ravel() + 0.5) * dx
    if jitter > 0.0:
        x = x + rng.uniform(-jitter * dx, jitter * dx, x.shape)
        y = y + rng.uniform(-jitter * dx, jitter * dx, y.shape)
    N = x.shape[0]
    u = -U * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = U * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    h = hdx * dx
    fluid = ParticleSet("fluid", FLUID, x, y, _zeros(N), u, v, _zeros(N),
                        np.full(N, rho0), np.full(N, rho0 * dx * dx))
    return Workload(name=f"taylor_green_2d_{n}x{n}", dim=2, kernel=QUINTIC, h=h,
                    lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 0.0], periodic=[1, 1, 0],
                    precision=precision, arrays=[fluid], rho0=rho0, c0=c0,
                    nu=U * 1.0 / re, dt=0.25 * h / c0, steps=steps)


def taylor_green_2d_edac(n: int = 100, hdx: float = 1.2, re: float = 100.0, U: float = 1.0,
                         rho0: float = 1.0, c0: float = 10.0, steps: int = 0,
                         jitter: float = 0.0, precision: int = PREC_FP64,
                         seed: Optional[int] = None, t_end: float = 2.0) -> Workload:
    """The Taylor-Green vortex as Sec. 4.1 runs it with the EDAC scheme: periodic unit
    square, n x n lattice (100 x 100 in the paper), quintic kernel with h = 1.2 dx, U = 1,
    Re = 100, up to t = 2 s. Velocity and pressure at t = 0 from the printed exact solution,
    p = -U^2 (cos(4 pi x) + cos(4 pi y)) / 4 (times rho0); the density stays rho0.
    ``steps`` = 0 takes t_end / dt steps."""
    wl = taylor_green_2d(n=n, jitter=jitter, re=re, U=U, rho0=rho0, c0=c0, precision=precision,
                         seed=seed, hdx=hdx)
    a = wl.arrays[0]
    a.p = -rho0 * U * U * (np.cos(4 * np.pi * a.x) + np.cos(4 * np.pi * a.y)) / 4.0
    wl.density = 2
    wl.name = f"taylor_green_2d_edac_{n}x{n}"
    wl.steps = steps if steps > 0 else int(round(t_end / wl.dt))
    return wl


def taylor_green_3d(n: int = 64, jitter: float = 0.05, re: float = 100.0, U: float = 1.0,
                    rho0: float = 1.0, c0: float = 10.0, steps: int = 50,
                    precision: int = PREC_FP32, seed: Optional[int] = None) -> Workload:
    """Periodic unit cube carrying the 2D Taylor-Green field extruded in z (w = 0)."""
    rng = _rng(seed, 2)
    dx = 1.0 / n
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    x = (i.ravel() + 0.5) * dx
    y = (j.ravel() + 0.5) * dx
    z = (k.ravel() + 0.5) * dx
    if jitter > 0.0:
        x = x + rng.uniform(-jitter * dx, jitter * dx, x.shape)
        y = y + rng.uniform(-jitter * dx, jitter * dx, y.shape)
        z = z + rng.uniform(-jitter * dx, jitter * dx, z.shape)
    N = x.shape[0]
    u = -U * np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = U * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    fluid = ParticleSet("fluid", FLUID, x, y, z, u, v, _zeros(N),
                        np.full(N, rho0), np.full(N, rho0 * dx ** 3))
    h = dx
    return Workload(name=f"taylor_green_3d_{n}^3", dim=3, kernel=QUINTIC, h=h,
                    lo=[0.0, 0.0, 0.0], hi=[1.0, 1.0, 1.0], periodic=[1, 1, 1],
                    precision=precision, arrays=[fluid], rho0=rho0, c0=c0,
                    nu=U * 1.0 / re, dt=0.25 * h / c0, steps=steps)


def dam_break_2d(dx: float = 0.01, fluid_w: float = 1.0, fluid_h: float = 2.0,
                 tank_w: float = 4.0, tank_h: float = 4.0, layers: int = 3,
                 hdx: float = 1.3, rho0: float = 1000.0, gravity: float = 9.81,
                 alpha: float = 0.1, xsph_eps: float = 0.5, steps: int = 2000,
                 precision: int = PREC_FP32, box_top: float = 8.0) -> Workload:
    """2D dam break (the Sec. 3.2 example problem) at the benchmark resolution.

    Fluid centres ((i+1/2)dx, (j+1/2)dx) fill [0, fluid_w] x [0, fluid_h]. The tank
    interior is [0, tank_w] x [0, tank_h]; its side walls are ``layers`` columns at
    -(k+1/2)dx and tank_w+(k+1/2)dx for the full tank height, its floor is
    ``layers`` rows at -(k+1/2)dx including the corners; the top is open.
    c0 = 10 sqrt(2 g H) with H the column height; dt = 0.25 h / c0.
    """
    nfx = int(round(fluid_w / dx))
    nfy = int(round(fluid_h / dx))
    i, j = np.meshgrid(np.arange(nfx), np.arange(nfy), indexing="ij")
    xf = (i.ravel() + 0.5) * dx
    yf = (j.ravel() + 0.5) * dx
    ntx = int(round(tank_w / dx))
    nty = int(round(tank_h / dx))
    xs, ys = [], []
    rows = (np.arange(nty) + 0.5) * dx
    for k in range(layers):
        for xw in (-(k + 0.5) * dx, tank_w + (k + 0.5) * dx):
            xs.append(np.full(nty, xw))
            ys.append(rows)
    cols = (np.arange(-layers, ntx + layers) + 0.5) * dx
    for k in range(layers):
        xs.append(cols)
        ys.append(np.full(cols.shape[0], -(k + 0.5) * dx))
    xw = np.concatenate(xs)
    yw = np.concatenate(ys)
    m = rho0 * dx * dx
    nf, nw = xf.shape[0], xw.shape[0]
    fluid = ParticleSet("fluid", FLUID, xf, yf, _zeros(nf), _zeros(nf), _zeros(nf), _zeros(nf),
                        np.full(nf, rho0), np.full(nf, m))
    wall = ParticleSet("wall", WALL, xw, yw, _zeros(nw), _zeros(nw), _zeros(nw), _zeros(nw),
                       np.full(nw, rho0), np.full(nw, m))
    h = hdx * dx
    c0 = 10.0 * math.sqrt(2.0 * gravity * fluid_h)
    pad = layers * dx
    return Workload(name=f"dam_break_2d_{nf}+{nw}", dim=2, kernel=WENDLAND_C2, h=h,
                    lo=[-pad, -pad, 0.0], hi=[tank_w + pad, box_top, 0.0],
                    periodic=[0, 0, 0], precision=precision, arrays=[fluid, wall],
                    rho0=rho0, c0=c0, alpha=alpha, xsph_eps=xsph_eps,
                    g=[0.0, -gravity, 0.0], dt=0.25 * h / c0, steps=steps)


def dam_break_3d(dx: float = 0.005, block=(1.0, 0.5, 0.5), tank=(3.2, 1.0, 1.0),
                 wall_height: float = 0.5, layers: int = 3, hdx: float = 1.3,
                 rho0: float = 1000.0, gravity: float = 9.81, alpha: float = 0.1,
                 xsph_eps: float = 0.5, steps: int = 1000,
                 precision: int = PREC_FP32) -> Workload:
    """3D dam break: fluid block at the x = 0 end of a tank, z vertical.

    The block fills [0, bx] x [0, by] x [0, bz]. Wall particles: ``layers`` floor
    layers under the tank footprint (corners included) and a ring of ``layers``
    layers around the footprint up to ``wall_height``. With the defaults this
    gives 2,000,000 fluid and 906,828 wall particles. The cell box reaches the
    tank top. c0 = 10 sqrt(2 g H) with H the block height.
    """
    nbx, nby, nbz = (int(round(b / dx)) for b in block)
    i, j, k = np.meshgrid(np.arange(nbx), np.arange(nby), np.arange(nbz), indexing="ij")
    xf = (i.ravel() + 0.5) * dx
    yf = (j.ravel() + 0.5) * dx
    zf = (k.ravel() + 0.5) * dx
    ntx, nty = int(round(tank[0] / dx)), int(round(tank[1] / dx))
    nwz = int(round(wall_height / dx))
    gx = np.arange(-layers, ntx + layers)
    gy = np.arange(-layers, nty + layers)
    GX, GY = np.meshgrid(gx, gy, indexing="ij")
    GX, GY = GX.ravel(), GY.ravel()
    ring = (GX < 0) | (GX >= ntx) | (GY < 0) | (GY >= nty)
    xs, ys, zs = [], [], []
    for l in range(layers):
        xs.append((GX + 0.5) * dx)
        ys.append((GY + 0.5) * dx)
        zs.append(np.full(GX.shape[0], -(l + 0.5) * dx))
    RX, RY = GX[ring], GY[ring]
    for kz in range(nwz):
        xs.append((RX + 0.5) * dx)
        ys.append((RY + 0.5) * dx)
        zs.append(np.full(RX.shape[0], (kz + 0.5) * dx))
    xw, yw, zw = np.concatenate(xs), np.concatenate(ys), np.concatenate(zs)
    m = rho0 * dx ** 3
    nf, nw = xf.shape[0], xw.shape[0]
    fluid = ParticleSet("fluid", FLUID, xf, yf, zf, _zeros(nf), _zeros(nf), _zeros(nf),
                        np.full(nf, rho0), np.full(nf, m))
    wall = ParticleSet("wall", WALL, xw, yw, zw, _zeros(nw), _zeros(nw), _zeros(nw),
                       np.full(nw, rho0), np.full(nw, m))
    h = hdx * dx
    c0 = 10.0 * math.sqrt(2.0 * gravity * block[2])
    pad = layers * dx
    return Workload(name=f"dam_break_3d_{nf}+{nw}", dim=3, kernel=WENDLAND_C2, h=h,
                    lo=[-pad, -pad, -pad], hi=[tank[0] + pad, tank[1] + pad, tank[2]],
                    periodic=[0, 0, 0], precision=precision, arrays=[fluid, wall],
                    rho0=rho0, c0=c0, alpha=alpha, xsph_eps=xsph_eps,
                    g=[0.0, 0.0, -gravity], dt=0.25 * h / c0, steps=steps)


def falling_cube_3d(n: int = 100, side: float = 1.0, hdx: float = 1.2, rho0: float = 1000.0,
                    gravity: float = 9.81, alpha: float = 0.1, xsph_eps: float = 0.0,
                    fall: float = 0.5, steps: int = 1000,
                    precision: int = PREC_FP32) -> Workload:
    """A cube of water falling freely under gravity, no walls (the problem of the
    performance measurements of Sec. 4.4), z vertical.

    n^3 fluid particles at the centres of a lattice of spacing dx = side / n filling
    [0, side]^3, at rest, rho = rho0; cubic spline kernel with h = hdx dx. The cell box
    leaves one support around the cube and ``fall`` below it (particles that leave it are
    clamped into the edge cells). c0 = 10 sqrt(2 g side), dt = 0.25 h / c0.
    """
    dx = side / n
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xf = (i.ravel() + 0.5) * dx
    yf = (j.ravel() + 0.5) * dx
    zf = (k.ravel() + 0.5) * dx
    nf = xf.shape[0]
    fluid = ParticleSet("fluid", FLUID, xf, yf, zf, _zeros(nf), _zeros(nf), _zeros(nf),
                        np.full(nf, rho0), np.full(nf, rho0 * dx ** 3))
    h = hdx * dx
    kh = 2.0 * h
    c0 = 10.0 * math.sqrt(2.0 * gravity * side)
    return Workload(name=f"falling_cube_3d_{n}^3", dim=3, kernel=CUBIC_SPLINE, h=h,
                    lo=[-kh, -kh, -fall], hi=[side + kh, side + kh, side + kh],
                    periodic=[0, 0, 0], precision=precision, arrays=[fluid],
                    rho0=rho0, c0=c0, alpha=alpha, xsph_eps=xsph_eps,
                    g=[0.0, 0.0, -gravity], dt=0.25 * h / c0, steps=steps)


def batch_tg2d(instances: int = 64, n_min: int = 2500, n_max: int = 40000,
               re_min: float = 50.0, re_max: float = 1000.0, steps: int = 500,
               precision: int = PREC_FP32, seed: Optional[int] = None) -> List[Workload]:
    """Independent 2D Taylor-Green instances of uneven size.

    For each instance k: N_k ~ U[n_min, n_max], n_k = round(sqrt(N_k)) particles per
    side, Re_k ~ U[re_min, re_max]; dx = 1/n_k, h = dx, dt_k = 0.25 h_k / c0.
    """
    rng = _rng(seed, 3)
    counts = rng.uniform(n_min, n_max, instances)
    res = rng.uniform(re_min, re_max, instances)
    out = []
    for k in range(instances):
        n = int(round(math.sqrt(counts[k])))
        w = taylor_green_2d(n=n, re=float(res[k]), steps=steps, precision=precision,
                            seed=SEED_BASE + 1000 + k)
        w.name = f"tg2d_instance{k}_{n}x{n}"
        out.append(w)
    return out


@dataclass
class VHSet:
    """Particles with their own smoothing lengths (the variable-support case of Sec. 2.2
    that the paper searches with an octree): positions, h and masses, all FP64."""
    name: str
    dim: int
    kernel: int
    precision: int
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    h: np.ndarray
    m: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def gaussian_blob(n: int = 1_000_000, dim: int = 3, eta: float = 1.2, cut: float = 3.0,
                  kernel: int = WENDLAND_C2, precision: int = PREC_FP32,
                  seed: Optional[int] = None) -> VHSet:
    """A self-gravitating-cloud-like particle set: n positions drawn from an isotropic
    normal distribution of unit variance, truncated at radius ``cut`` (draws beyond it are
    redrawn), equal masses 1 / n, and h_i = eta (m / rho(r_i))^(1/dim) from the number
    density of that distribution, rho(r) = exp(-r^2 / 2) / ((2 pi)^(dim/2) P(r < cut)).
    The support radius grows by exp(cut^2 / (2 dim)) from the centre to the edge (4.5x in
    3D, 9.5x in 2D) while the density falls by exp(cut^2 / 2) = 90x.
    """
    rng = _rng(seed, 7 if dim == 3 else 6)
    pts = np.zeros((0, dim))
    while pts.shape[0] < n:
        draw = rng.normal(size=(2 * (n - pts.shape[0]) + 16, dim))
        draw = draw[np.sum(draw * draw, axis=1) < cut * cut]
        pts = np.vstack([pts, draw[:n - pts.shape[0]]])
    r2 = np.sum(pts * pts, axis=1)
    if dim == 3:
        inside = math.erf(cut / math.sqrt(2.0)) - math.sqrt(2.0 / math.pi) * cut * math.exp(-cut * cut / 2)
    else:
        inside = 1.0 - math.exp(-cut * cut / 2)
    rho = np.exp(-0.5 * r2) / ((2.0 * math.pi) ** (dim / 2.0) * inside)
    m = np.full(n, 1.0 / n)
    h = eta * (m / rho) ** (1.0 / dim)
    z = pts[:, 2].copy() if dim == 3 else _zeros(n)
    return VHSet(name=f"gaussian_blob_{dim}d_{n}", dim=dim, kernel=kernel, precision=precision,
                 x=pts[:, 0].copy(), y=pts[:, 1].copy(), z=z, h=h, m=m)


def config(index: int, small: bool = False):
    """The five benchmark workloads by index (0..4).

    ``small`` returns a reduced copy of the same structure for quick checks.
    """
    if index == 0:
        return taylor_green_2d(n=20 if small else 50, steps=20 if small else 200)
    if index == 1:
        if small:
            return dam_break_2d(dx=0.04, steps=20)
        return dam_break_2d()
    if index == 2:
        return taylor_green_3d(n=16 if small else 64, steps=5 if small else 50)
    if index == 3:
        if small:
            return batch_tg2d(instances=4, n_min=400, n_max=1600, steps=10)
        return batch_tg2d()
    if index == 4:
        if small:
            return dam_break_3d(dx=0.04, steps=3)
        return dam_break_3d()
    raise ValueError(f"unknown workload index {index}")
