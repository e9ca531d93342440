"""Pins of the oracle's forward-mode derivative of the final kinetic energy, which is the
reference for the hand-written adjoint: the K = 0 closed form and central finite
differences of the plain FP64 run (the kernels vanish smoothly at the support edge, so
neighbour-set changes under a small perturbation contribute almost nothing)."""
import numpy as np
import pytest

import oracle as O
import workloads as W


def small_tg(n=12, dim=2):
    wl = W.taylor_green_2d(n=n) if dim == 2 else W.taylor_green_3d(n=n)
    wl.nu = 0.05
    return wl, O.state_of(wl)


def ke_of(st):
    fluid = st["role"] == W.FLUID
    return 0.5 * np.sum(st["m"][fluid] * (st["u"] ** 2 + st["v"] ** 2 + st["w"] ** 2)[fluid])


def test_k0_closed_form():
    wl, s = small_tg()
    rng = np.random.Generator(np.random.PCG64(1))
    du, dv = rng.normal(size=s["x"].shape), rng.normal(size=s["x"].shape)
    ke, dke = O.grad(wl, s, wl.dt, 0, du=du, dv=dv)
    assert abs(ke - ke_of(s)) < 1e-15
    assert abs(dke - np.sum(s["m"] * (s["u"] * du + s["v"] * dv))) < 1e-14
    _, dnu = O.grad(wl, s, wl.dt, 0, dnu=1.0)
    assert dnu == 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_velocity_direction_matches_central_differences(dim):
    wl, s = small_tg(12 if dim == 2 else 10, dim)
    K = 8
    rng = np.random.Generator(np.random.PCG64(2))
    d = {k: rng.normal(size=s["x"].shape) for k in ("u", "v", "w")[:dim]}
    norm = np.sqrt(sum(np.sum(v * v) for v in d.values()))
    d = {k: v / norm for k, v in d.items()}
    ke, dke = O.grad(wl, s, wl.dt, K, du=d.get("u"), dv=d.get("v"), dw=d.get("w"))
    unorm = np.sqrt(np.sum(s["u"] ** 2 + s["v"] ** 2 + s["w"] ** 2))
    eps = 1e-3 * unorm
    vals = []
    for sign in (1, -1):
        sp = dict(s)
        for k, v in d.items():
            sp[k] = s[k] + sign * eps * v
        st, _ = O.run(wl, sp, wl.dt, K)
        vals.append(ke_of(st))
    fd = (vals[0] - vals[1]) / (2 * eps)
    st, _ = O.run(wl, s, wl.dt, K)
    assert abs(ke - ke_of(st)) < 1e-14
    assert abs(dke - fd) < 1e-5 * abs(fd)


@pytest.mark.parametrize("alpha", [0.0, 0.1])
def test_viscosity_derivative_matches_central_differences(alpha):
    wl, s = small_tg()
    wl.alpha = alpha
    K = 10
    _, dke = O.grad(wl, s, wl.dt, K, dnu=1.0)
    eps = 1e-3 * wl.nu
    vals = []
    for sign in (1, -1):
        st, _ = O.run(wl, s, wl.dt, K, nu=wl.nu + sign * eps)
        vals.append(ke_of(st))
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert dke < 0.0  # more viscosity, less kinetic energy
    assert abs(dke - fd) < 1e-5 * abs(fd)


def test_alpha_derivative_matches_central_differences():
    wl, s = small_tg()
    wl.alpha = 0.1
    K = 10
    _, dke = O.grad(wl, s, wl.dt, K, dalpha=1.0)
    eps = 1e-3 * wl.alpha
    vals = []
    for sign in (1, -1):
        st, _ = O.run(wl, s, wl.dt, K, alpha=wl.alpha + sign * eps)
        vals.append(ke_of(st))
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(dke - fd) < 1e-4 * abs(fd)


def test_walls_and_gravity_direction_derivative():
    """Dam-break geometry (walls, AV, XSPH, gravity): derivative along a velocity direction."""
    wl = W.dam_break_2d(dx=0.08)
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(9))
    fluid = s["role"] == W.FLUID
    s["u"] = np.where(fluid, 0.3 * rng.normal(size=s["x"].shape), 0.0)
    s["v"] = np.where(fluid, 0.3 * rng.normal(size=s["x"].shape), 0.0)
    du = np.where(fluid, rng.normal(size=s["x"].shape), 0.0)
    K = 6
    _, dke = O.grad(wl, s, wl.dt, K, du=du)
    eps = 1e-4
    vals = []
    for sign in (1, -1):
        st, _ = O.run(wl, dict(s, u=s["u"] + sign * eps * du), wl.dt, K)
        vals.append(ke_of(st))
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(dke - fd) < 1e-4 * abs(fd)
