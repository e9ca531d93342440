"""Pins of the oracle's EDAC form (the entropically damped artificial compressibility scheme
of the scheme list of Sec. 2.3, with which Sec. 4.1 solves the Taylor-Green vortex):

  dp/dt = -rho0 c0^2 div u + nu_e lap p,   nu_e = edac_alpha h c0 / 8,   rho = rho0,

each discrete term against its continuum limit on a lattice, the order of the step (the
pressure advanced with the rate at the new positions and half-step velocities before the
momentum equation reads it) against the step composed by hand from single evaluations,
and the whole method against the exact Taylor-Green solution printed in Sec. 4.1."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from test_oracle_physics import block, with_


def _edac_block(kind, hdx):
    wl, s, inner = block(kind, hdx)
    wl.density = 2
    s = with_(s, p=np.zeros_like(s["x"]))
    return wl, s, inner


@pytest.mark.parametrize("kind,hdx,tol", [(W.QUINTIC, 1.0, 2e-3), (W.WENDLAND_C2, 2.0, 2e-3),
                                          (W.CUBIC_SPLINE, 2.0, 2e-3)])
def test_divergence_term_limit(kind, hdx, tol):
    """Uniform pressure, u = (beta x, 0): div u = beta, so dp/dt = -rho0 c0^2 beta."""
    wl, s, inner = _edac_block(kind, hdx)
    beta = 0.3
    r = O.rhs(wl, with_(s, u=beta * s["x"]))
    assert np.max(np.abs(r["arho"][inner] / (-wl.rho0 * wl.c0 ** 2 * beta) - 1.0)) < tol


@pytest.mark.parametrize("kind,hdx,tol", [(W.QUINTIC, 1.0, 1e-2), (W.WENDLAND_C2, 2.0, 2e-2),
                                          (W.CUBIC_SPLINE, 2.0, 2e-2)])
def test_pressure_diffusion_limit(kind, hdx, tol):
    """At rest with p = y^2: lap p = 2, so dp/dt = 2 nu_e with nu_e = alpha h c0 / 8 (the
    0.01 h^2 regulariser of the Laplacian form costs about 1 %, as in the laminar term)."""
    wl, s, inner = _edac_block(kind, hdx)
    for alpha in (0.5, 1.0):
        wl.edac_alpha = alpha
        r = O.rhs(wl, with_(s, p=s["y"] ** 2))
        nu_e = alpha * wl.h * wl.c0 / 8.0
        assert np.max(np.abs(r["arho"][inner] / (2.0 * nu_e) - 1.0)) < tol
    wl.edac_alpha = 0.0  # no diffusivity: a pressure field at rest does not change
    r = O.rhs(wl, with_(s, p=s["y"] ** 2))
    assert np.max(np.abs(r["arho"])) == 0.0


def test_pressure_drives_the_momentum_equation():
    """The momentum equation reads the EDAC pressure (not an EOS of the density): at rest
    with p = eps x, a_x = -dp/dx / rho0 in the interior."""
    wl, s, inner = _edac_block(W.QUINTIC, 1.0)
    eps = 0.02
    r = O.rhs(wl, with_(s, p=eps * s["x"]))
    assert np.max(np.abs(r["ax"][inner] / (-eps / wl.rho0) - 1.0)) < 2e-3
    assert np.all(r["rho"] == wl.rho0)  # the density is held


def test_one_step_composed_by_hand():
    """Kick-drift-kick with the pressure advanced like the density of the continuity form:
    u_half = u + dt/2 a(x, u, p); x1 = x + dt u_half; p1 = p + dt dp/dt(x1, u_half, p);
    u1 = u_half + dt/2 a(x1, u_half, p1)."""
    wl = W.taylor_green_2d_edac(n=20)
    s = O.state_of(wl)
    dt = wl.dt
    r0 = O.rhs(wl, s)
    uh = {k: s[k] + 0.5 * dt * r0["a" + a] for k, a in (("u", "x"), ("v", "y"))}
    x1 = np.mod(s["x"] + dt * uh["u"], 1.0)
    y1 = np.mod(s["y"] + dt * uh["v"], 1.0)
    mid = with_(s, x=x1, y=y1, u=uh["u"], v=uh["v"])
    p1 = s["p"] + dt * O.rhs(wl, mid)["arho"]
    r1 = O.rhs(wl, with_(mid, p=p1))
    st, _ = O.run(wl, s, dt, 1)
    assert np.max(np.abs(st["p"] - p1)) <= 1e-13 * np.max(np.abs(p1))
    for k, a in (("u", "x"), ("v", "y")):
        assert np.max(np.abs(st[k] - (uh[k] + 0.5 * dt * r1["a" + a]))) <= 1e-14
    assert np.max(np.abs(st["x"] - x1)) <= 1e-15 and np.all(st["rho"] == wl.rho0)


def test_taylor_green_decay_and_pressure():
    """Sec. 4.1: with the exact fields at t = 0, max |u| follows U exp(b t), b = -8 pi^2/Re,
    the velocity field stays on the exact one, and the pressure tracks the exact
    -U^2 exp(2 b t) (cos 4 pi x + cos 4 pi y) / 4 (the artificial compressibility lets it
    deviate by a few per cent over the first acoustic times)."""
    wl = W.taylor_green_2d_edac(n=50)
    s = O.state_of(wl)
    b = -8 * math.pi ** 2 / 100.0
    st = s
    t = 0.0
    for steps in (50, 50):
        st, h = O.run(wl, st, wl.dt, steps)
        t += steps * wl.dt
        assert abs(h[-1, 3] / math.exp(b * t) - 1.0) < 2e-3
        ue = -math.exp(b * t) * np.cos(2 * np.pi * st["x"]) * np.sin(2 * np.pi * st["y"])
        pe = -math.exp(2 * b * t) * (np.cos(4 * np.pi * st["x"]) + np.cos(4 * np.pi * st["y"])) / 4
        assert np.linalg.norm(st["u"] - ue) / np.linalg.norm(ue) < 1e-2
        assert np.linalg.norm(st["p"] - pe) / np.linalg.norm(pe) < 0.1
        assert np.all(st["rho"] == wl.rho0)
    assert abs(math.log(h[-1, 3]) / t / b - 1.0) < 0.02


def test_walls_and_the_midpoint_integrator_are_refused():
    wl = W.dam_break_2d(dx=0.1, precision=W.PREC_FP64)
    wl.density = 2
    with pytest.raises(ValueError):
        O.rhs(wl, O.state_of(wl))
    wl = W.taylor_green_2d_edac(n=10).with_integrator(1)
    with pytest.raises(ValueError):
        O.run(wl, O.state_of(wl), wl.dt, 1)
    with pytest.raises(ValueError):
        O.grad(W.taylor_green_2d_edac(n=10), O.state_of(W.taylor_green_2d_edac(n=10)), 1e-4, 1,
               dnu=1.0)
