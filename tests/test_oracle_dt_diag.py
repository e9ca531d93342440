"""Pins of the oracle's time-step selection and of its diagnostics record.

Time step (Sec. 2.1 asks for a CFL-type criterion and prints no formula; the reading
takes the three classical bounds): dt = min(0.25 h / (c0 + max|u|) [acoustic CFL,
Monaghan 1992], 0.25 sqrt(h / max|a|) [body force, Monaghan 1992],
0.125 h^2 / nu [explicit viscous diffusion, Morris, Fox and Zhu 1997]). Each test puts the
oracle in a regime where max|u| and max|a| are known in closed form from the physics (a
lone particle in free fall, a uniformly translating lattice, a fluid at rest), so a wrong
constant, a dropped bound or a stale max|u| changes the time sequence the run records.

Diagnostics record (t, dt, KE, max|u|, Px, Py, Pz, max|a|, pairs, candidates): checked
against numpy sums over the state the run returns and the rates of an independent
evaluation of the same state."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _lone(pos, vel, h=1.0, c0=0.1, g=(0.0, -9.81, 0.0), nu=0.0, dim=2, half=1e3):
    """One fluid particle in a box of half-width ``half`` (a few hundred cells per axis)."""
    fl = W.ParticleSet("fluid", W.FLUID, np.array([pos[0]]), np.array([pos[1]]),
                       np.array([pos[2]]), np.array([vel[0]]), np.array([vel[1]]),
                       np.array([vel[2]]), np.array([1000.0]), np.array([1.0]))
    return W.Workload(name="lone", dim=dim, kernel=W.WENDLAND_C2, h=h, lo=[-half] * 3,
                      hi=[half] * 3, periodic=[0, 0, 0], precision=W.PREC_FP64,
                      arrays=[fl], rho0=1000.0, c0=c0, nu=nu, g=list(g), dt=0.0)


def test_force_bound_then_acoustic_bound_in_free_fall():
    """A lone particle falling from rest: |a| = g exactly and |u_n| = g t_n exactly under
    kick-drift-kick, so the step sequence is dt_n = min(0.25 h / (c0 + g t_n),
    0.25 sqrt(h / g)). With h = 1 and c0 = 0.1 the force bound binds for the first steps
    and the acoustic bound after |u| passes about 3 m/s."""
    g, h, c0 = 9.81, 1.0, 0.1
    wl = _lone([0.0, 0.0, 0.0], [0.0, 0.0, 0.0], h=h, c0=c0)
    steps = 12
    st, hist = O.run(wl, O.state_of(wl), 0.0, steps)
    t = 0.0
    which = []
    for n in range(1, steps + 1):
        acoustic = 0.25 * h / (c0 + g * t)
        force = 0.25 * math.sqrt(h / g)
        dt = min(acoustic, force)
        which.append("force" if force < acoustic else "acoustic")
        assert hist[n, 1] == pytest.approx(dt, rel=1e-13, abs=0.0), n
        t += dt
        assert hist[n, 0] == pytest.approx(t, rel=1e-13, abs=0.0), n
        assert hist[n, 3] == pytest.approx(g * t, rel=1e-12), n   # max|u| = g t
        assert hist[n, 7] == pytest.approx(g, rel=1e-15), n       # max|a| = g
    assert "force" in which and "acoustic" in which  # both bounds were exercised
    assert st["v"][0] == pytest.approx(-g * t, rel=1e-12)


def test_acoustic_bound_for_a_uniform_translation():
    """A periodic lattice at rest density translating uniformly: every pair has v_ij = 0
    and p = 0, so a = 0 exactly and |u| = U for ever: dt = 0.25 h / (c0 + U) at every step
    (no force bound, no viscous bound)."""
    wl = W.taylor_green_2d(n=20, jitter=0.05, re=100.0)
    wl.nu = 0.0
    s = O.state_of(wl)
    U = (0.3, -0.4)
    s["u"][:] = U[0]
    s["v"][:] = U[1]
    speed = math.hypot(*U)
    st, hist = O.run(wl, s, 0.0, 5)
    expect = 0.25 * wl.h / (wl.c0 + speed)
    assert np.all(hist[:, 7] == 0.0)
    for n in range(1, 6):
        assert hist[n, 1] == pytest.approx(expect, rel=1e-14, abs=0.0)
        assert hist[n, 0] == pytest.approx(n * expect, rel=1e-13)
        assert hist[n, 3] == pytest.approx(speed, rel=1e-14)
    # the translation carries the lattice by U t (wrapped into the unit square)
    dx = np.mod(st["x"] - s["x"] - U[0] * 5 * expect + 0.5, 1.0) - 0.5
    assert np.max(np.abs(dx)) < 1e-13


def test_viscous_bound_for_a_very_viscous_taylor_green_vortex():
    """Re = 1 on a 20 x 20 lattice (h = 0.05, nu = 1): 0.125 h^2 / nu = 3.125e-4 lies below
    the acoustic bound 0.25 h / (c0 + U) ~ 1.1e-3 and the force bound 0.25 sqrt(h / |a|)
    with |a| ~ 8 pi^2 nu U ~ 79 (~6e-3), so every step takes the viscous bound."""
    wl = W.taylor_green_2d(n=20, re=1.0)
    assert wl.nu == 1.0
    s = O.state_of(wl)
    _, hist = O.run(wl, s, 0.0, 3)
    visc = 0.125 * wl.h * wl.h / wl.nu
    for n in range(1, 4):
        acoustic = 0.25 * wl.h / (wl.c0 + hist[n - 1, 3])
        force = 0.25 * math.sqrt(wl.h / hist[n - 1, 7])
        assert visc < acoustic and visc < force
        assert hist[n, 1] == pytest.approx(visc, rel=1e-15, abs=0.0)


def test_viscous_bound_for_a_fluid_at_rest():
    """A lone particle at rest with g = 0: a = 0, u = 0; nu = 1 > h c0 / 2 gives
    dt = 0.125 h^2 / nu, nu = 0 gives 0.25 h / c0."""
    h, c0 = 0.02, 10.0
    for nu, expect in ((1.0, 0.125 * h * h / 1.0), (0.0, 0.25 * h / c0)):
        wl = _lone([0.0, 0.0, 0.0], [0.0, 0.0, 0.0], h=h, c0=c0, g=(0.0, 0.0, 0.0), nu=nu,
                   half=1.0)
        _, hist = O.run(wl, O.state_of(wl), 0.0, 2)
        assert hist[1, 1] == pytest.approx(expect, rel=1e-15, abs=0.0)
        assert hist[2, 1] == pytest.approx(expect, rel=1e-15, abs=0.0)


def _perturbed_dam_break():
    wl = W.dam_break_2d(dx=0.04, precision=W.PREC_FP64)
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(5))
    fluid = s["role"] == W.FLUID
    s["rho"] = s["rho"] * (1.0 + 0.002 * rng.normal(size=s["rho"].shape))
    for k in ("u", "v"):
        s[k] = np.where(fluid, 0.3 * rng.normal(size=s[k].shape), 0.0)
    return wl, s, fluid


def _record_of(wl, st, rates, fluid):
    """KE, max|u|, momentum and max|a| over fluid particles by numpy."""
    dim = wl.dim
    u = np.stack([st[k] for k in ("u", "v", "w")[:dim]])[:, fluid]
    a = np.stack([rates[k] for k in ("ax", "ay", "az")[:dim]])[:, fluid]
    m = st["m"][fluid]
    ke = 0.5 * np.sum(m * np.sum(u * u, axis=0))
    mom = [float(np.sum(m * u[d])) for d in range(dim)] + [0.0] * (3 - dim)
    return ke, float(np.max(np.sqrt(np.sum(u * u, axis=0)))), mom, \
        float(np.max(np.sqrt(np.sum(a * a, axis=0))))


def test_record_of_the_initial_state():
    """No step: the record describes the given state and the rates of its evaluation (walls,
    artificial viscosity, XSPH, gravity all act)."""
    wl, s, fluid = _perturbed_dam_break()
    _, hist = O.run(wl, s, wl.dt, 0)
    r = O.rhs(wl, s)
    ke, umax, mom, amax = _record_of(wl, s, r, fluid)
    rec = hist[0]
    assert rec[0] == 0.0 and rec[1] == 0.0
    assert rec[2] == pytest.approx(ke, rel=1e-13)
    assert rec[3] == pytest.approx(umax, rel=1e-15)
    for d in range(3):
        assert rec[4 + d] == pytest.approx(mom[d], rel=1e-12, abs=1e-12 * np.sum(s["m"]))
    assert rec[7] == pytest.approx(amax, rel=1e-15)
    assert rec[8] == r["pairs"] and rec[9] == r["candidates"]
    assert rec[8] > 0 and rec[9] > rec[8]


def test_record_after_steps_matches_the_returned_state():
    """After three steps: KE, max|u| and momentum from the returned state; max|a| from an
    evaluation of that state, with the velocity-dependent terms off (no AV, viscosity or
    XSPH), so the rates of the step's last evaluation depend only on x and rho."""
    wl, s, fluid = _perturbed_dam_break()
    wl.alpha = 0.0
    wl.xsph_eps = 0.0
    st, hist = O.run(wl, s, wl.dt, 3)
    r = O.rhs(wl, st)
    ke, umax, mom, amax = _record_of(wl, st, r, fluid)
    rec = hist[3]
    assert rec[0] == pytest.approx(3 * wl.dt, rel=1e-15) and rec[1] == wl.dt
    assert rec[2] == pytest.approx(ke, rel=1e-13)
    assert rec[3] == pytest.approx(umax, rel=1e-15)
    for d in range(2):
        assert rec[4 + d] == pytest.approx(mom[d], rel=1e-12, abs=1e-12 * np.sum(s["m"]))
    assert rec[7] == pytest.approx(amax, rel=1e-14)
    assert rec[8] == r["pairs"] and rec[9] == r["candidates"]
