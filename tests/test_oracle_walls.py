"""Pins of the oracle's solid-wall pressure (the wall boundary condition of Adami, Hu and
Adams, 2012, listed among the schemes of Sec. 2.3) against what the formula fixes: the
kernel-weighted mean reproduces a uniform fluid pressure exactly, the hydrostatic term
extrapolates a linear hydrostatic field to the wall point exactly, a wall out of reach of
the fluid stays at rest density, and the wall density is the one the Tait EOS maps to
the wall pressure."""
import copy

import numpy as np

import oracle as O
import workloads as W


def tank(g=(0.0, -9.81, 0.0), c0=None):
    """Small 2D dam-break tank with the wall condition switched on."""
    wl = W.dam_break_2d(dx=0.05, precision=W.PREC_FP64).with_wall_bc(1)
    wl = copy.deepcopy(wl)
    wl.g = list(g)
    wl.alpha = 0.0
    wl.xsph_eps = 0.0
    if c0 is not None:
        wl.c0 = c0
    s = O.state_of(wl)
    return wl, s


def eos_p(wl, rho):
    B = wl.rho0 * wl.c0 ** 2 / wl.gamma
    return B * ((rho / wl.rho0) ** wl.gamma - 1.0)


def eos_rho(wl, p):
    B = wl.rho0 * wl.c0 ** 2 / wl.gamma
    return wl.rho0 * (1.0 + p / B) ** (1.0 / wl.gamma)


def wall_reach(wl, s):
    """Per wall particle: whether any fluid particle lies inside its support."""
    off, idx, _ = O.neighbors(wl, s["x"], s["y"])
    fluid = s["role"] == W.FLUID
    reach = np.zeros(s["x"].shape[0], bool)
    for i in np.nonzero(~fluid)[0]:
        reach[i] = fluid[idx[off[i]:off[i + 1]]].any()
    return reach


def test_uniform_pressure_is_reproduced():
    wl, s = tank(g=(0.0, 0.0, 0.0))
    fluid = s["role"] == W.FLUID
    rho1 = 1.01 * wl.rho0
    s["rho"][fluid] = rho1
    out = O.rhs(wl, s)
    reach = wall_reach(wl, s)
    walls = ~fluid
    assert reach[walls].sum() > 100 and (~reach[walls]).sum() > 100
    p1 = eos_p(wl, rho1)
    np.testing.assert_allclose(out["p"][walls & reach], p1, rtol=1e-12)
    np.testing.assert_allclose(out["rho"][walls & reach], rho1, rtol=1e-12)
    # out of reach of the fluid: no pressure, rest density
    assert np.all(out["p"][walls & ~reach] == 0.0)
    assert np.all(out["rho"][walls & ~reach] == wl.rho0)
    # the fluid keeps its own EOS pressure
    np.testing.assert_allclose(out["p"][fluid], p1, rtol=1e-12)


def test_linear_hydrostatic_field_is_extrapolated_to_the_wall():
    """p_f = rho0 g (H - y_f): the mean of a linear field is the field at the weighted mean
    height, and the body-force term carries it on to the wall height, so p_w equals
    rho0 g (H - y_w) up to the density variation (rho_f / rho0 - 1 < 1e-7 with this stiff
    EOS)."""
    gy = 9.81
    wl, s = tank(g=(0.0, -gy, 0.0), c0=1.0e4)
    fluid = s["role"] == W.FLUID
    H = 2.0
    p_f = wl.rho0 * gy * (H - s["y"][fluid])
    s["rho"][fluid] = eos_rho(wl, p_f)
    out = O.rhs(wl, s)
    walls = (~fluid) & wall_reach(wl, s)
    expect = wl.rho0 * gy * (H - s["y"][walls])
    scale = wl.rho0 * gy * H
    err = np.abs(out["p"][walls] - expect) / scale
    # (a flipped or dropped body-force term is off by rho0 g (y_mean - y_w) or twice that,
    # a few % of rho0 g H at these spacings)
    assert err.max() < 1e-6, err.max()
    # wall density: the EOS image of the wall pressure
    np.testing.assert_allclose(eos_p(wl, out["rho"][walls]), out["p"][walls],
                               rtol=1e-9, atol=1e-9 * scale)


def test_condition_off_keeps_continuity_walls():
    wl, s = tank()
    wl0 = copy.deepcopy(wl)
    wl0.wall_bc = 0
    fluid = s["role"] == W.FLUID
    s["rho"][fluid] = 1.01 * wl.rho0
    out0 = O.rhs(wl0, s)
    # continuity mode at rest: wall densities unchanged, pressure from the EOS of rho0
    assert np.all(out0["rho"][~fluid] == wl.rho0)
    assert np.all(out0["p"][~fluid] == 0.0)
    # the fluid's accelerations change only through the wall pressures
    out1 = O.rhs(wl, s)
    near = np.abs(out1["ay"] - out0["ay"]) > 0
    assert near[fluid].any() and not near[~fluid].any()
