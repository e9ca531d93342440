"""Solid-wall pressure (scheme option SPH_WALL_ADAMI, the wall condition of Adami, Hu and
Adams listed among the schemes of Sec. 2.3) through the C ABI against the oracle: one
evaluation and one step (FP64 mode <= 1e-10 normwise per field, FP32 pair loops
<= 1e-4 relative L2), the hydrostatic closed form at the walls, a batch of instances
bitwise equal to single runs, the persistent step form (its own wall phase) equal to
the graph bitwise, and the adjoint refusing the option."""
import copy

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import field_ok, normwise, oracle_wl, rel_l2, sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu

FIELDS_2D = ("x", "y", "u", "v", "rho")
FIELDS_3D = ("x", "y", "z", "u", "v", "w", "rho")
RATES_2D = ("arho", "ax", "ay", "xsx", "xsy")
RATES_3D = ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz")
CONFIGS = {"db2d": W.dam_break_2d(dx=0.02).with_wall_bc(1),
           "db3d": W.dam_break_3d(dx=0.04).with_wall_bc(1)}


def _perturbed(wl, seed=5):
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = s["role"] == W.FLUID
    s["rho"] = np.where(fluid, s["rho"] * (1.0 + 0.003 * rng.normal(size=s["rho"].shape)),
                        s["rho"])
    for k in ("u", "v", "w")[:wl.dim]:
        s[k] = np.where(fluid, s[k] + 0.05 * rng.normal(size=s[k].shape), 0.0)
    return s


def _close(prec, a, b):
    return normwise(a, b) <= 1e-10 if prec == G.PREC_FP64 else rel_l2(a, b) <= 1e-4


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_rhs_with_wall_pressure_matches_oracle(name, prec):
    wl = oracle_wl(CONFIGS[name], prec)
    s = _perturbed(wl)
    ref = O.rhs(wl, s)
    ref0 = O.rhs(copy.copy(wl).with_wall_bc(0), s)
    walls = s["role"] != W.FLUID
    assert np.max(np.abs(ref["rho"][walls] - ref0["rho"][walls])) > 0.0  # the option acts
    with sim_of(wl) as sim:
        for k in ["rho"] + ["u", "v", "w"][:wl.dim]:
            sim.set(k, s[k])
        sim.eval_rhs(G.scheme_of(wl))
        r = sim.rates()
        rho = sim.get("rho")
    assert _close(prec, rho, ref["rho"])
    assert _close(prec, rho[walls], ref["rho"][walls])
    rates = RATES_3D if wl.dim == 3 else RATES_2D
    for k in rates:
        assert _close(prec, r[k], ref[k]), k


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_one_step_with_wall_pressure(name, prec):
    wl = oracle_wl(CONFIGS[name], prec)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 1)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 1)
        g = sim.state()
        h = sim.history()
    for k in FIELDS_3D if wl.dim == 3 else FIELDS_2D:  # FP32: one-step increments
        assert field_ok(wl, k, g[k], st[k], s[k]), k
    assert h[0, 8] == hist[1, 8] and h[0, 9] == hist[1, 9]


def test_twenty_steps_fp64():
    wl = oracle_wl(CONFIGS["db2d"], G.PREC_FP64)
    s = O.state_of(wl)
    st, _ = O.run(wl, s, wl.dt, 20)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 20)
        g = sim.state()
    for k in ("x", "y", "u", "v", "rho"):
        assert normwise(g[k], st[k]) <= 1e-9, k


def test_hydrostatic_wall_pressure_closed_form():
    """Fluid at p_f = rho0 g (H - y_f) (stiff EOS, so rho_f ~ rho0): the walls within reach
    take rho0 g (H - y_w), read back through their density and the EOS."""
    wl = copy.deepcopy(oracle_wl(W.dam_break_2d(dx=0.05).with_wall_bc(1), G.PREC_FP64))
    wl.alpha = wl.xsph_eps = 0.0
    wl.c0 = 1.0e4
    gy, H = -wl.g[1], 2.0
    B = wl.rho0 * wl.c0 ** 2 / wl.gamma
    s = O.state_of(wl)
    fluid = s["role"] == W.FLUID
    p_f = wl.rho0 * gy * (H - s["y"][fluid])
    s["rho"][fluid] = wl.rho0 * (1.0 + p_f / B) ** (1.0 / wl.gamma)
    off, idx, _ = O.neighbors(wl, s["x"], s["y"])
    reach = np.array([fluid[idx[off[i]:off[i + 1]]].any() for i in range(len(fluid))])
    with sim_of(wl) as sim:
        sim.set("rho", s["rho"])
        sim.eval_rhs(G.scheme_of(wl))
        rho = sim.get("rho")
    w = (~fluid) & reach
    p_w = B * ((rho[w] / wl.rho0) ** wl.gamma - 1.0)
    err = np.abs(p_w - wl.rho0 * gy * (H - s["y"][w])) / (wl.rho0 * gy * H)
    assert w.sum() > 100 and err.max() < 1e-6
    assert np.all(rho[(~fluid) & ~reach] == wl.rho0)


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_batch_with_wall_pressure_equals_single_runs(precision):
    wls = [W.dam_break_2d(dx=dx, precision=precision).with_wall_bc(1) for dx in (0.05, 0.04)]
    wls.append(W.dam_break_2d(dx=0.06, precision=precision))  # one instance without it
    steps = 10
    batch = G.BatchSimulation(wls)
    batch.set_groups(2)
    batch.step_batch([G.scheme_of(w) for w in wls], [w.dt for w in wls], steps)
    for k, wl in enumerate(wls):
        with G.Simulation.from_workload(wl) as sim:
            sim.set_groups(2)
            sim.step(G.scheme_of(wl), wl.dt, steps)
            st = sim.state()
        bs = batch.instance_state(k)
        for f in ("x", "y", "u", "v", "rho"):
            assert np.array_equal(bs[f], st[f]), (k, f)
    batch.close()


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_persistent_form_with_wall_pressure(name, prec):
    """The persistent step runs the wall phase between its pair passes (one launch per
    step) and follows the graph bitwise; one step meets the oracle bar."""
    wl = oracle_wl(CONFIGS[name], prec)
    sch = G.scheme_of(wl)
    fields = FIELDS_3D if wl.dim == 3 else FIELDS_2D
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 1)
    with sim_of(wl) as a, sim_of(wl) as b:
        for sim in (a, b):
            sim.set_groups(4)
        a.set_step_mode(G.STEP_PERSISTENT)
        assert a.kernels_per_step(sch) == 1
        a.step(sch, wl.dt, 1)
        g = a.state()
        for f in fields:
            assert field_ok(wl, f, g[f], st[f], s[f]), f
        assert a.history()[0, 8] == hist[1, 8]
        a.step(sch, wl.dt, 4)
        b.step(sch, wl.dt, 5)
        sa, sb = a.state(), b.state()
        for f in fields:
            assert np.array_equal(sa[f], sb[f]), f


def test_adjoint_refuses_the_wall_pressure():
    wl = oracle_wl(CONFIGS["db2d"], G.PREC_FP32)
    sch = G.scheme_of(wl)
    with sim_of(wl) as b:
        sch0 = G.scheme_of(wl, wall_bc=G.WALL_DENSITY)
        assert b.kernels_per_step(sch) == b.kernels_per_step(sch0) + 1
        with pytest.raises(G.SphError):
            b.backward(sch, wl.dt, 3)


@pytest.mark.parametrize("wall_bc", [0, 1])
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_summation_density_with_walls(wall_bc, prec):
    """Summation density (Eq. 2) on the dam break: walls sum every neighbour (continuity
    walls) or take the solid-wall pressure after the summation."""
    wl = copy.deepcopy(oracle_wl(W.dam_break_2d(dx=0.02), prec)).with_wall_bc(wall_bc)
    wl.density = G.SUMMATION
    s = O.state_of(wl)
    ref = O.rhs(wl, s)
    st, _ = O.run(wl, s, wl.dt, 3)
    with sim_of(wl) as sim:
        sim.eval_rhs(G.scheme_of(wl))
        assert _close(prec, sim.get("rho"), ref["rho"])
        for k in RATES_2D[1:]:
            assert _close(prec, sim.get(k), ref[k]), k
        sim.step(G.scheme_of(wl), wl.dt, 3)
        for k in FIELDS_2D:  # FP32: three-step increments
            assert field_ok(wl, k, sim.get(k), st[k], s[k]), k


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_wall_with_one_fluid_neighbour_at_the_support_edge(prec):
    """A wall whose only fluid neighbour lies just inside the support: in FP64 mode the
    Wendland weight is (1 - q/2)^4 (2q + 1) sigma / h^2 with 1 - q/2 ~ 1e-12, a sum of
    ~1e-45, below FP32's range. The wall pressure is the ratio of sums that all carry that
    weight, p_w = p_f + rho_f g . (x_w - x_f): finite, and equal to the oracle's."""
    h = 0.02
    xw, yw = 0.5, 0.5
    # FP32 mode rounds the positions to float (~1e-6 of r): its gap must exceed that
    r = 2.0 * h * (1.0 - (1e-12 if prec == G.PREC_FP64 else 1e-4))
    ang = 0.3
    xf, yf = xw + r * np.cos(ang), yw + r * np.sin(ang)

    def one(name, role, x, y, rho):
        return W.ParticleSet(name, role, np.array([x]), np.array([y]), np.zeros(1), np.zeros(1),
                             np.zeros(1), np.zeros(1), np.array([rho]), np.array([0.4]))

    wl = W.Workload(name="edge_wall", dim=2, kernel=W.WENDLAND_C2, h=h, lo=[0.0, 0.0, 0.0],
                    hi=[1.0, 1.0, 1.0], periodic=[0, 0, 0], precision=prec,
                    arrays=[one("fluid", W.FLUID, xf, yf, 1001.0),
                            one("wall", W.WALL, xw, yw, 1000.0)],
                    rho0=1000.0, c0=20.0, g=[0.0, -9.81, 0.0], dt=0.25 * h / 20.0,
                    wall_bc=1)
    s = O.state_of(wl)
    ref = O.rhs(wl, s)
    assert ref["pairs"] == 2
    with sim_of(wl) as sim:
        sim.eval_rhs(G.scheme_of(wl))
        rho = sim.get("rho")
        d = sim.diagnostics()
    assert d[8] == 2
    assert np.all(np.isfinite(rho))
    # the wall's density is the EOS image of p_w = p_f + rho_f g . (x_w - x_f)
    if prec == G.PREC_FP64:
        assert abs(rho[1] - ref["rho"][1]) <= 1e-12 * ref["rho"][1]
    else:
        assert abs(rho[1] - ref["rho"][1]) <= 1e-6 * ref["rho"][1]
