"""Cubic (M4) B-spline kernel and the falling-cube problem of Sec. 4.4 through the C ABI
against the oracle: cells and neighbour sets bit-exact; rates after one evaluation and
fields after steps on perturbed states (FP64 mode <= 1e-10 normwise per field, FP32 pair
loops <= 1e-4 relative L2) with continuity and summation density, walls, artificial
viscosity and XSPH; free fall of the cube at rest; the persistent step form; and the
adjoint against the oracle's dual numbers (FP64 <= 1e-8, FP32 <= 1e-3 relative)."""
import copy

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import csr_equal, field_ok, normwise, oracle_wl, rel_l2, sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu

FIELDS_2D = ("x", "y", "u", "v", "rho")
FIELDS_3D = ("x", "y", "z", "u", "v", "w", "rho")
RATES_2D = ("arho", "ax", "ay", "xsx", "xsy")
RATES_3D = ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz")


def _cubic(wl, hdx=1.2):
    w = copy.deepcopy(wl)
    if w.kernel != G.CUBIC_SPLINE:
        w.h = w.h * hdx / (1.3 if w.kernel == G.WENDLAND_C2 else 1.0)
        w.kernel = G.CUBIC_SPLINE
        w.name = w.name + "_cubic"
    return w


CONFIGS = {"tg2d": lambda: _cubic(W.taylor_green_2d(n=50)),
           "db2d": lambda: _cubic(W.dam_break_2d(dx=0.02)),
           "fc3d": lambda: W.falling_cube_3d(n=16)}


def _perturbed(wl, seed=3):
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = s["role"] == W.FLUID
    s["rho"] = np.where(fluid, s["rho"] * (1.0 + 0.003 * rng.normal(size=s["rho"].shape)),
                        s["rho"])
    for k in ("u", "v", "w")[:wl.dim]:
        s[k] = np.where(fluid, s[k] + 0.1 * rng.normal(size=s[k].shape), 0.0)
    return s


def _close(prec, a, b, fp64_tol=1e-10):
    return normwise(a, b) <= fp64_tol if prec == G.PREC_FP64 else rel_l2(a, b) <= 1e-4


def _load(sim, s, dim):
    for k in ["rho"] + ["u", "v", "w"][:dim]:
        sim.set(k, s[k])


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_cells_and_neighbours_bit_exact(name, prec):
    wl = oracle_wl(CONFIGS[name](), prec)
    s = O.state_of(wl)
    with sim_of(wl) as sim:
        nc, cs, ncells = sim.grid()
        onc, ocs, oncells = O.grid(wl)
        assert nc == onc and cs == ocs and ncells == oncells
        cell_of, off, order = sim.cells()
        ocell, ooff, _ = O.cells(wl, s["x"], s["y"], s["z"])
        assert np.array_equal(cell_of, ocell) and np.array_equal(off, ooff)
        assert np.all(np.diff(cell_of[order].astype(np.int64)) >= 0)
        noff, nidx = sim.neighbors()
        ooff2, oidx, _ = O.neighbors(wl, s["x"], s["y"], s["z"])
        assert csr_equal(noff, nidx, ooff2, oidx)


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_rhs_and_step_on_a_perturbed_state(name, prec):
    wl = oracle_wl(CONFIGS[name](), prec)
    s = _perturbed(wl)
    ref = O.rhs(wl, s)
    st, _ = O.run(wl, s, wl.dt, 3)
    with sim_of(wl) as sim:
        _load(sim, s, wl.dim)
        sim.eval_rhs(G.scheme_of(wl))
        r = sim.rates()
        for k in RATES_3D if wl.dim == 3 else RATES_2D:
            assert _close(prec, r[k], ref[k]), k
        sim.step(G.scheme_of(wl), wl.dt, 3)
        g = sim.state()
    for k in FIELDS_3D if wl.dim == 3 else FIELDS_2D:  # FP32: three-step increments
        assert field_ok(wl, k, g[k], st[k], s[k]), k


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_summation_density(prec):
    wl = copy.deepcopy(oracle_wl(CONFIGS["tg2d"](), prec))
    wl.density = G.SUMMATION
    s = _perturbed(wl)
    ref = O.rhs(wl, s)
    with sim_of(wl) as sim:
        _load(sim, s, wl.dim)
        sim.eval_rhs(G.scheme_of(wl))
        assert _close(prec, sim.get("rho"), ref["rho"])
        r = sim.rates()
    for k in RATES_2D[1:]:
        assert _close(prec, r[k], ref[k]), k


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_falling_cube_at_rest_falls_freely(prec):
    """At rest with rho = rho0 every pressure vanishes and every velocity difference is
    zero: the cube falls rigidly, z = z0 + g t^2 / 2 (up to the rounding of the steps)."""
    wl = oracle_wl(W.falling_cube_3d(n=16), prec)
    s = O.state_of(wl)
    steps = 20
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, steps)
        g = sim.state()
        h = sim.history()
    t = steps * wl.dt
    assert np.max(np.abs(g["z"] - (s["z"] + 0.5 * wl.g[2] * t * t))) < 1e-12
    assert np.max(np.abs(g["w"] - wl.g[2] * t)) < 1e-12
    assert np.array_equal(g["x"], s["x"]) and np.all(g["rho"] == wl.rho0)
    assert np.all(h[:, 8] == h[0, 8])  # the neighbour count of a rigid body


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_persistent_form(prec):
    wl = oracle_wl(CONFIGS["db2d"](), prec)
    s = O.state_of(wl)
    st, _ = O.run(wl, s, wl.dt, 5)
    with sim_of(wl) as sim:
        sim.set_step_mode(G.STEP_PERSISTENT)
        sim.step(G.scheme_of(wl), wl.dt, 5)
        g = sim.state()
    for k in FIELDS_2D:  # FP32: five-step increments
        assert field_ok(wl, k, g[k], st[k], s[k]), k


@pytest.mark.parametrize("prec,tol", [(G.PREC_FP64, 1e-8), (G.PREC_FP32, 1e-3)])
def test_adjoint_against_dual_numbers(prec, tol):
    wl = _cubic(W.taylor_green_2d(n=20, precision=prec))
    wl.nu = 0.05
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(9))
    d = [rng.normal(size=s["x"].shape) for _ in range(2)]
    _, dke_u = O.grad(wl, s, wl.dt, 6, du=d[0], dv=d[1])
    _, dke_nu = O.grad(wl, s, wl.dt, 6, dnu=1.0)
    with sim_of(wl) as sim:
        gu, gnu, _ = sim.backward(G.scheme_of(wl), wl.dt, 6)
    got = sum(np.dot(gu[k], d[k]) for k in range(2))
    assert abs(got - dke_u) <= tol * abs(dke_u), (got, dke_u)
    assert abs(gnu - dke_nu) <= tol * abs(dke_nu), (gnu, dke_nu)
