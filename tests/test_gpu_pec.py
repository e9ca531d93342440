"""Midpoint predict-evaluate-correct integrator (scheme option SPH_INTEGRATOR_PEC, the
two-evaluation form of the predictor-corrector of Sec. 2.1 after Monaghan 2005) through
the C ABI against the oracle: one step on the four workload structures (FP64 mode
<= 1e-10 normwise per field, FP32 pair loops <= 1e-4 relative L2), ten steps, the
CFL-type step size, summation density and the solid-wall pressure, a switch of
integrator mid-run, save and resume, the persistent step form falling back to the
graph, a batch bitwise equal to single runs, and the adjoint refusing the option."""
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
PEC = G.INTEGRATOR_PEC

CONFIGS = {"tg2d": W.taylor_green_2d(n=50), "db2d": W.dam_break_2d(dx=0.02),
           "tg3d": W.taylor_green_3d(n=16), "db3d": W.dam_break_3d(dx=0.04)}


def _pec(wl, prec=None):
    return oracle_wl(wl, prec).with_integrator(PEC)


def _close(prec, a, b, fp64_tol=1e-10):
    return normwise(a, b) <= fp64_tol if prec == G.PREC_FP64 else rel_l2(a, b) <= 1e-4


def _fields(wl):
    return FIELDS_3D if wl.dim == 3 else FIELDS_2D


@pytest.mark.parametrize("name", sorted(CONFIGS))
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_one_step(name, prec):
    wl = _pec(CONFIGS[name], prec)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 1)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 1)
        g = sim.state()
        h = sim.history()
        d = sim.diagnostics()
    for k in _fields(wl):  # FP32: one-step increments
        assert field_ok(wl, k, g[k], st[k], s[k]), k
    assert h.shape[0] == 1
    assert abs(h[0, 0] - hist[1, 0]) < 1e-15 and h[0, 1] == hist[1, 1]
    assert h[0, 8] == hist[1, 8] and h[0, 9] == hist[1, 9]  # pairs at the end of the step
    assert d[10] == 1.0  # step count


@pytest.mark.parametrize("name", ["tg2d", "db2d"])
def test_ten_steps_fp64(name):
    wl = _pec(CONFIGS[name], G.PREC_FP64)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 10)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 10)
        g = sim.state()
        h = sim.history()
    for k in FIELDS_2D:
        assert normwise(g[k], st[k]) <= 1e-9, k
    assert np.max(np.abs(h[:, 0] - hist[1:, 0])) < 1e-14
    assert np.array_equal(h[:, 8], hist[1:, 8])
    # kinetic energy of every record (end-of-step state)
    assert np.max(np.abs(h[:, 2] - hist[1:, 2]) / np.abs(hist[1:, 2]).max()) < 1e-10


def test_adaptive_dt_fp64():
    wl = _pec(W.dam_break_2d(dx=0.04), G.PREC_FP64)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, 0.0, 10)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), 0.0, 10)
        h = sim.history()
        g = sim.state()
    assert np.max(np.abs(h[:, 1] - hist[1:, 1]) / hist[1:, 1]) < 1e-12
    for k in FIELDS_2D:
        assert normwise(g[k], st[k]) <= 1e-10, k


@pytest.mark.parametrize("variant", ["summation", "adami"])
@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_summation_density_and_wall_pressure(variant, prec):
    if variant == "summation":
        wl = copy.deepcopy(_pec(W.taylor_green_2d(n=40), prec))
        wl.density = G.SUMMATION
    else:
        wl = _pec(W.dam_break_2d(dx=0.02).with_wall_bc(1), prec)
    s = O.state_of(wl)
    st, _ = O.run(wl, s, wl.dt, 3)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 3)
        g = sim.state()
    for k in FIELDS_2D:  # FP32: three-step increments
        assert field_ok(wl, k, g[k], st[k], s[k], fp64_tol=1e-9), k


def test_switch_integrator_mid_run():
    """Three kick-drift-kick steps, then three midpoint steps: a change of scheme
    re-evaluates the rates at the current state, as the oracle's run does at its start."""
    wl = oracle_wl(W.dam_break_2d(dx=0.02), G.PREC_FP64)
    s = O.state_of(wl)
    s1, _ = O.run(wl, s, wl.dt, 3)
    s2, _ = O.run(wl.with_integrator(PEC), s1, wl.dt, 3)
    s3, _ = O.run(wl, s2, wl.dt, 2)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 3)
        sim.step(G.scheme_of(wl, integrator=PEC), wl.dt, 3)
        g2 = sim.state()
        sim.step(G.scheme_of(wl), wl.dt, 2)
        g3 = sim.state()
    for k in FIELDS_2D:
        assert normwise(g2[k], s2[k]) <= 1e-10, k
        assert normwise(g3[k], s3[k]) <= 1e-10, k


def test_resumable_and_persistent_form_runs_the_graph():
    wl = _pec(W.dam_break_2d(dx=0.02), G.PREC_FP32)
    sch = G.scheme_of(wl)
    with sim_of(wl) as a, sim_of(wl) as b:
        a.step(sch, wl.dt, 6)
        blob = a.save_state()
        a.step(sch, wl.dt, 5)
        b.set_step_mode(G.STEP_PERSISTENT)
        b.step(sch, wl.dt, 2)
        b.load_state(blob)
        b.step(sch, wl.dt, 5)
        for k in FIELDS_2D:
            assert np.array_equal(a.get(k), b.get(k)), k
        assert np.array_equal(a.diagnostics(), b.diagnostics())


def test_launch_count_and_refusals():
    wl = _pec(W.dam_break_2d(dx=0.04), G.PREC_FP32)
    sch = G.scheme_of(wl)
    with sim_of(wl) as sim:
        kdk = sim.kernels_per_step(G.scheme_of(wl, integrator=G.INTEGRATOR_KDK))
        sim.set_step_mode(G.STEP_GRAPH)
        kdk_graph = sim.kernels_per_step(G.scheme_of(wl, integrator=G.INTEGRATOR_KDK))
        assert sim.kernels_per_step(sch) == 2 * kdk_graph + 3 and kdk >= 1
        with pytest.raises(G.SphError):
            sim.backward(sch, wl.dt, 2)
        bad = G.scheme_of(wl)
        bad.integrator = 7
        with pytest.raises(G.SphError):
            sim.step(bad, wl.dt, 1)
    batch = G.BatchSimulation([W.dam_break_2d(dx=0.05), W.dam_break_2d(dx=0.06)])
    try:
        mixed = [sch, G.scheme_of(wl, integrator=G.INTEGRATOR_KDK)]
        with pytest.raises(G.SphError):  # the instances share the integrator
            batch.step_batch(mixed, [wl.dt, wl.dt], 1)
    finally:
        batch.close()


@pytest.mark.parametrize("precision", [W.PREC_FP64, W.PREC_FP32])
def test_batch_equals_single_runs(precision):
    """Instances of uneven size (one with the solid-wall pressure), each with its own fixed
    dt: every instance bitwise equal to its single run."""
    wls = [W.dam_break_2d(dx=dx, precision=precision).with_integrator(PEC)
           for dx in (0.05, 0.04, 0.06)]
    wls[1] = wls[1].with_wall_bc(1)
    dts = [w.dt for w in wls]
    steps = 8
    batch = G.BatchSimulation(wls)
    batch.set_groups(2)
    batch.step_batch([G.scheme_of(w) for w in wls], dts, steps)
    diag = batch.batch_diagnostics()
    try:
        for k, wl in enumerate(wls):
            with G.Simulation.from_workload(wl) as sim:
                sim.set_groups(2)
                sim.step(G.scheme_of(wl), dts[k], steps)
                st = sim.state()
                d = sim.diagnostics()
            bs = batch.instance_state(k)
            for f in FIELDS_2D:
                assert np.array_equal(bs[f], st[f]), (k, f)
            assert diag[k, 0] == d[0] and diag[k, 1] == d[1] and diag[k, 10] == steps, k
    finally:
        batch.close()
