"""The EDAC form (SPH_DENSITY_EDAC: the pressure equation of the scheme list of Sec. 2.3,
with which Sec. 4.1 solves the Taylor-Green vortex) through the C ABI against the oracle.
Bars: FP64 mode <= 1e-10 normwise per rate and field after one step; FP32 pair loops
<= 1e-4 relative L2 (rates, and fields as the change from the start); max |u| within 1 %
of the oracle at every step."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import field_ok, normwise, rel_l2, sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "u", "v", "p")
RATES = ("arho", "ax", "ay")


def _wl(prec, n=30):
    return W.taylor_green_2d_edac(n=n, jitter=0.05, precision=prec)


def _perturbed(wl, seed=7):
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(seed))
    s["u"] = s["u"] + 0.05 * rng.normal(size=s["u"].shape)
    s["v"] = s["v"] + 0.05 * rng.normal(size=s["v"].shape)
    s["p"] = s["p"] + 0.02 * rng.normal(size=s["p"].shape)
    return s


def _load(sim, s):
    for k in ("u", "v", "p"):
        sim.set(k, s[k])


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_rates_match_oracle(prec):
    wl = _wl(prec)
    s = _perturbed(wl)
    ref = O.rhs(wl, s)
    with sim_of(wl) as sim:
        _load(sim, s)
        sim.eval_rhs(G.scheme_of(wl))
        r = sim.rates()
        d = sim.diagnostics()
        st = sim.state()
    assert d[8] == ref["pairs"] and d[9] == ref["candidates"]
    for k in RATES:
        if prec == G.PREC_FP64:
            assert normwise(r[k], ref[k]) <= 1e-10, k
        else:
            assert rel_l2(r[k], ref[k]) <= 1e-4, k
    assert np.array_equal(st["p"], s["p"])  # an evaluation does not advance the pressure
    assert np.all(st["rho"] == wl.rho0)


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_one_step(prec):
    wl = _wl(prec)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 1)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 1)
        g = sim.state()
        h = sim.history()
    for k in FIELDS:  # FP32: one-step increments
        assert field_ok(wl, k, g[k], st[k], s[k]), k
    assert np.all(g["rho"] == wl.rho0)
    assert h[0, 8] == hist[1, 8] and h[0, 9] == hist[1, 9]


def test_ten_steps_fp64():
    wl = _wl(G.PREC_FP64)
    s = O.state_of(wl)
    st, hist = O.run(wl, s, wl.dt, 10)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, 10)
        g = sim.state()
        h = sim.history()
    for k in FIELDS:
        assert normwise(g[k], st[k]) <= 1e-9, k
    assert np.max(np.abs(h[:, 2] - hist[1:, 2]) / hist[1:, 2]) < 1e-10


@pytest.mark.parametrize("prec,tol", [(G.PREC_FP64, 1e-9), (G.PREC_FP32, 1e-2)])
def test_decay_curve(prec, tol):
    """The Sec. 4.1 setup at 50^2 (h = 1.2 dx) over 100 steps: max |u| against the oracle's
    at every step."""
    wl = W.taylor_green_2d_edac(n=50, precision=prec)
    s = O.state_of(wl)
    steps = 100
    st, hist = O.run(wl, s, wl.dt, steps)
    with sim_of(wl) as sim:
        sim.step(G.scheme_of(wl), wl.dt, steps)
        h = sim.history()
    err = np.max(np.abs(h[:, 3] - hist[1:, 3]) / hist[1:, 3])
    assert err <= 0.01 and err <= tol


def test_resume_carries_the_pressure():
    wl = _wl(G.PREC_FP32, n=24)
    sch = G.scheme_of(wl)
    with sim_of(wl) as a, sim_of(wl) as b:
        a.step(sch, wl.dt, 10)
        b.step(sch, wl.dt, 5)
        blob = b.save_state()
        b.load_state(blob)
        b.step(sch, wl.dt, 5)
        ga, gb = a.state(), b.state()
    for k in FIELDS:
        assert np.array_equal(ga[k], gb[k]), k


def test_batch_equals_single_runs_bitwise():
    wls = [_wl(G.PREC_FP32, n=20), _wl(G.PREC_FP32, n=26)]
    schemes = [G.scheme_of(w) for w in wls]
    batch = G.BatchSimulation(wls)
    batch.set_groups(2)
    batch.step_batch(schemes, [w.dt for w in wls], 4)
    for k, wl in enumerate(wls):
        with sim_of(wl) as sim:
            sim.set_groups(2)
            sim.step(schemes[k], wl.dt, 4)
            st = sim.state()
        bs = batch.instance_state(k)
        for f in FIELDS:
            assert np.array_equal(bs[f], st[f]), (k, f)
    batch.close()


@pytest.mark.parametrize("prec", [G.PREC_FP64, G.PREC_FP32])
def test_persistent_form_equals_the_graph(prec):
    """One cooperative launch per step (the reorder gathers the pressure there too),
    bitwise equal to the per-phase graph; a batch likewise."""
    wl = _wl(prec, n=24)
    sch = G.scheme_of(wl)
    out = []
    for mode in (G.STEP_GRAPH, G.STEP_PERSISTENT):
        with sim_of(wl) as sim:
            sim.set_groups(4)
            sim.set_step_mode(mode)
            if mode == G.STEP_PERSISTENT:
                assert sim.kernels_per_step(sch) == 1
            sim.step(sch, wl.dt, 3)
            out.append(sim.state())
    for k in FIELDS:
        assert np.array_equal(out[0][k], out[1][k]), k
    wls = [_wl(prec, n=20), _wl(prec, n=26), _wl(prec, n=14)]
    schemes = [G.scheme_of(w) for w in wls]
    res = []
    for mode in (G.STEP_GRAPH, G.STEP_PERSISTENT):
        batch = G.BatchSimulation(wls)
        batch.set_groups(2)
        batch.set_step_mode(mode)
        batch.step_batch(schemes, [w.dt for w in wls], 3)
        res.append([batch.instance_state(k) for k in range(len(wls))])
        batch.close()
    for k in range(len(wls)):
        for f in FIELDS:
            assert np.array_equal(res[0][k][f], res[1][k][f]), (k, f)


def test_refusals():
    db = W.dam_break_2d(dx=0.05, precision=W.PREC_FP64)
    with sim_of(db) as sim:
        with pytest.raises(G.SphError):  # wall particles
            sim.step(G.scheme_of(db, density=G.EDAC), db.dt, 1)
    wl = _wl(G.PREC_FP64, n=16)
    with sim_of(wl) as sim:
        with pytest.raises(G.SphError):  # the midpoint integrator
            sim.step(G.scheme_of(wl, integrator=G.INTEGRATOR_PEC), wl.dt, 1)
        with pytest.raises(G.SphError):  # the adjoint
            sim.backward(G.scheme_of(wl), wl.dt, 2)
