"""The tile shape of one lane per destination (the shape the autotuner picks for large 3D
problems) at sizes the oracle finishes in seconds: rates, pair and candidate counts against
the oracle, and against the two- and four-lane shapes, on periodic, walled, clustered and
batched inputs, in FP32 pair loops."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import rel_l2, sim_of

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu

RATES_2D = ("arho", "ax", "ay", "xsx", "xsy")
RATES_3D = ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz")


def _cases():
    f = W.PREC_FP32
    return {
        "tg2d": W.taylor_green_2d(n=50, precision=f),
        "db2d": W.dam_break_2d(dx=0.02, precision=f),
        "tg3d": W.taylor_green_3d(n=16, precision=f),
        "db3d": W.dam_break_3d(dx=0.04, precision=f),
        "cube": W.falling_cube_3d(n=18, precision=f),
        "edac": W.taylor_green_2d_edac(n=40, jitter=0.05, precision=f),
    }


CASES = _cases()


def _loaded(wl):
    # EDAC holds the density at rho0 and carries the pressure instead
    return (["p"] if wl.density == 2 else ["rho"]) + ["u", "v", "w"][:wl.dim]


def _perturbed(wl, seed):
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(seed))
    fluid = s["role"] == W.FLUID
    if wl.density == 2:
        s["p"] = s["p"] + 0.02 * rng.normal(size=s["p"].shape)
    else:
        s["rho"] = s["rho"] * (1.0 + 0.003 * rng.normal(size=s["rho"].shape))
    for k in ("u", "v", "w")[:wl.dim]:
        s[k] = np.where(fluid, s[k] + 0.05 * rng.normal(size=s[k].shape), 0.0)
    return s


def _rates(wl, s, lanes):
    with sim_of(wl) as sim:
        sim.set_groups(lanes)
        for k in _loaded(wl):
            sim.set(k, s[k])
        sim.eval_rhs(G.scheme_of(wl))
        return sim.rates(), sim.diagnostics()


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_lane_rates_and_counts_match_the_oracle(name):
    """Rates within the FP32 bar (1e-4 relative L2); interacting pairs and candidates of
    the full stencil exact."""
    wl = CASES[name]
    s = _perturbed(wl, 13)
    ref = O.rhs(wl, s)
    r, d = _rates(wl, s, 1)
    assert d[8] == ref["pairs"] and d[9] == ref["candidates"]
    for k in (RATES_3D if wl.dim == 3 else RATES_2D):
        if np.max(np.abs(ref[k])) == 0.0:
            assert np.max(np.abs(r[k])) < 1e-12, k
        else:
            assert rel_l2(r[k], ref[k]) <= 1e-4, k


@pytest.mark.parametrize("name", sorted(CASES))
def test_one_lane_equals_the_per_lane_walk(name):
    """One and two lanes per destination list the same sources in the same order: equal
    counts, rates equal up to the summation order of the list (the two shapes add the
    same list in different lane orders)."""
    wl = CASES[name]
    s = _perturbed(wl, 17)
    r1, d1 = _rates(wl, s, 1)
    r2, d2 = _rates(wl, s, 2)
    assert d1[8] == d2[8] and d1[9] == d2[9]
    for k in (RATES_3D if wl.dim == 3 else RATES_2D):
        assert rel_l2(r1[k], r2[k]) <= 1e-5, k


def _clustered_3d(n_clusters=12, per=700, background=3000, seed=3):
    """Dense clusters (a few hundred particles within one support radius) in a sparse
    background: long stencil runs and warps that straddle many cell rows."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 0.02
    centres = rng.uniform(0.15, 0.85, size=(n_clusters, 3))
    pts = [c + rng.normal(scale=0.6 * h, size=(per, 3)) for c in centres]
    pts.append(rng.uniform(0.02, 0.98, size=(background, 3)))
    pts = np.clip(np.concatenate(pts), 0.001, 0.999)
    n = pts.shape[0]
    vel = rng.normal(scale=0.1, size=(n, 3))
    fl = W.ParticleSet(name="fluid", role=W.FLUID, x=pts[:, 0].copy(), y=pts[:, 1].copy(),
                       z=pts[:, 2].copy(), u=vel[:, 0].copy(), v=vel[:, 1].copy(),
                       w=vel[:, 2].copy(), rho=1000.0 * (1.0 + 0.002 * rng.normal(size=n)),
                       m=np.full(n, 1000.0 * (0.6 * h) ** 3))
    return W.Workload(name="clusters", dim=3, kernel=W.WENDLAND_C2, h=h, lo=[0.0, 0.0, 0.0],
                      hi=[1.0, 1.0, 1.0], periodic=[0, 0, 0], precision=W.PREC_FP32,
                      arrays=[fl], rho0=1000.0, c0=20.0, alpha=0.1, xsph_eps=0.5,
                      g=[0.0, 0.0, -9.81], dt=0.25 * h / 20.0, steps=1)


def test_dense_clusters_in_a_sparse_background():
    wl = _clustered_3d()
    s = O.state_of(wl)
    ref = O.rhs(wl, s)
    r, d = _rates(wl, s, 1)
    assert d[8] == ref["pairs"] and d[9] == ref["candidates"]
    for k in RATES_3D:
        assert rel_l2(r[k], ref[k]) <= 1e-4, k
    r2, d2 = _rates(wl, s, 4)
    assert d2[8] == d[8] and d2[9] == d[9]


def _tg_instances():
    return [W.taylor_green_2d(n=n, precision=W.PREC_FP32, seed=5 + n) for n in (21, 34, 27)]


def _db_instances():
    return [W.dam_break_2d(dx=dx, precision=W.PREC_FP32) for dx in (0.05, 0.04)]


@pytest.mark.parametrize("maker", [_tg_instances, _db_instances])
def test_batch_with_one_lane_equals_single_runs_bitwise(maker):
    """Warps of a batch straddle instances of different grids; each instance still equals
    its single run bit for bit."""
    wls = maker()
    steps = 6
    batch = G.BatchSimulation(wls)
    batch.set_groups(1)
    batch.step_batch([G.scheme_of(w) for w in wls], [w.dt for w in wls], steps)
    diag = batch.batch_diagnostics()
    for k, wl in enumerate(wls):
        with G.Simulation.from_workload(wl) as sim:
            sim.set_groups(1)
            sim.step(G.scheme_of(wl), wl.dt, steps)
            st = sim.state()
            d = sim.diagnostics()
        bs = batch.instance_state(k)
        for f in ("x", "y", "u", "v", "rho"):
            assert np.array_equal(bs[f], st[f]), (k, f)
        assert diag[k, 8] == d[8] and diag[k, 9] == d[9]
    batch.close()


def test_steps_with_one_lane_follow_the_oracle():
    """Ten steps of the 3D dam break (walls, artificial viscosity, XSPH) with one lane per
    destination: pair counts exact after the first step (later, FP32 positions may decide a pair
    at the support edge the other way: within 1e-4), fields within the FP32 bar on
    increments."""
    from gpu_util import field_ok
    wl = CASES["db3d"]
    s = O.state_of(wl)
    steps = 10
    st, hist = O.run(wl, s, wl.dt, steps)
    with sim_of(wl) as sim:
        sim.set_groups(1)
        sim.step(G.scheme_of(wl), wl.dt, steps)
        g = sim.state()
        h = sim.history()
    assert h[0, 8] == hist[1, 8] and h[0, 9] == hist[1, 9]
    assert np.all(np.abs(h[:, 8] - hist[1:, 8]) <= 1e-4 * hist[1:, 8])
    for k in ("x", "y", "z", "u", "v", "w", "rho"):
        assert field_ok(wl, k, g[k], st[k], s[k]), k


@pytest.mark.parametrize("name", ["db3d", "cube"])
def test_one_lane_runs_repeat_bitwise(name):
    """With one lane per destination the warps take their chunks from counters, in whatever
    order the hardware schedules them; the state and every record (sums of momentum and
    kinetic energy included, reduced per chunk in a fixed order) repeat bit for bit."""
    wl = CASES[name]
    sch = G.scheme_of(wl)
    out = []
    for _ in range(2):
        with sim_of(wl) as sim:
            sim.set_groups(1)
            sim.step(sch, wl.dt, 8)
            out.append((sim.state(), sim.history()))
    (sa, ha), (sb, hb) = out
    for k in ("x", "y", "z", "u", "v", "w", "rho"):
        assert np.array_equal(sa[k], sb[k]), k
    assert np.array_equal(ha, hb)


def _collapsing_ball(n=4000, seed=9):
    """A ball of fluid whose particles all move towards its centre (a sound speed so low that
    the pressure does not stop them): within a few steps the neighbour counts grow far beyond
    the list capacity sized at the start."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h, r0 = 0.01, 0.1
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1)[:, None]
    pts = 0.5 + d * (r0 * rng.uniform(size=n) ** (1.0 / 3.0))[:, None]
    dt = 0.25 * h / 20.0
    vel = -(pts - 0.5) * (0.5 / (8 * dt))  # the radius halves in about 8 steps
    fl = W.ParticleSet(name="fluid", role=W.FLUID, x=pts[:, 0].copy(), y=pts[:, 1].copy(),
                       z=pts[:, 2].copy(), u=vel[:, 0].copy(), v=vel[:, 1].copy(),
                       w=vel[:, 2].copy(), rho=np.full(n, 1000.0),
                       m=np.full(n, 1000.0 * (4.19 * r0 ** 3 / n)))
    return W.Workload(name="ball", dim=3, kernel=W.WENDLAND_C2, h=h, lo=[0.0, 0.0, 0.0],
                      hi=[1.0, 1.0, 1.0], periodic=[0, 0, 0], precision=W.PREC_FP32,
                      arrays=[fl], rho0=1000.0, c0=0.5, alpha=0.1, xsph_eps=0.5,
                      g=[0.0, 0.0, 0.0], dt=dt, steps=1)


def test_list_overflow_then_the_state_set_again():
    """A list overflow stops the run with an error; set again, the context continues as a
    fresh one: the same pair and candidate counts, fields equal up to the summation order
    (the used context's particles keep their own order within a cell). A chunk counter left
    behind by the blocks that skipped their work after the overflow would drop chunks of
    destinations and change the counts."""
    wl = _collapsing_ball()
    sch = G.scheme_of(wl)
    s0 = O.state_of(wl)
    keys = ("x", "y", "z", "u", "v", "w", "rho")
    with sim_of(wl) as a, sim_of(wl) as b:
        for sim in (a, b):
            sim.set_groups(1)
        with pytest.raises(G.SphError, match="CAPACITY"):
            a.step(sch, wl.dt, 14)
        for k in keys:
            a.set(k, s0[k])
        a.step(sch, wl.dt, 2)
        b.step(sch, wl.dt, 2)
        sa, sb = a.state(), b.state()
        da, db = a.diagnostics(), b.diagnostics()
        assert da[8] == db[8] and da[9] == db[9]
        for k in keys:  # the change over the two steps
            assert rel_l2(sa[k] - s0[k], sb[k] - s0[k]) <= 1e-5, k
