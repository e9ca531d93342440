"""The octree search with a per-particle smoothing length (include/sph_vh.h) against the
oracle: neighbour sets bit-exact in both precision modes (every pair examined by the
oracle), the density of the same pass (FP64 <= 1e-12 normwise, FP32 <= 1e-5 relative L2:
FP32 pair terms carry a few 2^-23 of relative error and the sums are compensated), the
tree's invariants, the degenerate inputs, and the full-size set on sampled rows."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import normwise, rel_l2

import paper_1909_04504_gb300 as G

pytestmark = pytest.mark.gpu


def _rows(off, idx):
    return [np.sort(idx[off[i]:off[i + 1]]) for i in range(len(off) - 1)]


def _search(s, leaf=16, capacity=None, prec=None):
    prec = s.precision if prec is None else prec
    v = G.VariableHSearch(s.dim, s.kernel, prec, capacity or max(s.n, 1), leaf_size=leaf)
    v.set(s.x, s.y, s.z if s.dim == 3 else None, s.h, s.m)
    v.search()
    return v


def _blob(n, dim, kernel, prec, seed):
    s = W.gaussian_blob(n, dim=dim, kernel=kernel, precision=prec, seed=seed)
    return s


def _same_sets(v, s, prec):
    off, idx = v.neighbors()
    ro, ri = O.vh_neighbors(s.dim, s.kernel, prec, s.x, s.y, s.z, s.h)
    assert np.array_equal(off, ro)
    got, want = _rows(off, idx), _rows(ro, ri)
    for i in range(s.n):
        assert np.array_equal(got[i], want[i]), i
    return off


@pytest.mark.parametrize("dim,kernel", [(2, W.WENDLAND_C2), (3, W.WENDLAND_C2), (2, W.QUINTIC),
                                        (3, W.CUBIC_SPLINE), (3, W.QUINTIC)])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_neighbour_sets_and_density_match_oracle(dim, kernel, prec):
    s = _blob(5003 if dim == 3 else 7001, dim, kernel, prec, seed=40 + dim + kernel)
    with _search(s, leaf=16) as v:
        off = _same_sets(v, s, prec)
        rho = v.density()
        st = v.stats()
    want = O.vh_density(s.dim, s.kernel, prec, s.x, s.y, s.z, s.h, s.m)
    if prec == W.PREC_FP64:
        assert normwise(rho, want) <= 1e-12
    else:
        assert rel_l2(rho, want) <= 1e-5
    assert st["pairs"] == off[-1] and st["candidates"] >= st["pairs"]
    assert st["max_count"] == int(np.max(np.diff(off)))


@pytest.mark.parametrize("leaf", [1, 4, 64, 4096])
def test_leaf_sizes_give_the_same_sets(leaf):
    s = _blob(3001, 3, W.WENDLAND_C2, W.PREC_FP32, seed=9)
    with _search(s, leaf=leaf) as v:
        _same_sets(v, s, W.PREC_FP32)
        st = v.stats()
    if leaf == 4096:
        assert st["nodes"] == 1 and st["leaves"] == 1  # the root holds them all
    else:
        assert st["leaves"] >= s.n // leaf // 8


@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_tree_invariants(prec):
    s = _blob(20011, 3, W.QUINTIC, prec, seed=12)
    leaf = 12
    with _search(s, leaf=leaf) as v:
        t = v.tree()
        st = v.stats()
    perm = t["perm"]
    assert np.array_equal(np.sort(perm), np.arange(s.n))
    pts = np.stack([s.x, s.y, s.z], axis=1)[perm]
    h = s.h[perm]
    if prec == W.PREC_FP32:
        pts = pts.astype(np.float32).astype(np.float64)
        h = h.astype(np.float32).astype(np.float64)
    start, end, child, nch = t["start"], t["end"], t["child"], t["nchild"]
    assert start[0] == 0 and end[0] == s.n
    leaves = np.nonzero(child < 0)[0]
    assert len(leaves) == st["leaves"]
    cover = np.zeros(s.n, np.int32)
    for q in leaves:
        cover[start[q]:end[q]] += 1
    assert np.all(cover == 1)  # the leaves partition the particles
    depth = np.zeros(len(start), np.int32)
    for q in np.nonzero(child >= 0)[0]:
        kids = np.arange(child[q], child[q] + nch[q])
        assert 1 <= nch[q] <= 8
        assert end[q] - start[q] > leaf
        assert start[kids[0]] == start[q] and end[kids[-1]] == end[q]
        assert np.all(start[kids[1:]] == end[kids[:-1]]) and np.all(end[kids] > start[kids])
        depth[kids] = depth[q] + 1
    for q in leaves:
        assert end[q] - start[q] <= leaf or depth[q] == 10
    assert depth.max() == st["depth"] <= 10
    for q in range(len(start)):  # tight boxes and the largest h
        p = pts[start[q]:end[q]]
        assert np.array_equal(t["lo"][q], p.min(axis=0)) and np.array_equal(t["hi"][q], p.max(axis=0))
        assert t["hmax"][q] == h[start[q]:end[q]].max()


def test_degenerate_inputs():
    # no particles, one particle
    with G.VariableHSearch(3, W.WENDLAND_C2, W.PREC_FP64, 4) as v:
        v.set(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
        v.search()
        off, idx = v.neighbors()
        assert off.tolist() == [0] and idx.size == 0 and v.density().size == 0
        v.set([0.5], [0.5], [0.5], [2.0], [3.0])
        v.search()
        off, idx = v.neighbors()
        rho = v.density()
    w0, _ = O.kernel(W.WENDLAND_C2, 3, 2.0, 0.0)
    assert off.tolist() == [0, 0] and rho[0] == pytest.approx(3.0 * w0, rel=1e-15)
    # every particle at one point: a zero-extent root that cannot split below the last level
    n = 300
    x = np.full(n, 0.25)
    h = np.linspace(0.1, 0.2, n)
    m = np.ones(n)
    for prec in (W.PREC_FP64, W.PREC_FP32):
        s = W.VHSet("point", 3, W.CUBIC_SPLINE, prec, x, x.copy(), x.copy(), h, m)
        with _search(s, leaf=8) as v:
            off = _same_sets(v, s, prec)
            assert np.all(np.diff(off) == n - 1)
            st = v.stats()
            assert st["depth"] == 10 and st["query_runs"] == 2  # 299 neighbours > 64 slots


def test_a_wide_particle_and_two_far_clusters():
    rng = np.random.Generator(np.random.PCG64(77))
    a = rng.random((2000, 2))
    b = rng.random((2000, 2)) + 50.0
    pts = np.vstack([a, b, [[0.5, 0.5]]])
    h = np.full(len(pts), 0.01)
    h[-1] = 0.3  # sees a disc of radius 0.6 of the first cluster, and is seen from it
    s = W.VHSet("two", 2, W.WENDLAND_C2, W.PREC_FP64, pts[:, 0].copy(), pts[:, 1].copy(),
                np.zeros(len(pts)), h, np.ones(len(pts)))
    with _search(s, leaf=16) as v:
        off = _same_sets(v, s, W.PREC_FP64)
    d = np.hypot(a[:, 0] - 0.5, a[:, 1] - 0.5)
    assert off[-1] - off[-2] == int(np.sum(d < 0.6))


def test_list_slots_grow_once_and_repeat_searches_agree():
    s = _blob(4001, 3, W.QUINTIC, W.PREC_FP32, seed=3)
    with _search(s, leaf=16) as v:
        first = v.stats()
        o1, i1 = v.neighbors()
        r1 = v.density()
        v.search()
        second = v.stats()
        o2, i2 = v.neighbors()
        r2 = v.density()
    assert first["query_runs"] == 2 and second["query_runs"] == 1  # quintic: > 64 neighbours
    assert second["slots"] >= second["max_count"]
    assert np.array_equal(o1, o2) and np.array_equal(i1, i2)  # the walk order is fixed
    assert np.array_equal(r1, r2)


def test_refusals():
    with pytest.raises(G.SphError):
        G.VariableHSearch(4, W.WENDLAND_C2, W.PREC_FP64, 10)
    with pytest.raises(G.SphError):
        G.VariableHSearch(3, W.WENDLAND_C2, W.PREC_FP64, 10, leaf_size=0)
    with G.VariableHSearch(2, W.WENDLAND_C2, W.PREC_FP64, 10) as v:
        with pytest.raises(G.SphError):  # searched before any particles were set
            v.search()
        with pytest.raises(G.SphError):  # more particles than the capacity
            v.set(np.zeros(11), np.zeros(11), None, np.ones(11), np.ones(11))
        with pytest.raises(G.SphError):  # h must be positive
            v.set(np.zeros(3), np.zeros(3), None, np.array([1.0, 0.0, 1.0]), np.ones(3))


@pytest.mark.parametrize("dim", [3, 2])
def test_full_size_sampled_rows(dim):
    """The bench's set (10^6 particles, FP32) on 64 sampled particles, each against every
    other particle in the oracle: sets bit-exact, densities within the FP32 bar."""
    s = W.gaussian_blob(1_000_000, dim=dim, precision=W.PREC_FP32)
    rng = np.random.Generator(np.random.PCG64(8))
    rows = np.concatenate([rng.choice(s.n, 62, replace=False),
                           [int(np.argmin(s.h)), int(np.argmax(s.h))]])
    with _search(s, leaf=16) as v:
        off, idx = v.neighbors()
        rho = v.density()
        st = v.stats()
    ro, ri, rr = O.vh_rows(s.dim, s.kernel, s.precision, s.x, s.y, s.z, s.h, s.m, rows)
    for q, i in enumerate(rows):
        assert np.array_equal(np.sort(idx[off[i]:off[i + 1]]), ri[ro[q]:ro[q + 1]]), i
    assert np.max(np.abs(rho[rows] / rr - 1.0)) <= 1e-5
    assert st["pairs"] == off[-1]


def test_phase_timing():
    s = _blob(20000, 3, W.WENDLAND_C2, W.PREC_FP32, seed=21)
    with _search(s, leaf=16) as v:
        with pytest.raises(G.SphError):  # the last search was not timed
            v.phase_times()
        v.set_timing(True)
        v.search()
        ph = v.phase_times()
        v.set_timing(False)
        v.search()
        off, _ = v.neighbors()
        pairs = v.stats()["pairs"]
    assert ph["build"] > 0.0 and ph["query"] > 0.0
    assert off[-1] == pairs > 0
