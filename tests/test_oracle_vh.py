"""Pins of the oracle's variable-smoothing-length neighbour relation and density (the use
case of the octree search of Sec. 2.2, reading C-VH):

  j != i is a neighbour of i when |x_i - x_j| < k max(h_i, h_j),
  rho_i = m_i W(0, h_i) + sum_{j in N(i)} m_j W(|x_i - x_j|, (h_i + h_j) / 2),

against a library routine (scipy's k-d tree, which shares no code with the oracle), lattice
counts in closed form (including points exactly on the support boundary, which the strict
inequality excludes), the two-scale case a uniform grid handles badly, and the density
composed by hand from the pinned kernel."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

spatial = pytest.importorskip("scipy.spatial")


def _sets(off, idx):
    return [set(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]


def _kdtree_sets(pts, h, k):
    """j in S_i iff |x_i - x_j| <= k h_i or <= k h_j (ties have measure zero here)."""
    t = spatial.cKDTree(pts)
    n = len(pts)
    S = [set() for _ in range(n)]
    for i in range(n):
        for j in t.query_ball_point(pts[i], k * h[i]):
            if j != i:
                S[i].add(j)
                S[j].add(i)
    return S


@pytest.mark.parametrize("dim,kernel", [(2, W.WENDLAND_C2), (3, W.QUINTIC), (3, W.CUBIC_SPLINE)])
def test_random_sets_match_a_kdtree(dim, kernel):
    rng = np.random.Generator(np.random.PCG64(11 + dim))
    n = 600
    pts = rng.random((n, dim))
    h = 0.01 + 0.06 * rng.random(n) ** 3  # a wide spread of support radii
    k = 3.0 if kernel == W.QUINTIC else 2.0
    z = pts[:, 2] if dim == 3 else None
    off, idx = O.vh_neighbors(dim, kernel, W.PREC_FP64, pts[:, 0], pts[:, 1], z, h)
    got = _sets(off, idx)
    assert got == _kdtree_sets(pts, h, k)
    for i in range(n):  # ascending ids, symmetric relation
        row = idx[off[i]:off[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert all(i in got[j] for j in row)


@pytest.mark.parametrize("dim,kernel,hdx,count", [
    (2, W.WENDLAND_C2, 1.2, 20),   # |v|^2 < 5.76: shells 1, 2, 4, 5
    (2, W.QUINTIC, 1.0, 24),       # |v|^2 < 9: shells 1, 2, 4, 5, 8 (|v|^2 = 9 excluded)
    (3, W.WENDLAND_C2, 1.2, 56),   # shells 1, 2, 3, 4, 5
    (3, W.CUBIC_SPLINE, 1.0, 26),  # |v|^2 < 4: shells 1, 2, 3 (|v|^2 = 4 excluded)
])
@pytest.mark.parametrize("prec", [W.PREC_FP64, W.PREC_FP32])
def test_lattice_counts(dim, kernel, hdx, count, prec):
    """Integer lattice, uniform h: an interior particle has the closed-form count; the
    coordinates are exact in FP32, so both precision modes give it."""
    m = 9
    g = np.arange(m, dtype=np.float64)
    axes = np.meshgrid(*([g] * dim), indexing="ij")
    pts = np.stack([a.ravel() for a in axes], axis=1)
    h = np.full(len(pts), hdx)
    z = pts[:, 2] if dim == 3 else None
    off, idx = O.vh_neighbors(dim, kernel, prec, pts[:, 0], pts[:, 1], z, h)
    centre = int(np.argmin(np.sum((pts - (m - 1) / 2) ** 2, axis=1)))
    assert off[centre + 1] - off[centre] == count


def test_a_wide_particle_sees_and_is_seen():
    """A lattice of small h with one particle of large H at its centre: with the max
    criterion the wide particle's neighbours are the lattice points within k H, and each of
    them has the wide particle among its own neighbours (a gather-only search would miss
    that side)."""
    m = 21
    g = np.arange(m, dtype=np.float64)
    X, Y = np.meshgrid(g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel()], axis=1)
    pts = np.vstack([pts, [[10.25, 10.5]]])
    h = np.full(len(pts), 0.6)  # k h = 1.2: the four lattice neighbours only
    H = 3.1
    h[-1] = H
    off, idx = O.vh_neighbors(2, W.WENDLAND_C2, W.PREC_FP64, pts[:, 0], pts[:, 1], None, h)
    S = _sets(off, idx)
    wide = len(pts) - 1
    d = np.hypot(pts[:-1, 0] - 10.25, pts[:-1, 1] - 10.5)
    inside = set(np.nonzero(d < 2.0 * H)[0].tolist())
    assert S[wide] == inside and len(inside) == int(np.sum(d < 6.2))
    for j in range(wide):
        assert (wide in S[j]) == (j in inside)
    corner = 0  # a lattice corner, out of the wide particle's reach: two lattice neighbours
    assert S[corner] == {1, m}


def test_empty_and_single():
    off, idx = O.vh_neighbors(3, W.WENDLAND_C2, W.PREC_FP64, np.zeros(0), np.zeros(0),
                              np.zeros(0), np.zeros(0))
    assert off.tolist() == [0] and idx.size == 0
    off, idx = O.vh_neighbors(3, W.WENDLAND_C2, W.PREC_FP64, [0.5], [0.5], [0.5], [1.0])
    assert off.tolist() == [0, 0]
    rho = O.vh_density(3, W.WENDLAND_C2, W.PREC_FP64, [0.5], [0.5], [0.5], [2.0], [3.0])
    w0, _ = O.kernel(W.WENDLAND_C2, 3, 2.0, 0.0)
    assert rho[0] == 3.0 * w0


def test_density_of_two_particles_by_hand():
    """rho_1 = m_1 W(0, h_1) + m_2 W(r, (h_1 + h_2) / 2); a pair inside k max(h) but
    outside k h_12 adds exactly nothing."""
    h1, h2, m1, m2 = 0.4, 1.0, 2.0, 5.0
    for r in (0.3, 0.9, 1.15):
        x = np.array([0.0, r])
        rho = O.vh_density(2, W.WENDLAND_C2, W.PREC_FP64, x, np.zeros(2), None,
                           np.array([h1, h2]), np.array([m1, m2]))
        w11, _ = O.kernel(W.WENDLAND_C2, 2, h1, 0.0)
        w22, _ = O.kernel(W.WENDLAND_C2, 2, h2, 0.0)
        w12, _ = O.kernel(W.WENDLAND_C2, 2, 0.5 * (h1 + h2), r)
        assert rho[0] == pytest.approx(m1 * w11 + m2 * w12, rel=1e-14)
        assert rho[1] == pytest.approx(m2 * w22 + m1 * w12, rel=1e-14)
        if r >= 2.0 * 0.5 * (h1 + h2):
            assert w12 == 0.0 and rho[0] == m1 * w11


@pytest.mark.parametrize("dim,kernel", [(2, W.WENDLAND_C2), (3, W.WENDLAND_C2), (2, W.QUINTIC),
                                        (3, W.CUBIC_SPLINE)])
def test_uniform_lattice_density(dim, kernel):
    """Uniform h on a lattice of spacing dx and mass m = rho0 dx^d: an interior density is
    the lattice sum m sum_{v in Z^d, |v| dx < k h} W(|v| dx, h), formed here over the
    integer vectors from the pinned kernel; it is rho0 up to the kernel's lattice error
    (about 1 % for the Wendland C2 at h = 1.3 dx)."""
    dx, rho0, hdx = 0.1, 1000.0, 1.3
    m = 15 if dim == 2 else 11
    g = dx * np.arange(m)
    axes = np.meshgrid(*([g] * dim), indexing="ij")
    pts = np.stack([a.ravel() for a in axes], axis=1)
    n = len(pts)
    h = np.full(n, hdx * dx)
    mass = rho0 * dx ** dim
    z = pts[:, 2] if dim == 3 else None
    rho = O.vh_density(dim, kernel, W.PREC_FP64, pts[:, 0], pts[:, 1], z, h, np.full(n, mass))
    k = 3.0 if kernel == W.QUINTIC else 2.0
    edge = k * hdx * dx
    inner = np.all((pts >= g[0] + edge - 1e-12) & (pts <= g[-1] - edge + 1e-12), axis=1)
    assert inner.sum() > 0
    r = int(math.ceil(k * hdx))
    vs = np.stack([a.ravel() for a in np.meshgrid(*([np.arange(-r, r + 1)] * dim),
                                                  indexing="ij")], axis=1)
    lattice = sum(mass * O.kernel(kernel, dim, hdx * dx, float(np.linalg.norm(v)) * dx)[0]
                  for v in vs if float(np.dot(v, v)) < (k * hdx) ** 2)
    assert np.max(np.abs(rho[inner] / lattice - 1.0)) < 1e-12
    assert abs(lattice / rho0 - 1.0) < 0.015


def test_density_is_order_independent():
    rng = np.random.Generator(np.random.PCG64(3))
    n = 300
    pts = rng.random((n, 3))
    h = 0.05 + 0.1 * rng.random(n)
    m = 0.5 + rng.random(n)
    rho = O.vh_density(3, W.QUINTIC, W.PREC_FP64, pts[:, 0], pts[:, 1], pts[:, 2], h, m)
    p = rng.permutation(n)
    rp = O.vh_density(3, W.QUINTIC, W.PREC_FP64, pts[p, 0], pts[p, 1], pts[p, 2], h[p], m[p])
    assert np.allclose(rp, rho[p], rtol=1e-13, atol=0)
    assert math.isfinite(float(np.sum(rho)))


def test_selected_rows_agree_with_the_full_lists():
    """The selected-rows form (for sets too large for all-pairs lists) returns the rows and
    densities of the full form, bit for bit."""
    s = W.gaussian_blob(2000, dim=3, seed=5)
    rows = np.array([0, 17, 999, 1998])
    for prec in (W.PREC_FP64, W.PREC_FP32):
        off, idx = O.vh_neighbors(3, s.kernel, prec, s.x, s.y, s.z, s.h)
        rho = O.vh_density(3, s.kernel, prec, s.x, s.y, s.z, s.h, s.m)
        ro, ri, rr = O.vh_rows(3, s.kernel, prec, s.x, s.y, s.z, s.h, s.m, rows)
        for q, i in enumerate(rows):
            assert np.array_equal(ri[ro[q]:ro[q + 1]], idx[off[i]:off[i + 1]])
        assert np.array_equal(rr, rho[rows])
