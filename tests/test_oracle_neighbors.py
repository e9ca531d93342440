"""Pins of the oracle's neighbour search (Sec. 2.2, uniform grid with a 3^d stencil)
against brute force over all pairs, integer lattice counts and invariances."""
import itertools
import math

import numpy as np
import pytest

import oracle as O
import workloads as W


def _wl(dim, kind, h, lo, hi, periodic, precision):
    if dim == 2:
        wl = W.taylor_green_2d(n=4, jitter=0.0)
    else:
        wl = W.taylor_green_3d(n=4, jitter=0.0)
    wl.kernel, wl.h, wl.precision = kind, h, precision
    wl.lo, wl.hi, wl.periodic = list(lo), list(hi), list(periodic)
    return wl


def _points(kind_pts, dim, n, lo, hi, rng, spacing):
    lo, hi = np.array(lo[:dim]), np.array(hi[:dim])
    if kind_pts == "uniform":
        p = lo + (hi - lo) * rng.random((n, dim))
    elif kind_pts == "clustered":
        centres = lo + (hi - lo) * rng.random((5, dim))
        p = centres[rng.integers(0, 5, n)] + rng.normal(0, 0.7 * spacing, (n, dim))
        p = np.clip(p, lo, hi - 1e-12)
    elif kind_pts == "coincident":
        base = lo + (hi - lo) * rng.random((n // 4, dim))
        p = base[rng.integers(0, n // 4, n)]
    else:  # jittered lattice
        m = int(round(n ** (1.0 / dim)))
        axes = [lo[d] + (np.arange(m) + 0.5) * (hi[d] - lo[d]) / m for d in range(dim)]
        g = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, dim)
        p = g + rng.uniform(-0.05, 0.05, g.shape) * (hi - lo) / m
    cols = [np.ascontiguousarray(p[:, d]) for d in range(dim)]
    while len(cols) < 3:
        cols.append(np.zeros(p.shape[0]))
    return cols


CASES = list(itertools.product(
    [2, 3], [W.QUINTIC, W.WENDLAND_C2], [W.PREC_FP64, W.PREC_FP32],
    ["uniform", "clustered", "coincident", "lattice"], [0, 1]))


@pytest.mark.parametrize("dim,kind,prec,pts,periodic", CASES)
def test_cells_equal_brute_force(dim, kind, prec, pts, periodic):
    rng = np.random.Generator(np.random.PCG64(17 + dim + 3 * kind + 7 * prec))
    n = 900 if dim == 2 else 1000
    lo = [-0.3, 0.1, 2.0]
    hi = [0.7, 0.9, 2.8]
    h = 0.021 if dim == 2 else 0.04
    wl = _wl(dim, kind, h, lo, hi, [periodic] * dim + [0] * (3 - dim), prec)
    x, y, z = _points(pts, dim, n, lo, hi, rng, h)
    off_c, idx_c, cand = O.neighbors(wl, x, y, z)
    off_b, idx_b, _ = O.neighbors(wl, x, y, z, brute=True)
    assert np.array_equal(off_c, off_b)
    assert np.array_equal(idx_c, idx_b)
    assert idx_c.shape[0] > 0
    # symmetric relation, no self pairs, ascending rows
    rows = np.repeat(np.arange(x.shape[0]), np.diff(off_c))
    assert not np.any(rows == idx_c)
    pairs = set(zip(rows.tolist(), idx_c.tolist()))
    assert all((j, i) in pairs for i, j in pairs)
    for i in range(x.shape[0]):
        seg = idx_c[off_c[i]:off_c[i + 1]]
        assert np.all(np.diff(seg) > 0)


def _lattice_count(dim, radius):
    """Number of nonzero integer vectors with |k| < radius."""
    R = int(math.ceil(radius))
    c = 0
    for k in itertools.product(range(-R, R + 1), repeat=dim):
        s = sum(v * v for v in k)
        if 0 < s < radius * radius:
            c += 1
    return c


@pytest.mark.parametrize("dim,kind,hdx,expect", [
    (2, W.WENDLAND_C2, 1.3, 20), (3, W.WENDLAND_C2, 1.3, 80),
    (2, W.QUINTIC, 1.01, 28), (3, W.QUINTIC, 1.01, 122)])
def test_periodic_lattice_counts(dim, kind, hdx, expect):
    """On a periodic lattice every particle has the same neighbour count, equal to the
    number of integer vectors strictly inside the support radius (in units of dx)."""
    n = 20 if dim == 2 else 12
    support = 3.0 if kind == W.QUINTIC else 2.0
    assert _lattice_count(dim, support * hdx) == expect
    if dim == 2:
        wl = W.taylor_green_2d(n=n, jitter=0.0, hdx=hdx)
    else:
        wl = W.taylor_green_3d(n=n, jitter=0.0)
        wl.h = hdx / n
    wl.kernel = kind
    s = O.state_of(wl)
    for prec in (W.PREC_FP64, W.PREC_FP32):
        off, idx, cand = O.neighbors(wl, s["x"], s["y"], s["z"], precision=prec)
        assert np.all(np.diff(off) == expect)


def test_cell_table_is_a_stable_bucket_sort():
    wl = W.dam_break_2d(dx=0.05)
    s = O.state_of(wl)
    nc3, cs, ncells = O.grid(wl)
    cell_of, offsets, order = O.cells(wl, s["x"], s["y"])
    assert offsets[0] == 0 and offsets[-1] == s["x"].shape[0]
    assert np.all(np.diff(offsets.astype(np.int64)) >= 0)
    assert np.array_equal(np.bincount(cell_of, minlength=ncells), np.diff(offsets.astype(np.int64)))
    assert np.array_equal(order, np.argsort(cell_of, kind="stable"))
    # cell coordinates bracket the position: lo + c cs <= x < lo + (c + 1) cs (inside the box)
    cx = cell_of % nc3[0]
    cy = cell_of // nc3[0]
    for c, p, d in ((cx, s["x"], 0), (cy, s["y"], 1)):
        assert np.all(wl.lo[d] + c * cs[d] <= p + 1e-12)
        assert np.all(p < wl.lo[d] + (c + 1) * cs[d] + 1e-12)
    # cells are no smaller than the support radius
    assert min(cs[:2]) >= 2.0 * wl.h


def test_grid_rejects_short_periodic_axis():
    wl = W.taylor_green_2d(n=5, jitter=0.0)  # support 0.6 > L/3
    with pytest.raises(ValueError):
        O.grid(wl)


def test_permutation_invariance():
    wl = W.taylor_green_2d(n=30)
    s = O.state_of(wl)
    rng = np.random.Generator(np.random.PCG64(5))
    perm = rng.permutation(s["x"].shape[0])
    off, idx, _ = O.neighbors(wl, s["x"], s["y"])
    off_p, idx_p, _ = O.neighbors(wl, s["x"][perm], s["y"][perm])
    for k in range(0, perm.shape[0], 7):
        a = np.sort(perm[idx_p[off_p[k]:off_p[k + 1]]])
        b = idx[off[perm[k]]:off[perm[k] + 1]]
        assert np.array_equal(a, b)
