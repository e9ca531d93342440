"""The allocation-free cell sort (sph_cell_sort_noalloc), for callers that cannot allocate
device memory, gives the same permutation and cell table as the allocating path
(sph_create + sph_get_cells) and as the oracle's cell search on the same positions.

Called through the C ABI with device buffers owned by the test. Calls in a row on
different problems check that the shared scratch carries nothing from one call into the
next; the last call repeats the first. One problem holds exactly the largest accepted
count (2^20 particles, 256 sort tiles, three radix passes), so the whole scratch extent is
used. Integer outputs: compared bit for bit."""
import ctypes as C

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


def _lib():
    import paper_1909_04504_gb300 as G
    from paper_1909_04504_gb300 import binding
    L = G.load()
    f = L.sph_cell_sort_noalloc
    f.argtypes = [C.POINTER(binding.Domain), C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64,
                  C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p]
    f.restype = C.c_int
    return L, binding


def _domain(binding, wl):
    d = binding.Domain()
    d.dim, d.kernel, d.precision, d.h = wl.dim, wl.kernel, wl.precision, wl.h
    for k in range(3):
        d.periodic[k] = int(wl.periodic[k])
        d.lo[k] = float(wl.lo[k])
        d.hi[k] = float(wl.hi[k])
    return d


def _noalloc_sort(wl):
    import torch
    L, binding = _lib()
    dom = _domain(binding, wl)
    dev = torch.device("cuda", 0)
    xs = [torch.tensor(wl.concat(k), dtype=torch.float64, device=dev) for k in ("x", "y", "z")]
    n = xs[0].shape[0]
    ncells = C.c_int64()
    st = L.sph_cell_sort_noalloc(C.byref(dom), None, None, None, n, None, None, 0,
                                 C.byref(ncells), None)
    assert st == 0, L.sph_last_error(None)
    order = torch.empty(n, dtype=torch.int32, device=dev)
    offsets = torch.empty(ncells.value + 1, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = L.sph_cell_sort_noalloc(C.byref(dom), xs[0].data_ptr(), xs[1].data_ptr(),
                                 xs[2].data_ptr() if wl.dim == 3 else None, n,
                                 order.data_ptr(), offsets.data_ptr(), ncells.value + 1,
                                 C.byref(ncells), C.c_void_p(stream.cuda_stream))
    assert st == 0, L.sph_last_error(None)
    torch.cuda.synchronize()
    return (order.cpu().numpy().view(np.uint32).astype(np.int64),
            offsets.cpu().numpy().view(np.uint32))


def _allocating_sort(wl):
    import paper_1909_04504_gb300 as G
    with G.Simulation.from_workload(wl) as sim:
        _, offsets, order = sim.cells()
    return order, offsets


def test_noalloc_cell_sort_matches_allocating_path_twice():
    problems = [W.dam_break_2d(dx=0.02, precision=W.PREC_FP32),
                W.taylor_green_3d(n=24, precision=W.PREC_FP64),
                W.falling_cube_3d(n=20, precision=W.PREC_FP32)]  # cubic spline kernel
    assert problems[2].kernel == W.CUBIC_SPLINE
    for wl in problems + problems[:1]:
        order_n, off_n = _noalloc_sort(wl)
        order_a, off_a = _allocating_sort(wl)
        assert np.array_equal(off_n, off_a)
        assert np.array_equal(order_n, order_a)
        _, off_o, order_o = O.cells(wl, wl.concat("x"), wl.concat("y"), wl.concat("z"))
        assert np.array_equal(off_n, off_o)
        assert np.array_equal(order_n, order_o)


def test_noalloc_cell_sort_at_the_largest_accepted_count():
    wl = W.taylor_green_2d(n=1024, precision=W.PREC_FP32)
    assert wl.n_total == 1 << 20  # SPH_NOALLOC_MAX_PARTICLES
    small = W.dam_break_2d(dx=0.04, precision=W.PREC_FP64)
    for w in (wl, small, wl):
        order_n, off_n = _noalloc_sort(w)
        _, off_o, order_o = O.cells(w, w.concat("x"), w.concat("y"), w.concat("z"))
        assert np.array_equal(off_n, off_o)
        assert np.array_equal(order_n, order_o)


def test_noalloc_cell_sort_rejects_oversize_input():
    L, binding = _lib()
    wl = W.taylor_green_2d(n=20)
    dom = _domain(binding, wl)
    ncells = C.c_int64()
    buf = (C.c_uint32 * 1)()
    st = L.sph_cell_sort_noalloc(C.byref(dom), None, None, None, (1 << 20) + 1,
                                 C.addressof(buf), C.addressof(buf), 1, C.byref(ncells), None)
    assert st == 6  # SPH_ERR_CAPACITY, before any device work
    assert b"exceeds" in L.sph_last_error(None)
