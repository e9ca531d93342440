"""Helpers shared by the GPU parity tests (no SPH arithmetic here)."""
import numpy as np

import oracle as O
import paper_1909_04504_gb300 as G


def sim_of(wl, precision=None):
    return G.Simulation.from_workload(wl, precision=precision)


def oracle_wl(wl, precision=None):
    if precision is not None and precision != wl.precision:
        wl = wl.with_precision(precision)
    return wl


def normwise(a, b):
    """max_i |a_i - b_i| / max_i |b_i| (0 when both vanish)."""
    den = np.max(np.abs(b))
    num = np.max(np.abs(a - b))
    if den == 0.0:
        return num
    return num / den


def rel_l2(a, b):
    den = np.linalg.norm(b)
    num = np.linalg.norm(a - b)
    if den == 0.0:
        return num
    return num / den


def csr_equal(off_a, idx_a, off_b, idx_b):
    return np.array_equal(np.asarray(off_a, np.int64), np.asarray(off_b, np.int64)) and \
        np.array_equal(np.asarray(idx_a, np.int64), np.asarray(idx_b, np.int64))


_AXIS = {"x": 0, "y": 1, "z": 2}


def increment(wl, prop, new, old):
    """new - old, taken across the periodic boundary by the minimum image on periodic
    position axes (a particle that wrapped moved by the short way)."""
    d = np.asarray(new, np.float64) - np.asarray(old, np.float64)
    ax = _AXIS.get(prop)
    if ax is not None and wl.periodic[ax]:
        L = wl.hi[ax] - wl.lo[ax]
        d = d - L * np.round(d / L)
    return d


def field_error(wl, prop, gpu, ora, start):
    """Error measure of a field after steps from a common start: FP64 mode normwise on the
    field itself; FP32 mode relative L2 of the change from the start (a step moves x by
    ~1e-8 of its value and rho by ~1e-6, so an absolute-field L2 would not see a wrong
    drift or density update)."""
    if wl.precision == 0:
        return normwise(gpu, ora)
    return rel_l2(increment(wl, prop, gpu, start), increment(wl, prop, ora, start))


def field_ok(wl, prop, gpu, ora, start, fp64_tol=1e-10, fp32_tol=1e-4):
    tol = fp64_tol if wl.precision == 0 else fp32_tol
    return field_error(wl, prop, gpu, ora, start) <= tol
