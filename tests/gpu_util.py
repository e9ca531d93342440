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
