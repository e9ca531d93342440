"""CPU oracle for the WCSPH particle loop (FP64, plain loops, no shared code with CUDA).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never
does. The arithmetic lives in ``sph_oracle.cpp`` (compiled with
``-ffp-contract=off``); this module only marshals numpy arrays.

Functions (each follows the paper's passage named in the C source):
  kernel(kind, dim, h, r)          W and dW/dr (Sec. 2 kernel interpolation)
  grid(wl)                          cells per axis / cell sizes (Sec. 2.2)
  cells(wl, x, y, z)                linear cell per particle + cell offsets (Sec. 2.2)
  neighbors(wl, x, y, z, brute)     CSR neighbour sets, ascending ids (Sec. 2.2)
  rhs(wl, state)                    one RHS evaluation (Sec. 2 equations, Sec. 3.2 groups; the
                                    EDAC pressure equation of Sec. 2.3's scheme list)
  run(wl, state, dt, steps)         predictor-corrector steps (Sec. 2.1)
  grad(wl, state, dt, K, du, dnu)   forward-mode derivative of the final kinetic energy
  vh_neighbors(dim, kernel, prec, x, y, z, h)
                                    CSR neighbour sets with a per-particle smoothing length,
                                    every pair examined (Sec. 2.2, the octree's use case)
  vh_density(dim, kernel, prec, x, y, z, h, m)
                                    summation density with h_ij = (h_i + h_j) / 2 (Eq. 2)
  vh_rows(dim, kernel, prec, x, y, z, h, m, rows)
                                    both for selected particles only (large sets)
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Dict, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.cpp")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libsph_oracle.so")
HIST = 10  # t, dt, KE, max|u|, Px, Py, Pz, max|a|, pairs, candidates


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, no FP contraction, OpenMP over destinations)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c++17",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("density", C.c_int32), ("periodic", C.c_int32 * 3), ("brute", C.c_int32),
                ("wall_bc", C.c_int32), ("integrator", C.c_int32), ("h", C.c_double), ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("rho0", C.c_double), ("c0", C.c_double), ("gamma", C.c_double),
                ("nu", C.c_double), ("eta", C.c_double), ("alpha", C.c_double),
                ("xsph_eps", C.c_double), ("g", C.c_double * 3), ("edac_alpha", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d, i64, i32 = C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        u32, u8, P = C.POINTER(C.c_uint32), C.POINTER(C.c_uint8), C.POINTER(Params)
        _lib.ora_kernel.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double, d, d]
        _lib.ora_grid.argtypes = [P, i32, d, i64]
        _lib.ora_cells.argtypes = [P, C.c_int64, d, d, d, u32, u32, i64]
        _lib.ora_neighbors.argtypes = [P, C.c_int64, d, d, d, i64, i32, i64]
        _lib.ora_neighbors.restype = C.c_int64
        _lib.ora_rhs.argtypes = [P, C.c_int64] + [d] * 8 + [u8] + [d] * 9 + [i64, i64, d]
        _lib.ora_run.argtypes = [P, C.c_int64] + [d] * 7 + [d, u8, C.c_double, C.c_int32, d, d]
        _lib.ora_grad.argtypes = ([P, C.c_int64] + [d] * 8 + [u8, C.c_double, C.c_int32]
                                  + [d] * 3 + [C.c_double, C.c_double, d, d])
        _lib.ora_threads.restype = C.c_int
        _lib.ora_vh_neighbors.argtypes = [C.c_int32] * 3 + [C.c_int64] + [d] * 4 + [i64, i32]
        _lib.ora_vh_neighbors.restype = C.c_int64
        _lib.ora_vh_density.argtypes = [C.c_int32] * 3 + [C.c_int64] + [d] * 6
        _lib.ora_vh_rows.argtypes = ([C.c_int32] * 3 + [C.c_int64] + [d] * 5
                                     + [i64, C.c_int64, i64, i32, d])
        _lib.ora_vh_rows.restype = C.c_int64
    return _lib


def threads() -> int:
    return int(lib().ora_threads())


def params(wl, brute: bool = False, **over) -> Params:
    """Params from a ``workloads.Workload`` (keyword overrides allowed)."""
    p = Params()
    p.dim = wl.dim
    p.kernel = wl.kernel
    p.precision = wl.precision
    p.density = wl.density
    for d in range(3):
        p.periodic[d] = int(wl.periodic[d])
        p.lo[d] = float(wl.lo[d])
        p.hi[d] = float(wl.hi[d])
        p.g[d] = float(wl.g[d])
    p.brute = int(brute)
    p.wall_bc = int(getattr(wl, "wall_bc", 0))
    p.integrator = int(getattr(wl, "integrator", 0))
    p.h = wl.h
    p.rho0, p.c0, p.gamma = wl.rho0, wl.c0, wl.gamma
    p.nu, p.eta, p.alpha, p.xsph_eps = wl.nu, wl.eta, wl.alpha, wl.xsph_eps
    p.edac_alpha = getattr(wl, "edac_alpha", 0.5)
    for k, v in over.items():
        setattr(p, k, v)
    return p


def _d(a: Optional[np.ndarray]):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def state_of(wl) -> Dict[str, np.ndarray]:
    """Concatenated state of a workload (global ids in array order)."""
    s = {k: _f64(wl.concat(k)) for k in ("x", "y", "z", "u", "v", "w", "rho", "m", "p")}
    s["role"] = np.ascontiguousarray(wl.roles(), dtype=np.uint8)
    return s


def kernel(kind: int, dim: int, h: float, r: float):
    W, dW = C.c_double(), C.c_double()
    rc = lib().ora_kernel(kind, dim, h, r, C.byref(W), C.byref(dW))
    if rc:
        raise ValueError("bad kernel arguments")
    return W.value, dW.value


def grid(wl, **over):
    p = params(wl, **over)
    n = (C.c_int32 * 3)()
    cs = (C.c_double * 3)()
    nc = C.c_int64()
    rc = lib().ora_grid(C.byref(p), n, cs, C.byref(nc))
    if rc:
        raise ValueError(f"invalid grid ({rc})")
    return list(n), list(cs), nc.value


def cells(wl, x, y, z=None, **over):
    p = params(wl, **over)
    x, y = _f64(x), _f64(y)
    z = _f64(z) if z is not None else np.zeros_like(x)
    n = x.shape[0]
    _, _, nc = grid(wl, **over)
    cell_of = np.zeros(n, np.uint32)
    offsets = np.zeros(nc + 1, np.uint32)
    order = np.zeros(n, np.int64)
    rc = lib().ora_cells(C.byref(p), n, _d(x), _d(y), _d(z),
                         cell_of.ctypes.data_as(C.POINTER(C.c_uint32)),
                         offsets.ctypes.data_as(C.POINTER(C.c_uint32)),
                         order.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc:
        raise ValueError(f"cells failed ({rc})")
    return cell_of, offsets, order


def neighbors(wl, x, y, z=None, brute: bool = False, **over):
    """CSR (offsets int64[n+1], idx int32[nnz]) and the candidate count."""
    p = params(wl, brute=brute, **over)
    x, y = _f64(x), _f64(y)
    z = _f64(z) if z is not None else np.zeros_like(x)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int64)
    cand = C.c_int64()
    L = lib()
    i64 = C.POINTER(C.c_int64)
    nnz = L.ora_neighbors(C.byref(p), n, _d(x), _d(y), _d(z), off.ctypes.data_as(i64),
                          None, C.byref(cand))
    if nnz < 0:
        raise ValueError(f"neighbors failed ({nnz})")
    idx = np.zeros(max(nnz, 1), np.int32)
    L.ora_neighbors(C.byref(p), n, _d(x), _d(y), _d(z), off.ctypes.data_as(i64),
                    idx.ctypes.data_as(C.POINTER(C.c_int32)), C.byref(cand))
    return off, idx[:nnz], cand.value


def rhs(wl, s: Dict[str, np.ndarray], **over) -> Dict[str, np.ndarray]:
    """One RHS evaluation on state ``s``: arho, ax, ay, az, xsx, xsy, xsz, rho, p."""
    p = params(wl, **over)
    n = s["x"].shape[0]
    out = {k: np.zeros(n) for k in ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz", "rho", "p")}
    pairs, cand = C.c_int64(), C.c_int64()
    rc = lib().ora_rhs(C.byref(p), n, *(_d(_f64(s[k])) for k in ("x", "y", "z", "u", "v", "w",
                                                                  "rho", "m")),
                       s["role"].ctypes.data_as(C.POINTER(C.c_uint8)),
                       *(_d(out[k]) for k in ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz",
                                              "rho", "p")),
                       C.byref(pairs), C.byref(cand),
                       _d(_f64(s["p"])) if "p" in s else None)
    if rc:
        raise ValueError(f"rhs failed ({rc})")
    out["pairs"] = pairs.value
    out["candidates"] = cand.value
    return out


def run(wl, s: Dict[str, np.ndarray], dt: float, steps: int, **over):
    """Advance a copy of ``s`` by ``steps`` steps; returns (state, history[steps+1, 10])."""
    p = params(wl, **over)
    st = {k: np.array(v, copy=True) for k, v in s.items()}
    for k in ("x", "y", "z", "u", "v", "w", "rho", "m"):
        st[k] = _f64(st[k]).copy()
    n = st["x"].shape[0]
    st["p"] = _f64(st["p"]).copy() if "p" in st else np.zeros(n)
    hist = np.zeros((steps + 1, HIST))
    rc = lib().ora_run(C.byref(p), n, *(_d(st[k]) for k in ("x", "y", "z", "u", "v", "w", "rho")),
                       _d(st["m"]), st["role"].ctypes.data_as(C.POINTER(C.c_uint8)), float(dt),
                       int(steps), _d(hist), _d(st["p"]))
    if rc:
        raise ValueError(f"run failed ({rc})")
    return st, hist


def grad(wl, s: Dict[str, np.ndarray], dt: float, K: int, du=None, dv=None, dw=None,
         dnu: float = 0.0, dalpha: float = 0.0, **over):
    """(KE, dKE) with dKE the derivative of the final kinetic energy along the seed."""
    p = params(wl, **over)
    n = s["x"].shape[0]
    ke, dke = C.c_double(), C.c_double()
    dirs = [None if a is None else _f64(a) for a in (du, dv, dw)]
    rc = lib().ora_grad(C.byref(p), n, *(_d(_f64(s[k])) for k in ("x", "y", "z", "u", "v", "w",
                                                                   "rho", "m")),
                        s["role"].ctypes.data_as(C.POINTER(C.c_uint8)), float(dt), int(K),
                        *(_d(a) for a in dirs), float(dnu), float(dalpha),
                        C.byref(ke), C.byref(dke))
    if rc:
        raise ValueError(f"grad failed ({rc})")
    return ke.value, dke.value


def _vh_args(dim, x, y, z, h):
    x, y, h = _f64(x), _f64(y), _f64(h)
    z = _f64(z) if z is not None else np.zeros_like(x)
    if dim == 2:
        z = np.zeros_like(x)
    return x, y, z, h


def vh_neighbors(dim: int, kernel: int, precision: int, x, y, z, h):
    """CSR (offsets int64[n+1], idx int32[nnz]) of the variable-h neighbour relation
    |x_i - x_j| < k max(h_i, h_j), j != i, ascending ids."""
    x, y, z, h = _vh_args(dim, x, y, z, h)
    n = x.shape[0]
    off = np.zeros(n + 1, np.int64)
    L = lib()
    i64 = C.POINTER(C.c_int64)
    nnz = L.ora_vh_neighbors(dim, kernel, precision, n, _d(x), _d(y), _d(z), _d(h),
                             off.ctypes.data_as(i64), None)
    if nnz < 0:
        raise ValueError(f"vh_neighbors failed ({nnz})")
    idx = np.zeros(max(nnz, 1), np.int32)
    L.ora_vh_neighbors(dim, kernel, precision, n, _d(x), _d(y), _d(z), _d(h),
                       off.ctypes.data_as(i64), idx.ctypes.data_as(C.POINTER(C.c_int32)))
    return off, idx[:nnz]


def vh_density(dim: int, kernel: int, precision: int, x, y, z, h, m):
    """rho_i = m_i W(0, h_i) + sum_j m_j W(r_ij, (h_i + h_j) / 2) over the variable-h
    neighbour set of the precision mode."""
    x, y, z, h = _vh_args(dim, x, y, z, h)
    m = _f64(m)
    rho = np.zeros(x.shape[0])
    rc = lib().ora_vh_density(dim, kernel, precision, x.shape[0], _d(x), _d(y), _d(z), _d(h),
                              _d(m), _d(rho))
    if rc:
        raise ValueError(f"vh_density failed ({rc})")
    return rho


def vh_rows(dim: int, kernel: int, precision: int, x, y, z, h, m, rows):
    """(offsets, idx, rho) of the selected particles: CSR over the selection, ascending ids."""
    x, y, z, h = _vh_args(dim, x, y, z, h)
    m = _f64(m)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    nr = rows.shape[0]
    off = np.zeros(nr + 1, np.int64)
    rho = np.zeros(nr)
    L = lib()
    i64 = C.POINTER(C.c_int64)
    nnz = L.ora_vh_rows(dim, kernel, precision, x.shape[0], _d(x), _d(y), _d(z), _d(h), _d(m),
                        rows.ctypes.data_as(i64), nr, off.ctypes.data_as(i64), None, _d(rho))
    if nnz < 0:
        raise ValueError(f"vh_rows failed ({nnz})")
    idx = np.zeros(max(nnz, 1), np.int32)
    L.ora_vh_rows(dim, kernel, precision, x.shape[0], _d(x), _d(y), _d(z), _d(h), _d(m),
                  rows.ctypes.data_as(i64), nr, off.ctypes.data_as(i64),
                  idx.ctypes.data_as(C.POINTER(C.c_int32)), _d(rho))
    return off, idx[:nnz], rho
