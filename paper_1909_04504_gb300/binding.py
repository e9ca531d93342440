"""Thin ctypes binding of the C ABI in ``include/sph.h`` (argument marshalling only).

Every step of the particle loop runs in the CUDA library ``_build/libsph_gb300.so``.
There is no CPU fallback: loading fails loudly when the library is missing or no GPU
is present. PyTorch supplies the stream and, optionally, device memory through its
caching allocator.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

QUINTIC, WENDLAND_C2, CUBIC_SPLINE = 0, 1, 2
PREC_FP64, PREC_FP32 = 0, 1
FLUID, WALL = 0, 1
CONTINUITY, SUMMATION, EDAC = 0, 1, 2
WALL_DENSITY, WALL_ADAMI = 0, 1  # sph_wall_bc
INTEGRATOR_KDK, INTEGRATOR_PEC = 0, 1  # sph_integrator
STEP_GRAPH, STEP_PERSISTENT = 0, 1
DIAG_COUNT = 13
DIAG_NAMES = ("t", "dt", "ke", "umax", "px", "py", "pz", "amax", "pairs", "candidates",
              "step", "outside", "wall_pairs")
STATUS = {0: "SPH_OK", 1: "SPH_ERR_INVALID", 2: "SPH_ERR_CUDA", 3: "SPH_ERR_OOM",
          4: "SPH_ERR_NONFINITE", 5: "SPH_ERR_DOMAIN", 6: "SPH_ERR_CAPACITY",
          7: "SPH_ERR_TIMEOUT", 8: "SPH_ERR_STATE"}


class SphError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Domain(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("periodic", C.c_int32 * 3), ("h", C.c_double), ("lo", C.c_double * 3),
                ("hi", C.c_double * 3)]


class ArrayDesc(C.Structure):
    _fields_ = [("name", C.c_char_p), ("role", C.c_int32), ("n", C.c_int64)] + \
               [(k, C.POINTER(C.c_double)) for k in ("x", "y", "z", "u", "v", "w", "rho", "m")]


class Scheme(C.Structure):
    _fields_ = [("density", C.c_int32), ("wall_bc", C.c_int32), ("integrator", C.c_int32),
                ("reserved", C.c_int32), ("rho0", C.c_double),
                ("c0", C.c_double), ("gamma", C.c_double), ("nu", C.c_double),
                ("eta", C.c_double), ("alpha", C.c_double), ("xsph_eps", C.c_double),
                ("g", C.c_double * 3)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = None
EXPORTS = ("sph_create", "sph_destroy", "sph_last_error", "sph_count", "sph_grid",
           "sph_build_neighbors", "sph_get_cells", "sph_get_neighbors", "sph_eval_rhs",
           "sph_step", "sph_step_async", "sph_synchronize", "sph_set_timing", "sph_phase_times",
           "sph_kernels_per_step", "sph_set_groups", "sph_set_step_mode", "sph_set_wait_limit",
           "sph_get_tuning",
           "sph_autotune", "sph_backward", "sph_get", "sph_set", "sph_diagnostics", "sph_history",
           "sph_save_state", "sph_load_state", "sph_save_state_async", "sph_load_state_async",
           "sph_create_batch", "sph_step_batch",
           "sph_step_batch_async",
           "sph_batch_diagnostics")
VH_EXPORTS = ("sph_vh_create", "sph_vh_set", "sph_vh_search", "sph_vh_neighbors",
              "sph_vh_density", "sph_vh_stats", "sph_vh_tree", "sph_vh_set_timing",
              "sph_vh_phase_times", "sph_vh_last_error", "sph_vh_destroy")


class VhParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("kernel", C.c_int32), ("precision", C.c_int32),
                ("leaf_size", C.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first when asked). Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path}")
    L = C.CDLL(path)
    P, d, i32, i64 = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    u32 = C.POINTER(C.c_uint32)
    ctxp = C.c_void_p
    L.sph_create.argtypes = [C.POINTER(Domain), C.POINTER(ArrayDesc), C.c_int32, P, ALLOC_FN,
                             FREE_FN, P, C.POINTER(ctxp)]
    L.sph_destroy.argtypes = [ctxp]
    L.sph_destroy.restype = None
    L.sph_last_error.argtypes = [ctxp]
    L.sph_last_error.restype = C.c_char_p
    L.sph_count.argtypes = [ctxp, C.c_int32, i64]
    L.sph_grid.argtypes = [ctxp, i32, d, i64]
    L.sph_build_neighbors.argtypes = [ctxp]
    L.sph_get_cells.argtypes = [ctxp, u32, u32, i64]
    L.sph_get_neighbors.argtypes = [ctxp, i64, i32, i64]
    L.sph_eval_rhs.argtypes = [ctxp, C.POINTER(Scheme)]
    L.sph_step.argtypes = [ctxp, C.POINTER(Scheme), C.c_double, C.c_int32]
    L.sph_step_async.argtypes = [ctxp, C.POINTER(Scheme), C.c_double, C.c_int32]
    L.sph_synchronize.argtypes = [ctxp]
    L.sph_set_timing.argtypes = [ctxp, C.c_int32]
    L.sph_phase_times.argtypes = [ctxp, C.POINTER(C.c_float)]
    L.sph_kernels_per_step.argtypes = [ctxp, C.POINTER(Scheme), i32]
    L.sph_set_groups.argtypes = [ctxp, C.c_int32]
    L.sph_set_step_mode.argtypes = [ctxp, C.c_int32]
    L.sph_set_wait_limit.argtypes = [ctxp, C.c_uint64]
    L.sph_get_tuning.argtypes = [ctxp, i32, i32, i32]
    L.sph_backward.argtypes = [ctxp, C.POINTER(Scheme), C.c_double, C.c_int32, C.c_int32, d, d, d]
    L.sph_autotune.argtypes = [ctxp, C.POINTER(Scheme), i32]
    L.sph_create_batch.argtypes = [C.POINTER(Domain), C.POINTER(ArrayDesc), i32, C.c_int32, P,
                                   ALLOC_FN, FREE_FN, P, C.POINTER(ctxp)]
    L.sph_step_batch.argtypes = [ctxp, C.POINTER(Scheme), d, C.c_int32]
    L.sph_step_batch_async.argtypes = [ctxp, C.POINTER(Scheme), d, C.c_int32]
    L.sph_batch_diagnostics.argtypes = [ctxp, d]
    L.sph_get.argtypes = [ctxp, C.c_int32, C.c_char_p, d]
    L.sph_set.argtypes = [ctxp, C.c_int32, C.c_char_p, d]
    L.sph_diagnostics.argtypes = [ctxp, d]
    L.sph_history.argtypes = [ctxp, d, C.c_int32, i32]
    L.sph_save_state.argtypes = [ctxp, P, C.POINTER(C.c_size_t)]
    L.sph_load_state.argtypes = [ctxp, P, C.c_size_t]
    L.sph_save_state_async.argtypes = [ctxp, P, C.POINTER(C.c_size_t)]
    L.sph_load_state_async.argtypes = [ctxp, P, C.c_size_t]
    for name in EXPORTS:
        if name not in ("sph_destroy", "sph_last_error"):
            getattr(L, name).restype = C.c_int
    L.sph_vh_create.argtypes = [C.POINTER(VhParams), C.c_int64, P, ALLOC_FN, FREE_FN, P,
                                C.POINTER(ctxp)]
    L.sph_vh_set.argtypes = [ctxp, C.c_int64, d, d, d, d, d]
    L.sph_vh_search.argtypes = [ctxp]
    L.sph_vh_neighbors.argtypes = [ctxp, i64, i32, C.c_int64, i64]
    L.sph_vh_density.argtypes = [ctxp, d]
    L.sph_vh_stats.argtypes = [ctxp, i64]
    L.sph_vh_tree.argtypes = [ctxp, C.c_int64, i32, i32, i32, i32, d, d, d, i32]
    L.sph_vh_set_timing.argtypes = [ctxp, C.c_int32]
    L.sph_vh_phase_times.argtypes = [ctxp, C.POINTER(C.c_float)]
    L.sph_vh_last_error.argtypes = [ctxp]
    L.sph_vh_last_error.restype = C.c_char_p
    L.sph_vh_destroy.argtypes = [ctxp]
    L.sph_vh_destroy.restype = None
    for name in VH_EXPORTS:
        if name not in ("sph_vh_destroy", "sph_vh_last_error"):
            getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _dptr(a: Optional[np.ndarray]):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def make_scheme(density=CONTINUITY, rho0=1.0, c0=10.0, gamma=7.0, nu=0.0, eta=0.01, alpha=0.0,
                xsph_eps=0.0, g=(0.0, 0.0, 0.0), wall_bc=WALL_DENSITY,
                integrator=INTEGRATOR_KDK) -> Scheme:
    s = Scheme()
    s.density, s.rho0, s.c0, s.gamma = int(density), rho0, c0, gamma
    s.wall_bc = int(wall_bc)
    s.integrator = int(integrator)
    s.nu, s.eta, s.alpha, s.xsph_eps = nu, eta, alpha, xsph_eps
    for k in range(3):
        s.g[k] = float(g[k])
    return s


def scheme_of(wl, **over) -> Scheme:
    """Scheme from an object with the workload attributes (rho0, c0, gamma, nu, ...)."""
    kw = dict(density=wl.density, rho0=wl.rho0, c0=wl.c0, gamma=wl.gamma, nu=wl.nu, eta=wl.eta,
              alpha=wl.alpha, xsph_eps=wl.xsph_eps, g=wl.g,
              wall_bc=getattr(wl, "wall_bc", WALL_DENSITY),
              integrator=getattr(wl, "integrator", INTEGRATOR_KDK))
    kw.update(over)
    return make_scheme(**kw)


class _TorchAllocator:
    """Routes the library's device allocations through PyTorch's caching allocator."""

    def __init__(self, device: int, stream):
        import torch
        self._torch = torch
        self._device = device
        self._stream = stream
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, user):
        try:
            return int(self._torch.cuda.caching_allocator_alloc(int(nbytes), self._device,
                                                                 self._stream))
        except Exception:  # noqa: BLE001 - reported to the library as NULL
            return None

    def _free(self, ptr, user):
        if ptr:
            self._torch.cuda.caching_allocator_delete(ptr)


class Simulation:
    """One WCSPH problem resident on the GPU (a ``sph_ctx``)."""

    def __init__(self, dim: int, kernel: int, precision: int, h: float, lo: Sequence[float],
                 hi: Sequence[float], periodic: Sequence[int], arrays: Sequence[dict],
                 stream=None, torch_alloc: bool = True):
        self._L = load()
        dom = Domain()
        dom.dim, dom.kernel, dom.precision, dom.h = dim, kernel, precision, h
        for k in range(3):
            dom.periodic[k] = int(periodic[k])
            dom.lo[k] = float(lo[k])
            dom.hi[k] = float(hi[k])
        self.dim = dim
        self._keep = []
        descs = (ArrayDesc * len(arrays))()
        for a, arr in enumerate(arrays):
            dsc = descs[a]
            name = str(arr.get("name", f"array{a}")).encode()
            self._keep.append(name)
            dsc.name = name
            dsc.role = int(arr.get("role", FLUID))
            x = _f64(arr["x"])
            dsc.n = x.shape[0]
            for k in ("x", "y", "z", "u", "v", "w", "rho", "m"):
                v = arr.get(k)
                if v is None:
                    setattr(dsc, k, None)
                    continue
                v = _f64(v)
                if v.shape[0] != dsc.n:
                    raise ValueError(f"array {a}: {k} has {v.shape[0]} entries, expected {dsc.n}")
                self._keep.append(v)
                setattr(dsc, k, _dptr(v))
        self._stream_obj = None
        stream_handle = None
        self._alloc = None
        alloc_fn, free_fn = ALLOC_FN(), FREE_FN()
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the WCSPH library runs on the GPU only")
        if stream is None:
            self._stream_obj = torch.cuda.Stream()
            stream_handle = self._stream_obj.cuda_stream
        else:
            stream_handle = int(getattr(stream, "cuda_stream", stream))
        if torch_alloc:
            dev = torch.cuda.current_device()
            self._alloc = _TorchAllocator(dev, stream_handle)
            alloc_fn, free_fn = self._alloc.alloc, self._alloc.free
        ctx = C.c_void_p()
        st = self._L.sph_create(C.byref(dom), descs, len(arrays), C.c_void_p(stream_handle),
                                alloc_fn, free_fn, None, C.byref(ctx))
        self._keep = []
        if st != 0:
            raise SphError(st, self._L.sph_last_error(None).decode())
        self._ctx = ctx
        self.n = self.count(-1)

    @classmethod
    def from_workload(cls, wl, precision: Optional[int] = None, **kw) -> "Simulation":
        """A context holding the workload's arrays (and the pressure of the EDAC form where
        an array carries one)."""
        arrays = [dict(name=a.name, role=a.role, x=a.x, y=a.y, z=a.z, u=a.u, v=a.v, w=a.w,
                       rho=a.rho, m=a.m) for a in wl.arrays]
        sim = cls(wl.dim, wl.kernel, wl.precision if precision is None else precision, wl.h,
                  wl.lo, wl.hi, wl.periodic, arrays, **kw)
        for k, a in enumerate(wl.arrays):
            if getattr(a, "p", None) is not None:
                sim.set("p", a.p, array=k)
        return sim

    # ---------------------------------------------------------------- plumbing
    def _check(self, st: int):
        if st != 0:
            raise SphError(st, self._L.sph_last_error(self._ctx).decode())

    @property
    def stream(self):
        return self._stream_obj

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.sph_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- the C ABI
    def count(self, array: int = -1) -> int:
        n = C.c_int64()
        self._check(self._L.sph_count(self._ctx, array, C.byref(n)))
        return n.value

    def grid(self):
        nc = (C.c_int32 * 3)()
        cs = (C.c_double * 3)()
        total = C.c_int64()
        self._check(self._L.sph_grid(self._ctx, nc, cs, C.byref(total)))
        return list(nc), list(cs), total.value

    def build_neighbors(self):
        self._check(self._L.sph_build_neighbors(self._ctx))

    def cells(self):
        _, _, ncells = self.grid()
        cell_of = np.zeros(self.n, np.uint32)
        off = np.zeros(ncells + 1, np.uint32)
        order = np.zeros(self.n, np.int64)
        self._check(self._L.sph_get_cells(self._ctx, cell_of.ctypes.data_as(C.POINTER(C.c_uint32)),
                                          off.ctypes.data_as(C.POINTER(C.c_uint32)),
                                          order.ctypes.data_as(C.POINTER(C.c_int64))))
        return cell_of, off, order

    def neighbors(self):
        off = np.zeros(self.n + 1, np.int64)
        nnz = C.c_int64(0)
        i64 = C.POINTER(C.c_int64)
        self._check(self._L.sph_get_neighbors(self._ctx, off.ctypes.data_as(i64), None,
                                              C.byref(nnz)))
        idx = np.zeros(max(nnz.value, 1), np.int32)
        self._check(self._L.sph_get_neighbors(self._ctx, off.ctypes.data_as(i64),
                                              idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                              C.byref(nnz)))
        return off, idx[:nnz.value]

    def eval_rhs(self, scheme: Scheme):
        self._check(self._L.sph_eval_rhs(self._ctx, C.byref(scheme)))

    def step(self, scheme: Scheme, dt: float, nsteps: int = 1):
        self._check(self._L.sph_step(self._ctx, C.byref(scheme), float(dt), int(nsteps)))

    def step_async(self, scheme: Scheme, dt: float, nsteps: int = 1):
        self._check(self._L.sph_step_async(self._ctx, C.byref(scheme), float(dt), int(nsteps)))

    def synchronize(self):
        self._check(self._L.sph_synchronize(self._ctx))

    def set_timing(self, enable: bool = True):
        self._check(self._L.sph_set_timing(self._ctx, int(bool(enable))))

    PHASES = ("keys", "sort", "reorder", "cells", "density", "momentum")

    def phase_times(self) -> dict:
        out = (C.c_float * 6)()
        self._check(self._L.sph_phase_times(self._ctx, out))
        return dict(zip(self.PHASES, [float(v) for v in out]))

    def kernels_per_step(self, scheme: Scheme) -> int:
        n = C.c_int32()
        self._check(self._L.sph_kernels_per_step(self._ctx, C.byref(scheme), C.byref(n)))
        return n.value

    def set_groups(self, momentum_lanes: int):
        self._check(self._L.sph_set_groups(self._ctx, int(momentum_lanes)))

    def set_step_mode(self, mode: int):
        """STEP_GRAPH: per-phase kernels in a CUDA graph; STEP_PERSISTENT: one cooperative
        launch per step."""
        self._check(self._L.sph_set_step_mode(self._ctx, int(mode)))

    def tuning(self) -> tuple:
        """(momentum lanes per destination, step mode, density lanes per destination)."""
        lanes, mode, dl = C.c_int32(), C.c_int32(), C.c_int32()
        self._check(self._L.sph_get_tuning(self._ctx, C.byref(lanes), C.byref(mode), C.byref(dl)))
        return int(lanes.value), int(mode.value), int(dl.value)

    def step_mode(self) -> int:
        return self.tuning()[1]

    def set_wait_limit(self, ns: int):
        self._check(self._L.sph_set_wait_limit(self._ctx, int(ns)))

    def autotune(self, scheme: Optional[Scheme]) -> int:
        out = C.c_int32()
        self._check(self._L.sph_autotune(self._ctx, None if scheme is None else C.byref(scheme),
                                         C.byref(out)))
        return int(out.value)

    def backward(self, scheme: Scheme, dt: float, K: int, ckpt_every: int = 0):
        """Run K steps and return (dKE/du0 [dim, n] in original order, dKE/dnu, dKE/dalpha)."""
        out = np.zeros((self.dim, self.n))
        gnu, gal = C.c_double(), C.c_double()
        self._check(self._L.sph_backward(self._ctx, C.byref(scheme), float(dt), int(K),
                                         int(ckpt_every), _dptr(out), C.byref(gnu), C.byref(gal)))
        return out, gnu.value, gal.value

    def get(self, prop: str, array: int = -1) -> np.ndarray:
        out = np.zeros(self.count(array))
        self._check(self._L.sph_get(self._ctx, array, prop.encode(), _dptr(out)))
        return out

    def set(self, prop: str, values, array: int = -1):
        v = _f64(values)
        if v.shape[0] != self.count(array):
            raise ValueError("wrong length")
        self._check(self._L.sph_set(self._ctx, array, prop.encode(), _dptr(v)))

    def state(self) -> dict:
        return {k: self.get(k) for k in ("x", "y", "z", "u", "v", "w", "rho", "m", "p")}

    def rates(self) -> dict:
        return {k: self.get(k) for k in ("arho", "ax", "ay", "az", "xsx", "xsy", "xsz")}

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(DIAG_COUNT)
        self._check(self._L.sph_diagnostics(self._ctx, _dptr(out)))
        return out

    def history(self, max_records: int = 65536) -> np.ndarray:
        out = np.zeros((max_records, DIAG_COUNT))
        n = C.c_int32()
        self._check(self._L.sph_history(self._ctx, _dptr(out), max_records, C.byref(n)))
        return out[:n.value]

    def save_state(self) -> bytes:
        size = C.c_size_t(0)
        self._check(self._L.sph_save_state(self._ctx, None, C.byref(size)))
        buf = C.create_string_buffer(size.value)
        self._check(self._L.sph_save_state(self._ctx, buf, C.byref(size)))
        return buf.raw

    def state_bytes(self) -> int:
        size = C.c_size_t(0)
        self._check(self._L.sph_save_state(self._ctx, None, C.byref(size)))
        return int(size.value)

    def save_state_into(self, buf: np.ndarray) -> int:
        """Write the state into a contiguous uint8 array in place (a pinned host array is
        filled by the device copies without staging); returns the bytes written."""
        assert buf.dtype == np.uint8 and buf.flags.c_contiguous
        size = C.c_size_t(buf.nbytes)
        self._check(self._L.sph_save_state(self._ctx, C.c_void_p(buf.ctypes.data), C.byref(size)))
        return int(size.value)

    def save_state_into_async(self, buf: np.ndarray) -> int:
        """As save_state_into, but only enqueued on the context stream: buf (pinned, for the
        copies to overlap other work) holds the state once synchronize() returns."""
        assert buf.dtype == np.uint8 and buf.flags.c_contiguous
        size = C.c_size_t(buf.nbytes)
        self._check(self._L.sph_save_state_async(self._ctx, C.c_void_p(buf.ctypes.data),
                                                 C.byref(size)))
        return int(size.value)

    def load_state_async(self, buf: np.ndarray):
        """As load_state from a contiguous uint8 array, but only enqueued on the context
        stream: buf must stay unchanged until synchronize() returns."""
        assert buf.dtype == np.uint8 and buf.flags.c_contiguous
        self._check(self._L.sph_load_state_async(self._ctx, C.c_void_p(buf.ctypes.data), buf.nbytes))

    def load_state(self, blob):
        """Restore a state from bytes or from a contiguous uint8 numpy array (read in place,
        so a pinned host array is copied to the device without staging)."""
        if isinstance(blob, np.ndarray):
            assert blob.dtype == np.uint8 and blob.flags.c_contiguous
            self._check(self._L.sph_load_state(self._ctx, C.c_void_p(blob.ctypes.data),
                                               blob.nbytes))
            return
        buf = C.create_string_buffer(blob, len(blob))
        self._check(self._L.sph_load_state(self._ctx, buf, len(blob)))


def _domain_of(wl, precision=None) -> Domain:
    dom = Domain()
    dom.dim, dom.kernel, dom.h = wl.dim, wl.kernel, wl.h
    dom.precision = wl.precision if precision is None else precision
    for k in range(3):
        dom.periodic[k] = int(wl.periodic[k])
        dom.lo[k] = float(wl.lo[k])
        dom.hi[k] = float(wl.hi[k])
    return dom


class BatchSimulation(Simulation):
    """Many independent problems (a batch context) advanced in the same launches."""

    def __init__(self, workloads: Sequence, precision: Optional[int] = None, stream=None,
                 torch_alloc: bool = True):
        import torch
        self._L = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the WCSPH library runs on the GPU only")
        self.workloads = list(workloads)
        self.ninst = len(self.workloads)
        self.dim = self.workloads[0].dim
        doms = (Domain * self.ninst)(*[_domain_of(w, precision) for w in self.workloads])
        flat = [a for w in self.workloads for a in w.arrays]
        per = (C.c_int32 * self.ninst)(*[len(w.arrays) for w in self.workloads])
        descs = (ArrayDesc * len(flat))()
        keep = []
        for a, arr in enumerate(flat):
            dsc = descs[a]
            name = arr.name.encode()
            keep.append(name)
            dsc.name, dsc.role, dsc.n = name, int(arr.role), int(arr.n)
            for k in ("x", "y", "z", "u", "v", "w", "rho", "m"):
                v = _f64(getattr(arr, k))
                keep.append(v)
                setattr(dsc, k, _dptr(v))
        self._stream_obj = torch.cuda.Stream() if stream is None else None
        handle = self._stream_obj.cuda_stream if stream is None else int(getattr(stream, "cuda_stream", stream))
        self._alloc = None
        alloc_fn, free_fn = ALLOC_FN(), FREE_FN()
        if torch_alloc:
            self._alloc = _TorchAllocator(torch.cuda.current_device(), handle)
            alloc_fn, free_fn = self._alloc.alloc, self._alloc.free
        ctx = C.c_void_p()
        st = self._L.sph_create_batch(doms, descs, per, self.ninst, C.c_void_p(handle), alloc_fn,
                                      free_fn, None, C.byref(ctx))
        if st != 0:
            raise SphError(st, self._L.sph_last_error(None).decode())
        self._ctx = ctx
        self.n = self.count(-1)
        sizes = [sum(a.n for a in w.arrays) for w in self.workloads]
        self.bounds = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        if any(getattr(a, "p", None) is not None for w in self.workloads for a in w.arrays):
            self.set("p", np.concatenate([w.concat("p") for w in self.workloads]))

    def step_batch(self, schemes: Sequence[Scheme], dts: Sequence[float], nsteps: int = 1):
        arr = (Scheme * self.ninst)(*schemes)
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(self._L.sph_step_batch(self._ctx, arr, _dptr(d), int(nsteps)))

    def step_batch_async(self, schemes: Sequence[Scheme], dts: Sequence[float], nsteps: int = 1):
        arr = (Scheme * self.ninst)(*schemes)
        d = np.ascontiguousarray(dts, dtype=np.float64)
        self._check(self._L.sph_step_batch_async(self._ctx, arr, _dptr(d), int(nsteps)))

    def batch_diagnostics(self) -> np.ndarray:
        out = np.zeros((self.ninst, DIAG_COUNT))
        self._check(self._L.sph_batch_diagnostics(self._ctx, _dptr(out)))
        return out

    def instance_state(self, k: int) -> dict:
        st = self.state()
        b, e = self.bounds[k], self.bounds[k + 1]
        return {key: v[b:e] for key, v in st.items()}


def final_kinetic_energy(sim: "Simulation", scheme: Scheme, dt: float, K: int, u0, nu, alpha=None,
                         ckpt_every: int = 0):
    """KE after K steps as a differentiable function of the initial fluid velocities ``u0``
    (torch tensor [dim, n], original order) and the viscosities ``nu`` (and ``alpha``), via a
    torch.autograd.Function whose backward is the hand-written adjoint (sph_backward).
    Sets the simulation's velocities to u0 and leaves it K steps later."""
    import torch

    class _FinalKE(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u0_t, nu_t, alpha_t):
            sch = Scheme.from_buffer_copy(scheme)
            sch.nu = float(nu_t)
            sch.alpha = float(alpha_t)
            u = u0_t.detach().to("cpu", torch.float64).numpy()
            for k, name in enumerate(("u", "v", "w")[:sim.dim]):
                sim.set(name, u[k])
            gu, gnu, gal = sim.backward(sch, dt, K, ckpt_every)
            ke = float(sim.diagnostics()[2])
            ctx.save_for_backward(torch.as_tensor(gu, dtype=u0_t.dtype, device=u0_t.device),
                                  torch.tensor(gnu, dtype=nu_t.dtype, device=nu_t.device),
                                  torch.tensor(gal, dtype=alpha_t.dtype, device=alpha_t.device))
            return torch.tensor(ke, dtype=torch.float64, device=u0_t.device)

        @staticmethod
        def backward(ctx, g):
            gu, gnu, gal = ctx.saved_tensors
            return g * gu, g * gnu, g * gal

    if alpha is None:
        import torch as _t
        alpha = _t.tensor(float(scheme.alpha), dtype=_t.float64)
    return _FinalKE.apply(u0, nu, alpha)


class VariableHSearch:
    """Neighbour search and density with a per-particle smoothing length through an octree
    (a ``sph_vh`` context of ``include/sph_vh.h``)."""

    STATS = ("nodes", "leaves", "depth", "candidates", "pairs", "max_count", "slots",
             "query_runs")

    def __init__(self, dim: int, kernel: int, precision: int, capacity: int,
                 leaf_size: int = 32, stream=None, torch_alloc: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the search runs on the GPU only")
        self._L = load()
        prm = VhParams()
        prm.dim, prm.kernel, prm.precision, prm.leaf_size = dim, kernel, precision, leaf_size
        self.dim = dim
        self._stream_obj = None
        if stream is None:
            self._stream_obj = torch.cuda.Stream()
            handle = self._stream_obj.cuda_stream
        else:
            handle = int(getattr(stream, "cuda_stream", stream))
        self.stream_handle = handle
        self._alloc = None
        alloc_fn, free_fn = ALLOC_FN(), FREE_FN()
        if torch_alloc:
            self._alloc = _TorchAllocator(torch.cuda.current_device(), handle)
            alloc_fn, free_fn = self._alloc.alloc, self._alloc.free
        ctx = C.c_void_p()
        st = self._L.sph_vh_create(C.byref(prm), int(capacity), C.c_void_p(handle), alloc_fn,
                                   free_fn, None, C.byref(ctx))
        if st != 0:
            raise SphError(st, self._L.sph_vh_last_error(None).decode())
        self._ctx = ctx
        self.n = 0

    def _check(self, st: int):
        if st != 0:
            raise SphError(st, self._L.sph_vh_last_error(self._ctx).decode())

    def set(self, x, y, z, h, m):
        x, y, h, m = _f64(x), _f64(y), _f64(h), _f64(m)
        z = _f64(z) if z is not None else None
        self._check(self._L.sph_vh_set(self._ctx, x.shape[0], _dptr(x), _dptr(y), _dptr(z),
                                       _dptr(h), _dptr(m)))
        self.n = x.shape[0]

    def search(self):
        self._check(self._L.sph_vh_search(self._ctx))

    def neighbors(self):
        """CSR (offsets int64[n+1], idx int32[nnz]) in the caller's order, rows unsorted."""
        off = np.zeros(self.n + 1, np.int64)
        nnz = C.c_int64()
        i64 = C.POINTER(C.c_int64)
        self._check(self._L.sph_vh_neighbors(self._ctx, off.ctypes.data_as(i64), None, 0,
                                             C.byref(nnz)))
        idx = np.zeros(max(nnz.value, 1), np.int32)
        self._check(self._L.sph_vh_neighbors(self._ctx, off.ctypes.data_as(i64),
                                             idx.ctypes.data_as(C.POINTER(C.c_int32)),
                                             idx.shape[0], C.byref(nnz)))
        return off, idx[:nnz.value]

    def density(self) -> np.ndarray:
        rho = np.zeros(self.n)
        self._check(self._L.sph_vh_density(self._ctx, _dptr(rho)))
        return rho

    def stats(self) -> dict:
        out = np.zeros(8, np.int64)
        self._check(self._L.sph_vh_stats(self._ctx, out.ctypes.data_as(C.POINTER(C.c_int64))))
        return dict(zip(self.STATS, (int(v) for v in out)))

    def tree(self) -> dict:
        nn = self.stats()["nodes"]
        i32p = C.POINTER(C.c_int32)
        t = {k: np.zeros(max(nn, 1), np.int32) for k in ("start", "end", "child", "nchild")}
        lo, hi = np.zeros((max(nn, 1), 3)), np.zeros((max(nn, 1), 3))
        hmax = np.zeros(max(nn, 1))
        perm = np.zeros(max(self.n, 1), np.int32)
        self._check(self._L.sph_vh_tree(self._ctx, nn, *(t[k].ctypes.data_as(i32p)
                                                          for k in ("start", "end", "child", "nchild")),
                                        _dptr(lo), _dptr(hi), _dptr(hmax), perm.ctypes.data_as(i32p)))
        out = {k: v[:nn] for k, v in t.items()}
        out.update(lo=lo[:nn], hi=hi[:nn], hmax=hmax[:nn], perm=perm[:self.n])
        return out

    def set_timing(self, on: bool):
        self._check(self._L.sph_vh_set_timing(self._ctx, 1 if on else 0))

    def phase_times(self) -> dict:
        """ms of the last timed search: build (root box to node boxes) and query."""
        out = (C.c_float * 2)()
        self._check(self._L.sph_vh_phase_times(self._ctx, out))
        return {"build": float(out[0]), "query": float(out[1])}

    def close(self):
        if getattr(self, "_ctx", None):
            self._L.sph_vh_destroy(self._ctx)
            self._ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
