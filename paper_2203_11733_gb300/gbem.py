"""Python binding of libgbem (include/gbem.h): argument marshalling only.

Every step of the extraction runs in the library's CUDA kernels; this module
converts Python/numpy/torch arguments to plain pointers and sizes and raises
on error statuses.  Device memory for handles comes from PyTorch's caching
allocator through the ABI's allocator callback.  There is no CPU fallback:
if ``libgbem.so`` has not been built, importing the library fails loudly.

Names follow the C ABI: ``gbem_create``, ``gbem_mesh``, ``gbem_assemble``,
``gbem_factor``, ``gbem_solve``, ``gbem_capacitance`` ...; the classes below
are small conveniences over them.
"""
from __future__ import annotations

import atexit
import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

GBEM_OK = 0
STATUS = {
    0: "GBEM_OK", -1: "GBEM_ERR_ARG", -2: "GBEM_ERR_OOM", -3: "GBEM_ERR_CUDA",
    -4: "GBEM_ERR_NOT_SPD", -5: "GBEM_ERR_TIMEOUT", -6: "GBEM_ERR_NOCONV", -7: "GBEM_ERR_MESH",
    -8: "GBEM_ERR_STATE", -9: "GBEM_ERR_NODEV",
}
GBEM_FP64 = 0
GBEM_MIXED = 1
# gbem_unit_rate, in enum order
UNIT_RATE_NAMES = ("dfma", "ffma", "mufu_rsqrt", "dsqrt", "dlog", "datan", "drsqrt")
EPS0 = 8.8541878128e-12


class GbemError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Box(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("conductor", ctypes.c_int32)]


class _MeshParams(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("ratio", ctypes.c_double), ("h_min", ctypes.c_double)]


class _Tuning(ctypes.Structure):
    _fields_ = [("q_near_fp64", ctypes.c_double), ("q_near_mixed", ctypes.c_double),
                ("ir_tol", ctypes.c_double), ("ir_max_iter", ctypes.c_int), ("nb", ctypes.c_int)]


class _PartitionParams(ctypes.Structure):
    _fields_ = [("main_conductor", ctypes.c_int32), ("p1", ctypes.c_double), ("p2", ctypes.c_double),
                ("p3", ctypes.c_double), ("p5", ctypes.c_double), ("h_max", ctypes.c_double),
                ("has_enclosure", ctypes.c_int), ("encl_lo", ctypes.c_double * 3),
                ("encl_hi", ctypes.c_double * 3), ("encl_conductor", ctypes.c_int32)]


class ResultInfo(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("n_panels", ctypes.c_int),
                ("n_cond", ctypes.c_int), ("residual", ctypes.c_double), ("submit_s", ctypes.c_double),
                ("start_s", ctypes.c_double), ("done_s", ctypes.c_double), ("c_offset", ctypes.c_longlong)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()
_live_contexts = weakref.WeakSet()


@atexit.register
def _close_all():
    # release handles while the allocator (PyTorch) is still alive
    for c in list(_live_contexts):
        try:
            c.close()
        except Exception:
            pass

# symbol -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "gbem_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_size_t, ALLOC_FN, FREE_FN, _P]),
    "gbem_destroy": (None, [_P]),
    "gbem_last_error": (ctypes.c_char_p, [_P]),
    "gbem_set_tuning": (ctypes.c_int, [_P, ctypes.POINTER(_Tuning)]),
    "gbem_bytes_in_use": (ctypes.c_size_t, [_P]),
    "gbem_mesh": (ctypes.c_int, [_P, ctypes.POINTER(_Box), ctypes.c_int, ctypes.POINTER(_MeshParams),
                                 ctypes.POINTER(_P)]),
    "gbem_mesh_graded": (ctypes.c_int, [_P, ctypes.POINTER(_Box), ctypes.c_int, ctypes.POINTER(_PartitionParams),
                                        ctypes.POINTER(_P)]),
    "gbem_mesh_from_panels": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, ctypes.POINTER(_P)]),
    "gbem_mesh_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gbem_mesh_panels": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "gbem_mesh_refine": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, _P, _P]),
    "gbem_mesh_from_triangles": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "gbem_mesh_triangles": (ctypes.c_int, [_P, _P, _P]),
    "gbem_stack_mesh": (ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P]),
    "gbem_stack_info": (ctypes.c_int, [_P, _P, _P, _P]),
    "gbem_stack_panels": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "gbem_stack_assemble": (ctypes.c_int, [_P, ctypes.c_int, _P]),
    "gbem_stack_iterations": (ctypes.c_int, [_P, _P]),
    "gbem_stack_system": (ctypes.c_int, [_P, _P, _P]),
    "gbem_stack_capacitance": (ctypes.c_int, [_P, _P, _P, _P]),
    "gbem_stack_destroy": (None, [_P]),
    "gbem_mesh_destroy": (None, [_P]),
    "gbem_assemble": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "gbem_factor": (ctypes.c_int, [_P, _P]),
    "gbem_solve": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int), _P]),
    "gbem_capacitance": (ctypes.c_int, [_P, _P, ctypes.c_double, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "gbem_matrix_download": (ctypes.c_int, [_P, _P]),
    "gbem_matrix_status": (ctypes.c_int, [_P]),
    "gbem_matrix_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), _P]),
    "gbem_matrix_class_counts": (ctypes.c_int, [_P, _P]),
    "gbem_selftest_wait": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, _P]),
    "gbem_unit_rates": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "gbem_matrix_destroy": (None, [_P]),
    "gbem_set_timing": (ctypes.c_int, [_P, ctypes.c_int]),
    "gbem_get_stats": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "gbem_get_kernel_stats": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "gbem_batch_create": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.POINTER(_P)]),
    "gbem_batch_run": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P]),
    "gbem_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong), _P]),
    "gbem_batch_destroy": (None, [_P]),
    "gbem_batch_create_grouped": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                                 ctypes.POINTER(_P)]),
    "gbem_batch_config": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "gbem_batch_autotune": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(_P),
                                           _P]),
    "gbem_server_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_size_t, ctypes.c_int, ctypes.c_int,
                                          ctypes.POINTER(_P)]),
    "gbem_server_submit": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.POINTER(_Box), ctypes.c_int,
                                          ctypes.POINTER(_MeshParams), ctypes.c_double,
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "gbem_server_poll": (ctypes.c_int, [_P, ctypes.POINTER(ResultInfo), _P, ctypes.c_longlong, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "gbem_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "gbem_server_destroy": (None, [_P]),
}


class Stats(ctypes.Structure):
    """gbem_stats: per-phase device time and calls, kernels launched."""
    _fields_ = [("ms", ctypes.c_double * 5), ("calls", ctypes.c_longlong * 5), ("launches", ctypes.c_longlong)]


KERNELS = ["assemble", "factor", "sweep", "residual"]


class KernelStats(ctypes.Structure):
    """gbem_kernel_stats: per traced kernel, device time, launches and the
    algorithmic bytes and flops of those launches."""
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_longlong * 4),
                ("bytes", ctypes.c_double * 4), ("flops", ctypes.c_double * 4)]


def set_timing(ctx, level: int):
    """0 off, 1 phase events, 2 phase and per-kernel events."""
    ctx.check(ctx.lib.gbem_set_timing(ctx.h, int(level)))


def get_stats(ctx, reset: bool = False) -> dict:
    s = Stats()
    ctx.check(ctx.lib.gbem_get_stats(ctx.h, ctypes.byref(s), 1 if reset else 0))
    return {"ms": list(s.ms), "calls": list(s.calls), "launches": s.launches}


def get_kernel_stats(ctx, reset: bool = False) -> dict:
    s = KernelStats()
    ctx.check(ctx.lib.gbem_get_kernel_stats(ctx.h, ctypes.byref(s), 1 if reset else 0))
    return {k: {"ms": s.ms[i], "launches": s.launches[i], "bytes": s.bytes[i], "flops": s.flops[i]}
            for i, k in enumerate(KERNELS)}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgbem.so (raises if it is missing and building is not asked for)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(
                    f"libgbem.so not built ({path}); run __graft_entry__.build() or "
                    "python paper_2203_11733_gb300/build.py")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def exported_symbols():
    return list(_SIGS)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A library context on one CUDA device (or device=-1: host-only, meshing
    only).  ``torch_alloc`` routes device memory through PyTorch's caching
    allocator; otherwise the library uses cudaMalloc."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, torch_alloc: bool = True, refuse=None):
        """``refuse`` (tests of the allocation-failure path): a callable
        (call index, bytes) -> bool; when it returns True the allocator
        callback hands the library a NULL pointer instead of memory."""
        self.lib = load()
        self.device = device
        self._cb = None
        self.h = None
        self._children = weakref.WeakSet()
        self.alloc_calls = 0
        alloc, free = ALLOC_FN(), FREE_FN()
        if device >= 0 and torch_alloc:
            import torch

            def _alloc(nbytes, stream, user):
                k = self.alloc_calls
                self.alloc_calls += 1
                if refuse is not None and refuse(k, int(nbytes)):
                    return None
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), device, stream or 0)
                except Exception:   # refusal is reported through a NULL pointer
                    return None

            def _free(ptr, nbytes, stream, user):
                torch.cuda.caching_allocator_delete(ptr)

            alloc, free = ALLOC_FN(_alloc), FREE_FN(_free)
            self._cb = (alloc, free)
        h = ctypes.c_void_p()
        st = self.lib.gbem_create(ctypes.byref(h), int(device), int(hbm_budget), alloc, free, None)
        if st != GBEM_OK:
            raise GbemError(st, "gbem_create failed")
        self.h = h
        _live_contexts.add(self)

    def check(self, st: int):
        if st != GBEM_OK:
            msg = self.lib.gbem_last_error(self.h)
            raise GbemError(st, msg.decode() if msg else "")

    def set_tuning(self, q_near_fp64=0.0, q_near_mixed=0.0, ir_tol=0.0, ir_max_iter=0, nb=0):
        t = _Tuning(q_near_fp64, q_near_mixed, ir_tol, ir_max_iter, nb)
        self.check(self.lib.gbem_set_tuning(self.h, ctypes.byref(t)))


    def selftest_wait(self, set_flag: bool, limit_ms: float = 50.0, stream=None) -> int:
        """gbem_selftest_wait: the status of one bounded device wait for a flag
        that is set (GBEM_OK) or withheld (GBEM_ERR_TIMEOUT)."""
        return int(self.lib.gbem_selftest_wait(self.h, 1 if set_flag else 0, float(limit_ms),
                                               _stream_handle(stream)))

    def unit_rates(self, stream=None) -> dict:
        """gbem_unit_rates: operations per second of the units that bound the
        assembly, measured on this context's GPU."""
        out = (ctypes.c_double * len(UNIT_RATE_NAMES))()
        self.check(self.lib.gbem_unit_rates(self.h, out, len(UNIT_RATE_NAMES), _stream_handle(stream)))
        return {k: float(out[i]) for i, k in enumerate(UNIT_RATE_NAMES)}

    def bytes_in_use(self) -> int:
        return int(self.lib.gbem_bytes_in_use(self.h))

    def mesh(self, boxes, params) -> "Mesh":
        return gbem_mesh(self, boxes, params)

    def mesh_from_panels(self, axis, geo, cond) -> "Mesh":
        return gbem_mesh_from_panels(self, axis, geo, cond)

    def mesh_from_triangles(self, tri, cond) -> "Mesh":
        """gbem_mesh_from_triangles: tri float64[n, 9] (vertices), cond int32[n]."""
        t = np.ascontiguousarray(tri, dtype=np.float64).reshape(-1, 9)
        c = np.ascontiguousarray(cond, dtype=np.int32)
        if len(c) != len(t):
            raise ValueError("one conductor id per triangle")
        out = _P()
        self.check(self.lib.gbem_mesh_from_triangles(self.h, len(t), _ptr(t), _ptr(c), ctypes.byref(out)))
        return Mesh(self, out)

    def close(self):
        """Destroy the context; matrices and meshes made from it go first."""
        if getattr(self, "h", None):
            kids = list(self._children)
            for k in kids:
                if isinstance(k, (Matrix, Batch)):
                    k.close()
            for k in kids:
                k.close()
            self.lib.gbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    def __init__(self, ctx: Context, handle):
        self.ctx, self.h = ctx, handle
        ctx._children.add(self)
        n, nc = ctypes.c_int(), ctypes.c_int()
        ctx.check(ctx.lib.gbem_mesh_info(handle, ctypes.byref(n), ctypes.byref(nc)))
        self.n, self.n_cond = n.value, nc.value

    def panels(self):
        """(axis int8[n], geo float64[n,5], cond int32[n], conductor ids int32[n_c])"""
        axis = np.empty(self.n, np.int8)
        geo = np.empty((self.n, 5), np.float64)
        cond = np.empty(self.n, np.int32)
        ids = np.empty(self.n_cond, np.int32)
        self.ctx.check(self.ctx.lib.gbem_mesh_panels(self.h, _ptr(axis), _ptr(geo), _ptr(cond), _ptr(ids)))
        return axis, geo, cond, ids

    def assemble(self, precision=GBEM_FP64, stream=None) -> "Matrix":
        return gbem_assemble(self, precision, stream)

    def triangles(self):
        """(tri float64[n, 9], conductor ids int32[n]) of a triangle mesh."""
        t = np.empty((self.n, 9), np.float64)
        c = np.empty(self.n, np.int32)
        self.ctx.check(self.ctx.lib.gbem_mesh_triangles(self.h, _ptr(t), _ptr(c)))
        return t, c

    def close(self):
        if getattr(self, "h", None):
            if self.ctx.h is not None:
                self.ctx.lib.gbem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Matrix:
    def __init__(self, mesh: Mesh, handle, precision):
        self.mesh, self.ctx, self.h, self.precision = mesh, mesh.ctx, handle, precision
        self.n = mesh.n
        mesh.ctx._children.add(self)

    def factor(self, stream=None):
        gbem_factor(self, stream)

    def solve(self, B, X=None, stream=None):
        return gbem_solve(self, B, X, stream)

    def capacitance(self, eps_r: float, stream=None):
        return gbem_capacitance(self.mesh, self, eps_r, stream)

    def download(self) -> np.ndarray:
        A = np.empty((self.n, self.n), np.float64, order="F")
        self.ctx.check(self.ctx.lib.gbem_matrix_download(self.h, _ptr(A)))
        return A

    def status(self):
        self.ctx.check(self.ctx.lib.gbem_matrix_status(self.h))

    def info(self):
        n = ctypes.c_int()
        counts = np.zeros(7, np.int64)
        self.ctx.check(self.ctx.lib.gbem_matrix_info(self.h, ctypes.byref(n), _ptr(counts)))
        return n.value, counts

    def class_counts(self):
        """Pairs per evaluation class: [0] near parallel, [1] near
        perpendicular, [2n] / [2n+1] far parallel / perpendicular of order n."""
        counts = np.zeros(14, np.int64)
        self.ctx.check(self.ctx.lib.gbem_matrix_class_counts(self.h, _ptr(counts)))
        return counts

    def close(self):
        if getattr(self, "h", None):
            if self.ctx.h is not None:
                self.ctx.lib.gbem_matrix_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchTuning(ctypes.Structure):
    """gbem_batch_tuning: the configuration the autotuner chose."""
    _fields_ = [("groups", ctypes.c_int), ("iters", ctypes.c_int), ("ms", ctypes.c_double),
                ("from_cache", ctypes.c_int)]


class Batch:
    """Batched extraction of independent structures (one CUDA graph per
    group of structures; the groups run concurrently)."""

    def __init__(self, ctx: Context, meshes, iters: int = 0, groups: int = 1, _handle=None):
        self.ctx, self.meshes = ctx, list(meshes)
        if _handle is None:
            arr = self._mesh_array(self.meshes)
            h = ctypes.c_void_p()
            ctx.check(ctx.lib.gbem_batch_create_grouped(ctx.h, len(self.meshes), ctypes.cast(arr, ctypes.c_void_p),
                                                        int(groups), int(iters), ctypes.byref(h)))
        else:
            h = _handle
        self.h = h
        ctx._children.add(self)
        cnt, tot = ctypes.c_int(), ctypes.c_longlong()
        self.c_offset = np.zeros(len(self.meshes), np.int64)
        ctx.check(ctx.lib.gbem_batch_info(h, ctypes.byref(cnt), ctypes.byref(tot), _ptr(self.c_offset)))
        self.c_total = tot.value

    @staticmethod
    def _mesh_array(meshes):
        return (ctypes.c_void_p * len(meshes))(*[m.h.value if isinstance(m.h, ctypes.c_void_p) else m.h
                                                 for m in meshes])

    @classmethod
    def autotune(cls, ctx: Context, meshes, max_iters: int = 0, cache_path: str | None = None):
        """The fastest of 1, 2 and 4 groups with the fewest refinement passes
        that meet the tolerance (gbem_batch_autotune); returns (batch, choice)."""
        meshes = list(meshes)
        arr = cls._mesh_array(meshes)
        h = ctypes.c_void_p()
        rep = BatchTuning()
        ctx.check(ctx.lib.gbem_batch_autotune(ctx.h, len(meshes), ctypes.cast(arr, ctypes.c_void_p), int(max_iters),
                                              cache_path.encode() if cache_path else None, ctypes.byref(h),
                                              ctypes.byref(rep)))
        choice = {"groups": rep.groups, "iters": rep.iters, "ms": rep.ms, "from_cache": bool(rep.from_cache)}
        return cls(ctx, meshes, _handle=h), choice

    @property
    def config(self):
        g, i = ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.gbem_batch_config(self.h, ctypes.byref(g), ctypes.byref(i)))
        return {"groups": g.value, "iters": i.value}

    def run(self, eps_r: float, stream=None):
        """List of capacitance matrices (farads) and the residual of each."""
        C = np.empty(self.c_total, np.float64)
        res = np.empty(len(self.meshes), np.float64)
        self.ctx.check(self.ctx.lib.gbem_batch_run(self.h, float(eps_r), _ptr(C), _ptr(res), _stream_handle(stream)))
        out = []
        for b, m in enumerate(self.meshes):
            o = int(self.c_offset[b])
            out.append(C[o:o + m.n_cond * m.n_cond].reshape(m.n_cond, m.n_cond))
        return out, res

    def close(self):
        if getattr(self, "h", None):
            if self.ctx.h is not None:
                self.ctx.lib.gbem_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _boxes(boxes):
    arr = (_Box * len(boxes))()
    for i, (lo, hi, c) in enumerate(boxes):
        arr[i].lo[:] = [float(v) for v in lo]
        arr[i].hi[:] = [float(v) for v in hi]
        arr[i].conductor = int(c)
    return arr


MAX_LAYERS = 16
FACE_GROUND, FACE_NEUMANN, PANEL_INTERFACE = -1, -2, -3


class _Stack(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("n_layers", ctypes.c_int32),
                ("z", ctypes.c_double * (MAX_LAYERS + 1)), ("eps_r", ctypes.c_double * MAX_LAYERS),
                ("face_bc", ctypes.c_int32 * 6), ("h", ctypes.c_double), ("h_outer", ctypes.c_double),
                ("graded", ctypes.c_int32), ("main_conductor", ctypes.c_int32), ("p1", ctypes.c_double),
                ("p2", ctypes.c_double), ("p3", ctypes.c_double), ("p5", ctypes.c_double)]


class Stack:
    """A layered dielectric stack and its system (gbem_stack_*, Sec. 4)."""

    def __init__(self, ctx: Context, lo, hi, z, eps_r, face_bc, boxes, h: float, h_outer: float = 0.0,
                 graded=None):
        """graded = (main conductor id, p1, p2, p3, p5): the paper's partition
        for that main net instead of uniform cells."""
        p = _Stack()
        p.lo[:] = [float(v) for v in lo]
        p.hi[:] = [float(v) for v in hi]
        p.n_layers = len(eps_r)
        if len(z) != len(eps_r) + 1 or len(eps_r) > MAX_LAYERS:
            raise ValueError("z needs one more entry than eps_r, at most MAX_LAYERS layers")
        for a, v in enumerate(z):
            p.z[a] = float(v)
        for a, v in enumerate(eps_r):
            p.eps_r[a] = float(v)
        p.face_bc[:] = [int(v) for v in face_bc]
        p.h, p.h_outer = float(h), float(h_outer)
        if graded is not None:
            p.graded = 1
            p.main_conductor = int(graded[0])
            p.p1, p.p2, p.p3, p.p5 = (float(v) for v in graded[1:])
        self.ctx, self.h = ctx, None
        self.eps_r = [float(v) for v in eps_r]
        arr = _boxes(boxes) if boxes else None
        out = _P()
        ctx.check(ctx.lib.gbem_stack_mesh(ctx.h, ctypes.byref(p), arr, len(boxes), ctypes.byref(out)))
        self.h = out
        ctx._children.add(self)
        n, neq, nc = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ctx.check(ctx.lib.gbem_stack_info(out, ctypes.byref(n), ctypes.byref(neq), ctypes.byref(nc)))
        self.n, self.n_eq, self.n_cond = n.value, neq.value, nc.value

    def panels(self) -> dict:
        """The panels as arrays (the same keys as the oracle's stack mesh)."""
        n = self.n
        d = {"axis": np.empty(n, np.int8), "geo": np.empty((n, 5), np.float64), "kind": np.empty(n, np.int32),
             "cond": np.empty(n, np.int32), "region_a": np.empty(n, np.int32), "region_b": np.empty(n, np.int32),
             "sign": np.empty(n, np.int8)}
        ids = np.empty(self.n_cond, np.int32)
        self.ctx.check(self.ctx.lib.gbem_stack_panels(
            self.h, _ptr(d["axis"]), _ptr(d["geo"]), _ptr(d["kind"]), _ptr(d["cond"]), _ptr(d["region_a"]),
            _ptr(d["region_b"]), _ptr(d["sign"]), _ptr(ids)))
        d["cond_ids"] = ids
        return d

    def assemble(self, precision=GBEM_FP64, stream=None):
        self.ctx.check(self.ctx.lib.gbem_stack_assemble(self.h, int(precision), _stream_handle(stream)))

    def iterations(self) -> int:
        it = ctypes.c_int()
        self.ctx.check(self.ctx.lib.gbem_stack_iterations(self.h, ctypes.byref(it)))
        return it.value

    def system(self):
        """(M float64[n_eq, n_eq], B float64[n_eq, n_cond]) as assembled."""
        M = np.empty((self.n_eq, self.n_eq), np.float64)
        B = np.empty((self.n_eq, self.n_cond), np.float64)
        self.ctx.check(self.ctx.lib.gbem_stack_system(self.h, _ptr(M), _ptr(B)))
        return M, B

    def capacitance(self, stream=None):
        """(C float64[n_cond, n_cond] in farads, relative residual)."""
        C = np.empty((self.n_cond, self.n_cond), np.float64)
        r = ctypes.c_double()
        self.ctx.check(self.ctx.lib.gbem_stack_capacitance(self.h, _stream_handle(stream), _ptr(C), ctypes.byref(r)))
        return C, r.value

    def close(self):
        if getattr(self, "h", None):
            if self.ctx.h is not None:
                self.ctx.lib.gbem_stack_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Extraction server with continuous batching (gbem_server_*)."""

    def __init__(self, device: int = 0, hbm_budget: int = 64 << 30, slots: int = 4, precision=GBEM_MIXED):
        self.lib = load()
        h = ctypes.c_void_p()
        st = self.lib.gbem_server_create(int(device), int(hbm_budget), int(slots), int(precision), ctypes.byref(h))
        if st != GBEM_OK:
            raise GbemError(st, "gbem_server_create failed")
        self.h = h

    def submit(self, rid: int, boxes, params, eps_r: float) -> int:
        arr = _boxes(boxes)
        p = _MeshParams(float(params["h"]), float(params.get("ratio", 1.0)), float(params.get("h_min", 0.0)))
        need = ctypes.c_size_t(0)
        st = self.lib.gbem_server_submit(self.h, int(rid), arr, len(boxes), ctypes.byref(p), float(eps_r),
                                         ctypes.byref(need))
        if st != GBEM_OK:
            raise GbemError(st, "gbem_server_submit failed")
        return need.value

    def poll(self, wait_ms: int = 0, max_results: int = 256):
        """List of (info dict, C) for completed requests."""
        infos = (ResultInfo * max_results)()
        C = np.empty(max_results * 256, np.float64)
        cnt = ctypes.c_int(0)
        st = self.lib.gbem_server_poll(self.h, infos, _ptr(C), len(C), max_results, ctypes.byref(cnt), int(wait_ms))
        if st != GBEM_OK:
            raise GbemError(st, "gbem_server_poll failed")
        out = []
        for k in range(cnt.value):
            i = infos[k]
            info = {f: getattr(i, f) for f, _ in ResultInfo._fields_}
            n = i.n_cond
            Ck = C[i.c_offset:i.c_offset + n * n].reshape(n, n).copy() if n else None
            out.append((info, Ck))
        return out

    def stats(self):
        q, r = ctypes.c_int(), ctypes.c_int()
        res, peak = ctypes.c_size_t(), ctypes.c_size_t()
        self.lib.gbem_server_stats(self.h, ctypes.byref(q), ctypes.byref(r), ctypes.byref(res), ctypes.byref(peak))
        return {"queued": q.value, "running": r.value, "reserved": res.value, "peak_reserved": peak.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbem_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- ABI-named calls

def gbem_create(device: int = 0, hbm_budget: int = 0, torch_alloc: bool = True) -> Context:
    return Context(device, hbm_budget, torch_alloc)


def gbem_mesh(ctx: Context, boxes, params) -> Mesh:
    arr = (_Box * len(boxes))()
    for i, (lo, hi, c) in enumerate(boxes):
        arr[i].lo[:] = [float(v) for v in lo]
        arr[i].hi[:] = [float(v) for v in hi]
        arr[i].conductor = int(c)
    p = _MeshParams(float(params["h"]), float(params.get("ratio", 1.0)), float(params.get("h_min", 0.0)))
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.gbem_mesh(ctx.h, arr, len(boxes), ctypes.byref(p), ctypes.byref(h)))
    return Mesh(ctx, h)


def gbem_mesh_graded(ctx: Context, boxes, main: int, p1: float, p2: float, p3: float, p5: float,
                     h_max: float = 0.0, enclosure=None) -> Mesh:
    """gbem_mesh_graded: the paper's distance-graded partition for main net
    `main`; enclosure = (lo, hi, conductor id) of a grounded box, or None."""
    arr = _boxes(boxes)
    p = _PartitionParams()
    p.main_conductor = int(main)
    p.p1, p.p2, p.p3, p.p5, p.h_max = float(p1), float(p2), float(p3), float(p5), float(h_max)
    if enclosure is not None:
        lo, hi, c = enclosure
        p.has_enclosure = 1
        p.encl_lo[:] = [float(v) for v in lo]
        p.encl_hi[:] = [float(v) for v in hi]
        p.encl_conductor = int(c)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.gbem_mesh_graded(ctx.h, arr, len(boxes), ctypes.byref(p), ctypes.byref(h)))
    return Mesh(ctx, h)


def gbem_mesh_refine(mesh: Mesh, density, theta: float):
    """gbem_mesh_refine: bisect the panels whose indicator |I_j| |dq/dtau|_j
    is at least theta times the largest; density per panel of `mesh` (its
    panel order).  Returns (new Mesh, indicators float64[n], panels bisected)."""
    density = np.ascontiguousarray(density, dtype=np.float64)
    if density.shape != (mesh.n,):
        raise ValueError("density needs one value per panel")
    eta = np.empty(mesh.n, np.float64)
    h = ctypes.c_void_p()
    nm = ctypes.c_int(0)
    mesh.ctx.check(mesh.ctx.lib.gbem_mesh_refine(mesh.h, _ptr(density), float(theta), _ptr(eta), ctypes.byref(h),
                                                 ctypes.byref(nm)))
    return Mesh(mesh.ctx, h), eta, nm.value


def gbem_mesh_from_panels(ctx: Context, axis, geo, cond) -> Mesh:
    axis = np.ascontiguousarray(axis, dtype=np.int8)
    geo = np.ascontiguousarray(geo, dtype=np.float64).reshape(-1, 5)
    cond = np.ascontiguousarray(cond, dtype=np.int32)
    h = ctypes.c_void_p()
    ctx.check(ctx.lib.gbem_mesh_from_panels(ctx.h, len(axis), _ptr(axis), _ptr(geo), _ptr(cond),
                                            ctypes.byref(h)))
    return Mesh(ctx, h)


def gbem_assemble(mesh: Mesh, precision=GBEM_FP64, stream=None) -> Matrix:
    h = ctypes.c_void_p()
    ctx = mesh.ctx
    ctx.check(ctx.lib.gbem_assemble(mesh.h, int(precision), _stream_handle(stream), ctypes.byref(h)))
    return Matrix(mesh, h, precision)


def gbem_factor(mat: Matrix, stream=None):
    mat.ctx.check(mat.ctx.lib.gbem_factor(mat.h, _stream_handle(stream)))


def gbem_solve(mat: Matrix, B, X=None, stream=None):
    """Solve A X = B on device; B, X are torch float64 CUDA tensors of shape
    (N, nrhs) in column-major layout (i.e. B.t() contiguous) or (N,).
    Returns (X, refinement iterations)."""
    import torch
    if B.dim() == 1:
        B = B[:, None]
    Bc = B.t().contiguous()          # (nrhs, N) row-major == (N, nrhs) column-major
    n, nrhs = B.shape
    Xc = torch.empty_like(Bc) if X is None else X.t()
    it = ctypes.c_int(0)
    mat.ctx.check(mat.ctx.lib.gbem_solve(mat.h, ctypes.c_void_p(Bc.data_ptr()), nrhs, n,
                                         ctypes.c_void_p(Xc.data_ptr()), n, ctypes.byref(it),
                                         _stream_handle(stream)))
    return Xc.t(), it.value


def gbem_capacitance(mesh: Mesh, mat: Matrix, eps_r: float, stream=None, want_residual: bool = True):
    """Maxwell capacitance matrix in farads (n_c x n_c, ascending conductor
    ids) and the final relative residual."""
    C = np.empty((mesh.n_cond, mesh.n_cond), np.float64)
    r = ctypes.c_double(0.0)
    mesh.ctx.check(mesh.ctx.lib.gbem_capacitance(mesh.h, mat.h, float(eps_r), _ptr(C),
                                                 ctypes.byref(r) if want_residual else None,
                                                 _stream_handle(stream)))
    return C, r.value


def extract(ctx: Context, boxes, params, eps_r: float, precision=GBEM_FP64, stream=None):
    """Mesh, assemble, factor, solve and reduce: one full extraction."""
    mesh = gbem_mesh(ctx, boxes, params)
    try:
        mat = gbem_assemble(mesh, precision, stream)
        try:
            return gbem_capacitance(mesh, mat, eps_r, stream)
        finally:
            mat.close()
    finally:
        mesh.close()
