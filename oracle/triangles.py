"""FP64 CPU oracle for flat-triangle panels (general, non-Manhattan
conductors; the paper meshes conductors with cuboids, Sec. 3.3, and flat
panels of any shape fit its Galerkin formulation of Sec. 3.1 unchanged).

TEST INFRASTRUCTURE ONLY: the tests are the only callers.  The product path
never imports this module, and this module imports nothing from the product.

* ``tri_potential``  -- int_T 1/|x - y| dy, the exact potential of a uniformly
                        charged flat triangle (edge-by-edge closed form, in
                        ``gbem_oracle.c``).
* ``tri_entries`` / ``tri_assemble`` -- a_ij = (1/(4 pi |T_i||T_j|)) int int
                        1/|x - y| over triangles, the matrix of Eq. "matrix":
                        the exact potential under an adaptive collapsed
                        Gauss-Legendre rule, or a collapsed rule on both
                        triangles for separated pairs.
* ``tri_capacitance`` -- the solve and charges of Eqs. "lineareq1" and
                        "electriccharge" (Cholesky, as for rectangles).

A triangle is 9 numbers, its vertices (a, b, c).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import oracle as O


def _load():
    lib = O._load()
    if not getattr(lib, "_tri_ready", False):
        P = ctypes.c_void_p
        lib.orc_tri_potential_at.restype = ctypes.c_double
        lib.orc_tri_potential_at.argtypes = [P, P]
        lib.orc_tri_entries.restype = ctypes.c_int
        lib.orc_tri_entries.argtypes = [ctypes.c_int, P, ctypes.c_int64, P, P, P, ctypes.c_int]
        lib._tri_ready = True
    return lib


def tri_potential(tri, x) -> float:
    t = np.ascontiguousarray(tri, dtype=np.float64).reshape(9)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc_tri_potential_at(O._ptr(t), O._ptr(xx)))


def tri_areas(tris) -> np.ndarray:
    t = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
    return 0.5 * np.linalg.norm(np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0]), axis=1)


def tri_entries(tris, I, J, nthreads: int = 0) -> np.ndarray:
    t = np.ascontiguousarray(tris, dtype=np.float64).reshape(-1, 9)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    out = np.empty(len(I), dtype=np.float64)
    nf = _load().orc_tri_entries(len(t), O._ptr(t), len(I), O._ptr(I), O._ptr(J), O._ptr(out), int(nthreads))
    if nf:
        raise RuntimeError(f"oracle: {nf} triangle quadratures did not converge")
    return out


def tri_assemble(tris, nthreads: int = 0) -> np.ndarray:
    """The full symmetric matrix (lower triangle evaluated, mirrored)."""
    n = len(np.asarray(tris).reshape(-1, 9))
    I, J = np.tril_indices(n)
    v = tri_entries(tris, I, J, nthreads)
    A = np.zeros((n, n))
    A[I, J] = v
    A[J, I] = v
    return A


def tri_capacitance(tris, cond, eps_r: float, nthreads: int = 0) -> np.ndarray:
    A = tri_assemble(tris, nthreads)
    return O.capacitance_from_matrix(A, np.asarray(cond), eps_r)
