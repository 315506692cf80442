"""FP64 CPU oracle for GBEM (Wu & Li, arXiv 2203.11733).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path never
imports this module, and this module imports nothing from the product.

It implements, plainly and slowly, every step of the extraction:

* ``mesh_boxes``      -- the boundary partition into rectangles I_j of a set of
                         cuboid conductors (Sec. 3.1, before Eq. "myequation";
                         Sec. 3.3: every conductor is a union of cuboids).
* ``entries`` / ``assemble`` -- the Galerkin matrix of Eq. "matrix",
                         a_ij = (1/(4 pi |I_i||I_j|)) int int 1/|x-y|, computed
                         in ``gbem_oracle.c`` (see its header for the method).
* ``refine``          -- the error-driven refinement behind Sec. 3.2's
                         Proposition "error" (charge error bounded by
                         C sup_j |I_j| sup |dq/dtau| on I_j): indicators from
                         the densities of touching panels, bisection of the
                         panels with the largest ones.
* ``capacitance``     -- the right-hand sides b of Eq. "lineareq1" (f0 = 1 on
                         the main net, 0 elsewhere, Sec. 3.1), the solve A X = b
                         by Cholesky (Sec. 3.2: A is symmetric positive
                         definite, Theorem 1) and the charge of Eq.
                         "electriccharge", Q_n = eps * sum_{I_j on net n} X_j.

Units: lengths in micrometres, so A is in 1/um and X in um; the capacitance in
farads is eps0 * eps_r * 1e-6 * X.

Two sibling modules extend it: ``dielectric`` (several dielectrics, Sec. 4:
double-layer entries, the per-layer system, LU) and ``triangles`` (flat
triangle panels).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbem_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

EPS0 = 8.8541878128e-12  # F/m, CODATA 2018

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, strict IEEE arithmetic)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        P = ctypes.c_void_p
        lib.orc_rect_potential.restype = d
        lib.orc_rect_potential.argtypes = [ctypes.c_int, P, P]
        lib.orc_pair_integral.restype = d
        lib.orc_pair_integral.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P]
        lib.orc_entries.restype = ctypes.c_int
        lib.orc_entries.argtypes = [ctypes.c_int, P, P, i64, P, P, P, ctypes.c_int]
        lib.orc_assemble.restype = ctypes.c_int
        lib.orc_assemble.argtypes = [ctypes.c_int, P, P, P, ctypes.c_int]
        lib.orc_gl_nodes.restype = ctypes.c_int
        lib.orc_gl_nodes.argtypes = [ctypes.c_int, P, P]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads() -> int:
    return int(_load().orc_max_threads())


# --------------------------------------------------------------------------
# Boundary partition (Sec. 3.1 and Sec. 3.3)
# --------------------------------------------------------------------------

def divide(lo: float, hi: float, h: float, ratio: float = 1.0, h_min: float = 0.0) -> list[float]:
    """Nodes of a 1-D division of [lo, hi].

    Uniform (ratio <= 1): n = ceil(L/h) equal cells.  Edge-graded: cells of
    h_min, h_min*ratio, ... grow from both ends while they stay below h; the
    middle is split into equal cells no longer than h.
    """
    L = hi - lo
    if ratio <= 1.0 or h_min <= 0.0 or h_min >= h:
        n = max(1, math.ceil(L / h - 1e-9))
        return [lo + (L * k) / n for k in range(n)] + [hi]
    sizes = []
    s = h_min
    while s < h:
        sizes.append(s)
        s = s * ratio
    m = len(sizes)
    while m > 0 and 2.0 * sum(sizes[:m]) > L:
        m -= 1
    if m == 0:
        n = max(1, math.ceil(L / h - 1e-9))
        return [lo + (L * k) / n for k in range(n)] + [hi]
    left = [lo]
    acc = lo
    for k in range(m):
        acc = acc + sizes[k]
        left.append(acc)
    right = [hi]
    acc = hi
    for k in range(m):
        acc = acc - sizes[k]
        right.append(acc)
    right.reverse()
    xl, xr = left[-1], right[0]
    M = xr - xl
    nodes = left[:-1]
    if M > 1e-12 * L:
        nmid = max(1, math.ceil(M / h - 1e-9))
        nodes += [xl + (M * k) / nmid for k in range(nmid)]
    nodes += right
    return nodes


def mesh_boxes(boxes, h: float, ratio: float = 1.0, h_min: float = 0.0):
    """Panels of the surfaces of disjoint cuboids.

    ``boxes``: iterable of (lo[3], hi[3], conductor).  Returns (axis int32[n],
    geo float64[n,5] = (c, lo0, hi0, lo1, hi1), cond int32[n]).  Every face of
    a box is cut on the tensor grid of the 1-D divisions of its two edges.
    """
    axis, geo, cond = [], [], []
    for lo, hi, c in boxes:
        for k in range(3):
            p, q = [a for a in range(3) if a != k]
            np_ = divide(lo[p], hi[p], h, ratio, h_min)
            nq = divide(lo[q], hi[q], h, ratio, h_min)
            for plane in (lo[k], hi[k]):
                for a in range(len(np_) - 1):
                    for b in range(len(nq) - 1):
                        axis.append(k)
                        geo.append((plane, np_[a], np_[a + 1], nq[b], nq[b + 1]))
                        cond.append(c)
    return (np.asarray(axis, dtype=np.int32), np.asarray(geo, dtype=np.float64).reshape(-1, 5),
            np.asarray(cond, dtype=np.int32))


def mesh_graded(boxes, main, p1, p2, p3, p5, h_max=0.0, enclosure=None):
    """The paper's distance-graded partition for the main net `main`
    (Sec. 3.3).  A panel I on a face may stay when
        |I| <= p4                  for d < p5,
        |I| <= p4 p3 (d / p5)^3    for d >= p5,
    d the distance from I to the main net's nearest box; p4 = p1 on faces
    that look toward the main net (some of it lies beyond the face's plane on
    the outward side; the main net's own faces and an enclosure's inner
    faces always do), p4 = p1 p2 on faces that look away.  Larger panels are
    halved across their longer edge (the first in-plane axis on a tie), and
    so on.  h_max > 0 also bounds both edges.  `enclosure` = (lo, hi, cond):
    the inner faces of a grounded box, meshed as conductor cond.  Returns
    (axis, geo, cond) as mesh_boxes does, faces in box order, each face's
    panels in depth-first order, first halves first."""
    mains = [(lo, hi) for lo, hi, c in boxes if c == main]
    if not mains:
        raise ValueError("no box of the main net")
    mlo = [min(b[0][d] for b in mains) for d in range(3)]
    mhi = [max(b[1][d] for b in mains) for d in range(3)]

    def dist(k, c, a0, b0, a1, b1):
        p, q = [x for x in range(3) if x != k]
        lo = [0.0] * 3
        hi = [0.0] * 3
        lo[k] = hi[k] = c
        lo[p], hi[p], lo[q], hi[q] = a0, b0, a1, b1
        best = math.inf
        for blo, bhi in mains:
            s = 0.0
            for d in range(3):
                g = max(0.0, max(blo[d] - hi[d], lo[d] - bhi[d]))
                s += g * g
            best = min(best, math.sqrt(s))
        return best

    faces = []
    for lo, hi, c in boxes:
        for k in range(3):
            p, q = [x for x in range(3) if x != k]
            for side, plane in ((0, lo[k]), (1, hi[k])):
                toward = c == main or (mhi[k] > plane if side == 1 else mlo[k] < plane)
                faces.append((k, plane, lo[p], hi[p], lo[q], hi[q], c, toward))
    if enclosure is not None:
        elo, ehi, ec = enclosure
        for k in range(3):
            p, q = [x for x in range(3) if x != k]
            for plane in (elo[k], ehi[k]):
                faces.append((k, plane, elo[p], ehi[p], elo[q], ehi[q], ec, True))
    axis, geo, cond = [], [], []

    def refine(k, plane, a0, b0, a1, b1, c, p4):
        d = dist(k, plane, a0, b0, a1, b1)
        limit = p4 if d < p5 else p4 * p3 * ((d / p5) * (d / p5) * (d / p5))
        e0, e1 = b0 - a0, b1 - a1
        if not (e0 * e1 > limit or (h_max > 0.0 and max(e0, e1) > h_max)):
            axis.append(k)
            geo.append((plane, a0, b0, a1, b1))
            cond.append(c)
            return
        if e0 >= e1:
            m = 0.5 * (a0 + b0)
            refine(k, plane, a0, m, a1, b1, c, p4)
            refine(k, plane, m, b0, a1, b1, c, p4)
        else:
            m = 0.5 * (a1 + b1)
            refine(k, plane, a0, b0, a1, m, c, p4)
            refine(k, plane, a0, b0, m, b1, c, p4)

    for k, plane, a0, b0, a1, b1, c, toward in faces:
        refine(k, plane, a0, b0, a1, b1, c, p1 if toward else p1 * p2)
    return (np.asarray(axis, dtype=np.int32), np.asarray(geo, dtype=np.float64).reshape(-1, 5),
            np.asarray(cond, dtype=np.int32))


def refine(axis, geo, cond, density, theta: float):
    """Error-driven refinement (Sec. 3.2, Proposition "error": the charge
    error on a net is at most C sup_j |I_j| sup_{x in I_j} |dq/dtau|).

    The density is constant on each panel, so its tangential derivative on
    panel j is estimated with difference quotients to the panels that share a
    piece of its boundary: the same conductor and closed rectangles that meet
    in a segment of positive length (also across the edge between two faces;
    a common corner alone does not count), quotient
    |density_k - density_j| / |centre_k - centre_j|, the largest one kept.
    eta_j = |I_j| times it.  Panels with eta_j >= theta * max(eta) (none when
    max(eta) is 0) are halved across their longer edge (the first in-plane
    axis on a tie).  Plain O(N^2) neighbour search.

    Returns (axis, geo, cond) of the refined panels (input order, each
    bisected panel replaced by its lower half then its upper half), eta and
    the number of bisected panels."""
    axis = np.asarray(axis, dtype=np.int64)
    geo = np.asarray(geo, dtype=np.float64).reshape(-1, 5)
    cond = np.asarray(cond)
    d = np.asarray(density, dtype=np.float64)
    n = len(axis)
    lo = np.zeros((n, 3))
    hi = np.zeros((n, 3))
    for i in range(n):
        k = int(axis[i])
        p = 1 if k == 0 else 0
        q = 1 if k == 2 else 2
        lo[i, k] = hi[i, k] = geo[i, 0]
        lo[i, p], hi[i, p] = geo[i, 1], geo[i, 2]
        lo[i, q], hi[i, q] = geo[i, 3], geo[i, 4]
    ctr = 0.5 * (lo + hi)
    area = (geo[:, 2] - geo[:, 1]) * (geo[:, 4] - geo[:, 3])
    tol = 1e-9 * (1.0 + np.max(np.abs(geo)))
    grad = np.zeros(n)
    for j in range(n):
        ov = np.minimum(hi[j], hi) - np.maximum(lo[j], lo)   # overlap per axis
        touch = np.all(ov >= -tol, axis=1) & (np.max(ov, axis=1) > tol)
        touch &= cond == cond[j]
        touch[j] = False
        k = np.nonzero(touch)[0]
        if len(k):
            dist = np.sqrt(np.sum((ctr[k] - ctr[j]) ** 2, axis=1))
            grad[j] = np.max(np.abs(d[k] - d[j]) / dist)
    eta = area * grad
    emax = eta.max() if n else 0.0
    a2, g2, c2 = [], [], []
    marked = 0
    for i in range(n):
        c0, l0, h0, l1, h1 = geo[i]
        if not (emax > 0.0 and eta[i] >= theta * emax):
            a2.append(axis[i]); g2.append((c0, l0, h0, l1, h1)); c2.append(cond[i])
            continue
        marked += 1
        if h0 - l0 >= h1 - l1:
            m = 0.5 * (l0 + h0)
            halves = [(c0, l0, m, l1, h1), (c0, m, h0, l1, h1)]
        else:
            m = 0.5 * (l1 + h1)
            halves = [(c0, l0, h0, l1, m), (c0, l0, h0, m, h1)]
        for h_ in halves:
            a2.append(axis[i]); g2.append(h_); c2.append(cond[i])
    return (np.array(a2, np.int32), np.array(g2, np.float64).reshape(-1, 5), np.array(c2, np.int32), eta, marked)


def areas(geo: np.ndarray) -> np.ndarray:
    return (geo[:, 2] - geo[:, 1]) * (geo[:, 4] - geo[:, 3])


# --------------------------------------------------------------------------
# Matrix entries (Sec. 3.4, Eq. "matrix")
# --------------------------------------------------------------------------

def rect_potential(axis: int, geo, x) -> float:
    """int over the panel of 1/|x - y| dy (the inner integral)."""
    g = np.ascontiguousarray(geo, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc_rect_potential(int(axis), _ptr(g), _ptr(xx)))


def pair_integral(axis_i: int, geo_i, axis_j: int, geo_j, method: int = 0):
    """int_{I_i} int_{I_j} 1/|x-y| (no 1/(4 pi), no area factors).

    method 0 chooses 4-D Gauss-Legendre for well separated pairs and the
    split-outer quadrature otherwise; method 1 always splits.  Returns
    (value, number of quadratures that did not meet their convergence test).
    """
    gi = np.ascontiguousarray(geo_i, dtype=np.float64)
    gj = np.ascontiguousarray(geo_j, dtype=np.float64)
    nf = ctypes.c_int(0)
    v = _load().orc_pair_integral(int(axis_i), _ptr(gi), int(axis_j), _ptr(gj), int(method),
                                  ctypes.byref(nf))
    return float(v), int(nf.value)


def entries(axis, geo, I, J, nthreads: int = 0):
    """a_ij for the index pairs (I[t], J[t])."""
    axis = np.ascontiguousarray(axis, dtype=np.int32)
    geo = np.ascontiguousarray(geo, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    out = np.empty(len(I), dtype=np.float64)
    nf = _load().orc_entries(len(axis), _ptr(axis), _ptr(geo), len(I), _ptr(I), _ptr(J), _ptr(out),
                             int(nthreads))
    if nf:
        raise RuntimeError(f"oracle: {nf} quadratures did not converge")
    return out


def assemble(axis, geo, nthreads: int = 0) -> np.ndarray:
    """The full symmetric N x N matrix A of Eq. "matrix"."""
    axis = np.ascontiguousarray(axis, dtype=np.int32)
    geo = np.ascontiguousarray(geo, dtype=np.float64)
    n = len(axis)
    A = np.empty((n, n), dtype=np.float64)
    nf = _load().orc_assemble(n, _ptr(axis), _ptr(geo), _ptr(A), int(nthreads))
    if nf:
        raise RuntimeError(f"oracle: {nf} quadratures did not converge")
    return A


# --------------------------------------------------------------------------
# Solve and charge (Eqs. "lineareq1" and "electriccharge")
# --------------------------------------------------------------------------

def rhs(cond: np.ndarray):
    """b for every main net: column k is 1 on the panels of conductor k.

    Returns (B float64[N, n_c], conductor ids in column order)."""
    ids = np.unique(cond)
    B = (cond[:, None] == ids[None, :]).astype(np.float64)
    return B, ids


def solve(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """X = A^{-1} B by Cholesky (A is symmetric positive definite)."""
    import scipy.linalg as sla
    c = sla.cho_factor(A, lower=True, check_finite=True)
    return sla.cho_solve(c, B)


def capacitance_from_matrix(A: np.ndarray, cond: np.ndarray, eps_r: float) -> np.ndarray:
    """Maxwell capacitance matrix in farads: C[m, k] = charge on conductor m
    when conductor k is at 1 V and every other conductor at 0 V."""
    B, _ = rhs(cond)
    X = solve(A, B)
    return EPS0 * eps_r * 1e-6 * (B.T @ X)


def capacitance(axis, geo, cond, eps_r: float, nthreads: int = 0) -> np.ndarray:
    A = assemble(axis, geo, nthreads)
    return capacitance_from_matrix(A, np.asarray(cond), eps_r)


def gauss_legendre(n: int):
    x = np.empty(n)
    w = np.empty(n)
    if _load().orc_gl_nodes(int(n), _ptr(x), _ptr(w)) != 0:
        raise ValueError(n)
    return x, w
