"""FP64 CPU oracle for the multi-dielectric case of GBEM (Wu & Li, arXiv
2203.11733, Sec. 4).

TEST INFRASTRUCTURE ONLY: the tests and the CPU baseline leg of ``bench.py``
are the only callers.  The product path never imports this module, and this
module imports nothing from the product.

The domain is split into dielectric regions Omega_a.  On the boundary of each
region the representation formula of Sec. 2, tested with the indicator of a
panel I_i and with u and q = du/dn (n the outward normal of Omega_a) constant
on every panel, gives the equation of Sec. 4 ("Linear Equation"):

    (1/2) |I_i| u_i + sum_k Q^a_ik u_k - sum_j U_ij q^a_j = 0,

    U_ij   = int_{I_i} int_{I_j} 1 / (4 pi |x - y|),
    Q^a_ik = int_{I_i} int_{I_k} <x - y, n_a(y)> / (4 pi |x - y|^3)

(u* and q* of Sec. 2).  This module restates that system for layered stacks
(``mesh_stack``): horizontal dielectric layers inside a box enclosure, whose
faces are grounded (u = 0), insulating (q = 0) or held at a conductor's
potential, with disjoint cuboid conductors inside the layers.

* ``mesh_stack``        -- the panels: conductor surfaces (mesh_boxes rule),
                           enclosure faces (the side faces cut at the layer
                           heights) and the interfaces between layers, with
                           the regions on each side and the outward normal.
* ``dlayer_entries``    -- d_ij = Q_ij for the normal +e_k of I_j, from the C
                           oracle (exact solid angle inside, adaptive outer
                           quadrature; see gbem_oracle.c).
* ``system``            -- the matrix and right-hand sides of the equations
                           above, one row per (region, panel of its
                           boundary), with the interface conditions
                           u_a = u_b and eps_a q_a = -eps_b q_b.
* ``capacitance``       -- LU with partial pivoting (Sec. 4: the operators
                           are not elliptic, the matrix is not symmetric),
                           then the charge on each conductor,
                           Q_n = eps0 sum_j eps_a q^a_j |I_j|.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import oracle as O

GROUND = -1      # enclosure face at 0 V
NEUMANN = -2     # insulating enclosure face, q = 0
INTERFACE = -3   # panel between two layers

KIND_CONDUCTOR, KIND_FACE, KIND_INTERFACE = 0, 1, 2


def _load():
    lib = O._load()
    if not getattr(lib, "_dl_ready", False):
        P = ctypes.c_void_p
        lib.orc_rect_dlayer.restype = ctypes.c_double
        lib.orc_rect_dlayer.argtypes = [ctypes.c_int, P, P]
        lib.orc_dl_entries.restype = ctypes.c_int
        lib.orc_dl_entries.argtypes = [ctypes.c_int, P, P, ctypes.c_int64, P, P, P, ctypes.c_int]
        lib._dl_ready = True
    return lib


def rect_dlayer(axis: int, geo, x) -> float:
    """int over the panel of (x_k - y_k) / |x - y|^3 dy, k its normal axis:
    the signed solid angle the panel subtends at x."""
    g = np.ascontiguousarray(geo, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    return float(_load().orc_rect_dlayer(int(axis), O._ptr(g), O._ptr(xx)))


def dlayer_entries(axis, geo, I, J, nthreads: int = 0) -> np.ndarray:
    """d_ij = (1/(4 pi)) int_{I_i} int_{I_j} (x_k - y_k) / |x - y|^3, k the
    normal axis of I_j, for the index pairs (I[t], J[t])."""
    axis = np.ascontiguousarray(axis, dtype=np.int32)
    geo = np.ascontiguousarray(geo, dtype=np.float64)
    I = np.ascontiguousarray(I, dtype=np.int32)
    J = np.ascontiguousarray(J, dtype=np.int32)
    out = np.empty(len(I), dtype=np.float64)
    nf = _load().orc_dl_entries(len(axis), O._ptr(axis), O._ptr(geo), len(I), O._ptr(I), O._ptr(J),
                                O._ptr(out), int(nthreads))
    if nf:
        raise RuntimeError(f"oracle: {nf} double-layer quadratures did not converge")
    return out


def slayer_entries(axis, geo, I, J, nthreads: int = 0) -> np.ndarray:
    """U_ij = (1/(4 pi)) int int 1/|x - y| = |I_i| |I_j| a_ij."""
    a = O.entries(axis, geo, I, J, nthreads)
    ar = O.areas(np.asarray(geo, dtype=np.float64))
    return a * ar[np.asarray(I)] * ar[np.asarray(J)]


# --------------------------------------------------------------------------
# Layered stacks
# --------------------------------------------------------------------------

class Stack:
    """Box enclosure [lo, hi] cut by the planes z[1] < ... < z[R-1] into R
    horizontal layers (z[0] = lo[2], z[R] = hi[2]) of relative permittivity
    eps[a].  face_bc[2k + s] is the condition on the enclosure face normal to
    axis k at lo[k] (s = 0) or hi[k] (s = 1): GROUND, NEUMANN or a conductor
    id >= 0 (the face is held at that conductor's potential)."""

    def __init__(self, lo, hi, z, eps, face_bc):
        self.lo = [float(v) for v in lo]
        self.hi = [float(v) for v in hi]
        self.z = [float(v) for v in z]
        self.eps = [float(v) for v in eps]
        self.face_bc = [int(v) for v in face_bc]
        if len(self.z) != len(self.eps) + 1 or self.z[0] != self.lo[2] or self.z[-1] != self.hi[2]:
            raise ValueError("layer planes must run from lo[2] to hi[2], one more than the layers")
        if any(b <= a for a, b in zip(self.z, self.z[1:])):
            raise ValueError("layer planes must increase")
        if len(self.face_bc) != 6 or any(v < NEUMANN for v in self.face_bc):
            raise ValueError("six face conditions")


def _cells(lo, hi, h):
    return O.divide(lo, hi, h)


def _graded_cells(k, plane, a0, b0, a1, b1, p4, p3, p5, power, hmax, mains):
    """Rectangles of one face under the paper's partition: bisect the longer
    edge (the first on a tie), first half first, until |I| <= p4 within p5 of
    the main net and |I| <= p4 p3 (d / p5)**power beyond, and both edges <= hmax
    (d the distance to the nearest box of the main net)."""
    out = []

    def dist(c0, c1, c2, c3):
        lo = [0.0] * 3
        hi = [0.0] * 3
        p, q = [x for x in range(3) if x != k]
        lo[k] = hi[k] = plane
        lo[p], hi[p], lo[q], hi[q] = c0, c1, c2, c3
        best = math.inf
        for blo, bhi in mains:
            s2 = sum(max(0.0, blo[d] - hi[d], lo[d] - bhi[d]) ** 2 for d in range(3))
            best = min(best, math.sqrt(s2))
        return best

    def split(c0, c1, c2, c3):
        d = dist(c0, c1, c2, c3)
        limit = p4 if d < p5 else p4 * p3 * (d / p5) ** power
        e0, e1 = c1 - c0, c3 - c2
        if not (e0 * e1 > limit or (hmax > 0.0 and max(e0, e1) > hmax)):
            out.append((c0, c1, c2, c3))
            return
        if e0 >= e1:
            m = 0.5 * (c0 + c1)
            split(c0, m, c2, c3)
            split(m, c1, c2, c3)
        else:
            m = 0.5 * (c2 + c3)
            split(c0, c1, c2, m)
            split(c0, c1, m, c3)

    split(a0, b0, a1, b1)
    return out


def mesh_stack(stack: Stack, boxes, h: float, h_outer: float = 0.0, graded=None):
    """Panels of a layered stack.  Conductor boxes (disjoint, strictly inside
    the enclosure, their bottom and top off the layer planes; a box may cross
    layer planes, as a via does) are cut as mesh_boxes cuts them (edge cells
    ceil(L / h)), their side faces also where they cross a layer plane;
    enclosure faces and interfaces with cells of at most h_outer (h when 0),
    interfaces cut along the footprints of the boxes that cross them and
    holed there.  Returns a dict of arrays: axis, geo (c, lo0, hi0,
    lo1, hi1), kind, cond (conductor id, GROUND, NEUMANN or INTERFACE),
    region_a, region_b (-1 unless an interface: region_a the layer below),
    sign (the outward normal of region_a is sign * e_axis).

    graded = (main, p1, p2, p3, p5) meshes by the paper's partition for the
    main net `main` instead: conductor faces by the rule of Sec. 3.3 (|I| <=
    p4 near the main net, p4 p3 (d/p5)^3 beyond; p4 = p1 on faces that look
    toward the main net, p1 p2 on those that look away), the enclosure's
    faces by the same rule with p4 = p1, the interfaces by the rule of Sec. 4
    (p4 p3 (d/p5)^2 beyond, p4 = p1); h and h_outer then cap the panel
    edges."""
    h_out = h_outer if h_outer > 0.0 else h
    R = len(stack.eps)
    rows = []   # (axis, geo, kind, cond, ra, rb, sign)
    if graded is not None:
        main, p1, p2, p3, p5 = graded
        mains = [([float(v) for v in lo], [float(v) for v in hi]) for lo, hi, c in boxes if int(c) == int(main)]
        if not mains:
            raise ValueError("no box of the main net")
        mlo = [min(b[0][d] for b in mains) for d in range(3)]
        mhi = [max(b[1][d] for b in mains) for d in range(3)]

    def cells2(k, plane, a0, b0, a1, b1, hcap, rule, toward=True):
        """The face's cells: a uniform grid, or the paper's partition."""
        if graded is None:
            cp, cq = _cells(a0, b0, hcap), _cells(a1, b1, hcap)
            return [(cp[i], cp[i + 1], cq[j], cq[j + 1]) for i in range(len(cp) - 1) for j in range(len(cq) - 1)]
        p4 = p1 if toward else p1 * p2
        return _graded_cells(k, plane, a0, b0, a1, b1, p4, p3, p5, 3 if rule == "conductor" else 2, hcap, mains)

    def layer_of(zz):
        return [a for a in range(R) if stack.z[a] < zz < stack.z[a + 1]][0]

    fboxes = []
    for lo, hi, c in boxes:
        lo = [float(v) for v in lo]
        hi = [float(v) for v in hi]
        if int(c) < 0:
            raise ValueError("conductor ids must be >= 0")
        inside = all(stack.lo[d] < lo[d] < hi[d] < stack.hi[d] for d in range(3))
        on_plane = any(v in stack.z for v in (lo[2], hi[2]))
        if not inside or on_plane:
            raise ValueError("every box must lie strictly inside the enclosure, its bottom and top off the "
                             "layer planes")
        fboxes.append((lo, hi, int(c)))
        spans = [a for a in range(R) if stack.z[a] < hi[2] and lo[2] < stack.z[a + 1]]
        for k in range(3):
            p, q = [x for x in range(3) if x != k]
            for plane, sgn, side in ((lo[k], 1, 0), (hi[k], -1, 1)):
                toward = True
                if graded is not None:
                    toward = int(c) == int(main) or (mhi[k] > plane if side == 1 else mlo[k] < plane)
                if k == 2:
                    pieces = [(layer_of(plane), lo[q], hi[q])]
                else:
                    # q == 2: a side face is cut where it crosses a layer plane
                    pieces = [(a, max(lo[2], stack.z[a]), min(hi[2], stack.z[a + 1])) for a in spans]
                for a, q0, q1 in pieces:
                    for g0, g1, g2, g3 in cells2(k, plane, lo[p], hi[p], q0, q1, h, "conductor", toward):
                        rows.append((k, (plane, g0, g1, g2, g3), KIND_CONDUCTOR, int(c), a, -1, sgn))
    for k in range(3):
        p, q = [x for x in range(3) if x != k]
        for s in (0, 1):
            plane = stack.hi[k] if s else stack.lo[k]
            sgn = 1 if s else -1
            bc = stack.face_bc[2 * k + s]
            if k == 2:
                a = R - 1 if s else 0
                for g0, g1, g2, g3 in cells2(k, plane, stack.lo[p], stack.hi[p], stack.lo[q], stack.hi[q], h_out,
                                             "conductor"):
                    rows.append((k, (plane, g0, g1, g2, g3), KIND_FACE, bc, a, -1, sgn))
            else:
                # q == 2 for k in {0, 1}: the face is cut at every layer plane
                for a in range(R):
                    for g0, g1, g2, g3 in cells2(k, plane, stack.lo[p], stack.hi[p], stack.z[a], stack.z[a + 1],
                                                 h_out, "conductor"):
                        rows.append((k, (plane, g0, g1, g2, g3), KIND_FACE, bc, a, -1, sgn))
    for a in range(1, R):
        za = stack.z[a]
        holes = [(lo, hi) for lo, hi, c in fboxes if lo[2] < za < hi[2]]
        # the interface is cut along the footprints of the conductors that
        # cross it; cells inside a footprint are holes
        bx = sorted({stack.lo[0], stack.hi[0]} | {v for lo, hi in holes for v in (lo[0], hi[0])})
        by = sorted({stack.lo[1], stack.hi[1]} | {v for lo, hi in holes for v in (lo[1], hi[1])})
        for i in range(len(bx) - 1):
            for j in range(len(by) - 1):
                cx, cy = 0.5 * (bx[i] + bx[i + 1]), 0.5 * (by[j] + by[j + 1])
                if any(lo[0] < cx < hi[0] and lo[1] < cy < hi[1] for lo, hi in holes):
                    continue
                for g0, g1, g2, g3 in cells2(2, za, bx[i], bx[i + 1], by[j], by[j + 1], h_out, "interface"):
                    rows.append((2, (za, g0, g1, g2, g3), KIND_INTERFACE, INTERFACE, a - 1, a, 1))
    return {
        "axis": np.array([r[0] for r in rows], dtype=np.int32),
        "geo": np.array([r[1] for r in rows], dtype=np.float64).reshape(-1, 5),
        "kind": np.array([r[2] for r in rows], dtype=np.int32),
        "cond": np.array([r[3] for r in rows], dtype=np.int32),
        "region_a": np.array([r[4] for r in rows], dtype=np.int32),
        "region_b": np.array([r[5] for r in rows], dtype=np.int32),
        "sign": np.array([r[6] for r in rows], dtype=np.int32),
    }


# --------------------------------------------------------------------------
# The system of Sec. 4
# --------------------------------------------------------------------------

def layout(mesh):
    """Rows and columns of the system.

    Rows: for each region a = 0, 1, ... the panels of its boundary in panel
    order.  Columns: for each panel in order, its unknown potential u (NEUMANN
    faces and interfaces) and then its unknown flux q (every panel except
    NEUMANN faces; on an interface the flux of the lower layer).  Returns
    (rows [(a, i)], ucol int[n] (-1: u known), qcol int[n] (-1: q known),
    conductor ids in right-hand-side order)."""
    cond, ra, rb = mesh["cond"], mesh["region_a"], mesh["region_b"]
    n = len(cond)
    R = int(max(ra.max(), rb.max())) + 1
    rows = [(a, i) for a in range(R) for i in range(n) if ra[i] == a or rb[i] == a]
    ucol = np.full(n, -1, dtype=np.int64)
    qcol = np.full(n, -1, dtype=np.int64)
    col = 0
    for i in range(n):
        if cond[i] in (NEUMANN, INTERFACE):
            ucol[i] = col
            col += 1
        if cond[i] != NEUMANN:
            qcol[i] = col
            col += 1
    ids = np.unique(cond[cond >= 0])
    return rows, ucol, qcol, ids


def system(mesh, eps, nthreads: int = 0):
    """Matrix M (n_eq x n_eq) and right-hand sides B (n_eq x n_c, column m:
    conductor ids[m] at 1 V, every other conductor and GROUND at 0 V) of the
    equations of Sec. 4, in the layout of ``layout``."""
    axis, geo, cond = mesh["axis"], mesh["geo"], mesh["cond"]
    ra, rb, sign = mesh["region_a"], mesh["region_b"], mesh["sign"]
    rows, ucol, qcol, ids = layout(mesh)
    n_eq = len(rows)
    if n_eq != int(max(ucol.max(), qcol.max())) + 1:
        raise ValueError("the stack's system is not square")
    area = O.areas(geo)
    eps = [float(e) for e in eps]
    M = np.zeros((n_eq, n_eq))
    B = np.zeros((n_eq, len(ids)))
    colof = {int(c): m for m, c in enumerate(ids)}
    R = len(eps)
    for a in range(R):
        P = np.nonzero((ra == a) | (rb == a))[0]
        I = np.repeat(P, len(P))
        J = np.tile(P, len(P))
        U = slayer_entries(axis, geo, I, J, nthreads).reshape(len(P), len(P))
        D = dlayer_entries(axis, geo, I, J, nthreads).reshape(len(P), len(P))
        r0 = [r for r, (aa, _) in enumerate(rows) if aa == a][0]
        for li, i in enumerate(P):
            r = r0 + li
            for lk, k in enumerate(P):
                own = ra[k] == a
                s = sign[k] if own else -sign[k]
                cu = (0.5 * area[i] if i == k else 0.0) + s * D[li, lk]
                g = 1.0 if own else -eps[ra[k]] / eps[a]
                cq = -U[li, lk] * g
                if ucol[k] >= 0:
                    M[r, ucol[k]] = cu
                elif cond[k] >= 0:
                    B[r, colof[int(cond[k])]] -= cu
                if qcol[k] >= 0:
                    M[r, qcol[k]] = cq
    return M, B, ids


def charges(mesh, eps, X, ids):
    """Maxwell capacitance matrix in farads from the solution X: the charge
    on conductor ids[n] for the right-hand side m is
    eps0 * 1e-6 * sum over its panels of eps_a q_j |I_j| (lengths in um)."""
    cond, ra, geo = mesh["cond"], mesh["region_a"], mesh["geo"]
    _, _, qcol, _ = layout(mesh)
    area = O.areas(geo)
    C = np.zeros((len(ids), X.shape[1]))
    for nidx, c in enumerate(ids):
        P = np.nonzero(cond == c)[0]
        w = np.array([eps[ra[j]] * area[j] for j in P])
        C[nidx] = O.EPS0 * 1e-6 * (w @ X[qcol[P]])
    return C


def capacitance(mesh, eps, nthreads: int = 0):
    """C (farads), with M and B, by LU with partial pivoting."""
    import scipy.linalg as sla
    M, B, ids = system(mesh, eps, nthreads)
    X = sla.lu_solve(sla.lu_factor(M, check_finite=True), B)
    return charges(mesh, eps, X, ids), ids


def plate_capacitance_1d(area: float, d, eps) -> float:
    """Capacitance of a stack of dielectric slabs between two plates that
    cover its whole cross-section (the field is normal to the layers):
    eps0 * area / sum_a (d_a / eps_a), lengths in um."""
    return O.EPS0 * 1e-6 * area / sum(da / ea for da, ea in zip(d, eps))


def square_solid_angle(a: float, w: float) -> float:
    """Solid angle of a square of side 2a seen from the point at height w
    above its centre: 4 atan(a^2 / (w sqrt(2 a^2 + w^2)))."""
    return 4.0 * math.atan(a * a / (w * math.sqrt(2.0 * a * a + w * w)))
