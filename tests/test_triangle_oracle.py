"""Pins of the flat-triangle oracle against facts outside it: brute-force
quadrature of a triangle's potential, rectangles cut into triangles (the
rectangle oracle and its closed forms are pinned on their own), the published
closed form of a triangle's self-integral, scaling and translation, the
capacitance of a sphere approached from below by inscribed icospheres, the
variational bound under a refinement from rectangles to triangles, and a
trapezoid wire between the cuboids of its two widths."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import triangles as T
from paper_2203_11733_gb300 import workloads as W

TRI = [0.1, 0.2, 0.0, 1.3, -0.1, 0.2, 0.4, 0.9, -0.3]


def brute_potential(tri, x, n=40, levels=3):
    """int_T 1/|x - y| by the collapsed Gauss-Legendre rule of order n on the
    4**levels midpoint children of T (numpy's nodes)."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    tris = [np.asarray(tri, float).reshape(3, 3)]
    for _ in range(levels):
        nxt = []
        for a, b, c in tris:
            ab, bc, ca = (a + b) / 2, (b + c) / 2, (c + a) / 2
            nxt += [np.array(t) for t in ((a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca))]
        tris = nxt
    s = 0.0
    for a, b, c in tris:
        j2 = np.linalg.norm(np.cross(b - a, c - b))
        xi, eta = np.meshgrid(g, g, indexing="ij")
        y = a + xi[..., None] * ((b - a) + eta[..., None] * (c - b))
        r = np.linalg.norm(y - np.asarray(x, float), axis=-1)
        s += j2 * np.sum(np.outer(w, w) * xi / r)
    return s


def test_potential_matches_brute_force():
    for x in ([0.5, 0.3, 0.7], [0.5, 0.3, -0.2], [2.0, 1.0, 0.5], [1.5, -0.8, 0.25]):
        assert T.tri_potential(TRI, x) == pytest.approx(brute_potential(TRI, x), rel=1e-12)


def _raw(tris, i, j):
    a = T.tri_areas(tris)
    return T.tri_entries(tris, [i], [j])[0] * 4 * math.pi * a[i] * a[j]


def test_rectangles_cut_into_triangles():
    """int int over rectangles (rectangle oracle) = the sum over their
    triangles: self, coplanar neighbours and perpendicular neighbours."""
    sq = [[0, 0, 0, 1, 0, 0, 1, 1, 0], [0, 0, 0, 1, 1, 0, 0, 1, 0]]            # z = 0, [0,1]^2
    nb = [[1, 0, 0, 2, 0, 0, 2, 1, 0], [1, 0, 0, 2, 1, 0, 1, 1, 0]]            # z = 0, [1,2] x [0,1]
    wall = [[0, 0, 0, 0, 1, 0, 0, 1, 1], [0, 0, 0, 0, 1, 1, 0, 0, 1]]          # x = 0, [0,1]^2
    cases = [(sq, sq, (2, [0, 0, 1, 0, 1]), (2, [0, 0, 1, 0, 1])),
             (sq, nb, (2, [0, 0, 1, 0, 1]), (2, [0, 1, 2, 0, 1])),
             (sq, wall, (2, [0, 0, 1, 0, 1]), (0, [0, 0, 1, 0, 1]))]
    for A, B, ra, rb in cases:
        tris = A + B
        tot = sum(_raw(tris, i, 2 + j) for i in range(2) for j in range(2))
        ref = O.pair_integral(ra[0], ra[1], rb[0], rb[1])[0]
        assert tot == pytest.approx(ref, rel=2e-10)


def test_self_integral_closed_form():
    """int_T int_T 1/|x - y| = (4 |T|^2 / 3) sum over the sides l_i (with the
    next sides l_j, l_k in turn) of ln(((l_i + l_j)^2 - l_k^2) /
    (l_j^2 - (l_i - l_k)^2)) / l_i (the published closed form for a flat
    triangle's self-term)."""
    for tri in (TRI, [0, 0, 0, 1, 0, 0, 0, 1, 0], [0, 0, 0, 2, 0, 0, 1, math.sqrt(3), 0], [0, 0, 0, 5, 0, 0, 0.3, 0.4, 0]):
        p = np.asarray(tri, float).reshape(3, 3)
        A = T.tri_areas([tri])[0]
        l = [np.linalg.norm(p[1] - p[0]), np.linalg.norm(p[2] - p[1]), np.linalg.norm(p[0] - p[2])]
        s = sum(math.log(((l[i] + l[(i + 1) % 3]) ** 2 - l[(i + 2) % 3] ** 2) /
                         (l[(i + 1) % 3] ** 2 - (l[i] - l[(i + 2) % 3]) ** 2)) / l[i] for i in range(3))
        assert _raw([tri], 0, 0) == pytest.approx(4 * A * A / 3 * s, rel=1e-10)


def test_scaling_and_translation():
    tris = np.array([TRI, [1.3, -0.1, 0.2, 0.4, 0.9, -0.3, 1.5, 0.8, 0.1], [3.0, 3.0, 1.0, 4.0, 3.2, 1.1, 3.3, 4.0, 0.9]])
    I, J = [0, 0, 0, 1], [0, 1, 2, 2]
    base = T.tri_entries(tris, I, J)
    assert np.allclose(T.tri_entries(2.5 * tris, I, J), base / 2.5, rtol=1e-10, atol=0)
    assert np.allclose(T.tri_entries(tris + np.tile([7.0, -3.0, 2.0], 3), I, J), base, rtol=1e-10, atol=0)


def test_icosphere_capacitance_rises_toward_sphere():
    """Inscribed polyhedra: below 4 pi eps R and rising with refinement."""
    vals = []
    for level in (0, 1):
        tris = W.icosphere(1.0, level)
        C = T.tri_capacitance(tris, np.zeros(len(tris), np.int32), 1.0)
        vals.append(C[0, 0] / (4 * math.pi * O.EPS0 * 1e-6))
    assert vals[0] < vals[1] < 1.0 and vals[1] > 0.95


def _split(axis, geo):
    """Each axis-aligned rectangle cut along a diagonal into two triangles."""
    out = []
    for k, (c, a0, b0, a1, b1) in zip(axis, geo):
        p, q = [x for x in range(3) if x != k]
        corners = []
        for u, v in ((a0, a1), (b0, a1), (b0, b1), (a0, b1)):
            x = [0.0] * 3
            x[k], x[p], x[q] = c, u, v
            corners.append(x)
        out.append(corners[0] + corners[1] + corners[2])
        out.append(corners[0] + corners[2] + corners[3])
    return np.array(out)


def test_triangles_refine_rectangles():
    """Cutting every rectangle of a mesh into two triangles enlarges the
    Galerkin space, so the capacitance can only rise (variational bound), and
    only by the discretisation error."""
    a, g, c = O.mesh_boxes([([0, 0, 0], [2.0, 0.5, 0.25], 0)], 0.25)
    C_rect = O.capacitance(a, g, c, 1.0)[0, 0]
    tris = _split(a, g)
    C_tri = T.tri_capacitance(tris, np.zeros(len(tris), np.int32), 1.0)[0, 0]
    assert C_rect * (1 - 1e-12) <= C_tri < C_rect * 1.02


def test_trapezoid_wire_between_its_cuboids():
    """A wire of trapezoidal cross-section (the paper stacks cuboids for such
    shapes, Sec. 3.3; here flat triangles describe it exactly) has a
    capacitance between those of the cuboids of its top and bottom widths."""
    tris = W.trapezoid_bar(0.0, 2.0, 0.5, 0.25, 0.0, 0.25, n_len=8, n_w=2, n_h=2)
    C_trap = T.tri_capacitance(tris, np.zeros(len(tris), np.int32), 1.0)[0, 0]
    caps = []
    for w in (0.25, 0.5):
        a, g, c = O.mesh_boxes([([0, -w / 2, 0], [2.0, w / 2, 0.25], 0)], 0.125)
        caps.append(O.capacitance(a, g, c, 1.0)[0, 0])
    assert caps[0] < C_trap < caps[1]
