"""Pins of the multi-dielectric oracle (Sec. 4) against facts that do not come
from the oracle itself: the textbook solid angle of a square, Gauss's theorem
for the double-layer kernel on closed surfaces, the antisymmetry of that
kernel between parallel panels, the algebraic equality of the direct
formulation of Sec. 4 and the indirect one of Sec. 3 when every boundary value
is given, the exact capacitance of layered plates whose field is
one-dimensional, and the linearity of C in the permittivities."""
import math

import numpy as np
import pytest

from oracle import dielectric as D
from oracle import oracle as O


def two_layer_stack(bc=D.GROUND):
    return D.Stack([0, 0, 0], [4, 4, 3], [0, 1.5, 3], [1.0, 3.0], [bc] * 6)


BOXES = [([1, 1, 0.5], [2, 3, 1], 0), ([2.5, 1, 1.8], [3, 3, 2.5], 1)]


def test_square_solid_angle():
    # a square of side 2 seen from its axis: 4 asin(a^2 / (a^2 + w^2)), a = 1
    g = [0.0, -1.0, 1.0, -1.0, 1.0]
    for w in (0.05, 0.3, 1.0, 5.0, 40.0):
        ref = 4.0 * math.asin(1.0 / (1.0 + w * w))
        assert D.rect_dlayer(2, g, [0.0, 0.0, w]) == pytest.approx(ref, rel=1e-13)
        assert D.rect_dlayer(2, g, [0.0, 0.0, -w]) == pytest.approx(-ref, rel=1e-13)
    assert D.rect_dlayer(2, g, [3.0, 0.5, 0.0]) == 0.0
    # just above the middle of the panel the solid angle tends to 2 pi
    assert D.rect_dlayer(2, g, [0.1, -0.2, 1e-9]) == pytest.approx(2 * math.pi, rel=1e-8)


def test_gauss_identity_on_every_region():
    """int_{dOmega} q*(x, y) dy = -1/2 for x on the boundary of a region (Sec.
    2's representation formula with u = 1): every row of every region's block
    satisfies |I_i|/2 + sum_k s_k d_ik = 0."""
    st = two_layer_stack()
    m = D.mesh_stack(st, BOXES, 0.5, 1.0)
    ra, rb, sg = m["region_a"], m["region_b"], m["sign"]
    area = O.areas(m["geo"])
    for a in range(2):
        P = np.nonzero((ra == a) | (rb == a))[0]
        I, J = np.repeat(P, len(P)), np.tile(P, len(P))
        Dm = D.dlayer_entries(m["axis"], m["geo"], I, J).reshape(len(P), len(P))
        s = np.where(ra[P] == a, sg[P], -sg[P])
        assert np.abs(Dm @ s + 0.5 * area[P]).max() <= 1e-13 * area[P].max()
        # antisymmetry between parallel panels, zeros between coplanar ones
        ax, c = m["axis"][P], m["geo"][P, 0]
        par = ax[:, None] == ax[None, :]
        assert np.abs((Dm + Dm.T)[par]).max() <= 1e-15 * area[P].max()
        assert np.all(Dm[par & (c[:, None] == c[None, :])] == 0.0)
    # a point outside a closed surface sees total solid angle 0: the
    # enclosure's panels against the faces of conductor 0 (outward normals)
    box = np.nonzero(m["cond"] == 0)[0]
    face = np.nonzero(m["kind"] == D.KIND_FACE)[0]
    I, J = np.repeat(face, len(box)), np.tile(box, len(face))
    Dm = D.dlayer_entries(m["axis"], m["geo"], I, J).reshape(len(face), len(box))
    assert np.abs(Dm @ (-m["sign"][box])).max() <= 1e-13 * area.max()


def test_single_region_direct_equals_indirect():
    """One dielectric and every boundary value given: the direct system of
    Sec. 4 and the single-layer system of Sec. 3 (enclosure as a grounded
    conductor) give the same charges, because the Galerkin double layer of a
    closed surface reproduces |I_i|/2 exactly."""
    st = D.Stack([0, 0, 0], [4, 4, 3], [0, 3], [2.5], [D.GROUND] * 6)
    boxes = [([1.5, 1.5, 1.0], [2.5, 2.5, 2.0], 0), ([0.5, 0.5, 0.5], [1.0, 3.5, 1.2], 1)]
    m = D.mesh_stack(st, boxes, 0.5, 1.0)
    Cd, ids = D.capacitance(m, st.eps)
    cond = np.where(m["cond"] >= 0, m["cond"], 9)
    Ci = O.capacitance(m["axis"], m["geo"], cond, 2.5)[:2, :2]
    assert list(ids) == [0, 1]
    assert np.abs(Cd - Ci).max() <= 1e-12 * np.abs(Ci).max()


def test_layered_plates_converge_to_one_dimensional_field():
    """Plates covering the whole cross-section of insulating side walls: the
    field is normal to the layers and C = eps0 A / sum d_a / eps_a."""
    st = D.Stack([0, 0, 0], [2, 2, 2], [0, 1, 2], [1.0, 4.0], [D.NEUMANN] * 4 + [D.GROUND, 0])
    ref = D.plate_capacitance_1d(4.0, [1.0, 1.0], [1.0, 4.0])
    err = []
    for h in (0.5, 0.25):
        C, ids = D.capacitance(D.mesh_stack(st, [], h), st.eps)
        assert list(ids) == [0]
        err.append(abs(C[0, 0] / ref - 1.0))
    assert err[1] < 0.04 and err[1] < 0.45 * err[0]


def test_permittivity_scaling_reciprocity_and_equal_layers():
    st = two_layer_stack()
    m = D.mesh_stack(st, BOXES, 0.5, 1.0)
    C, _ = D.capacitance(m, st.eps)
    C3, _ = D.capacitance(m, [3.0 * e for e in st.eps])
    assert np.abs(C3 - 3.0 * C).max() <= 1e-12 * np.abs(C).max()
    # Maxwell matrix: positive diagonal, negative coupling, nearly symmetric
    assert C[0, 0] > 0 and C[1, 1] > 0 and C[0, 1] < 0 and C[1, 0] < 0
    assert abs(C[0, 1] - C[1, 0]) < 0.02 * abs(C[0, 1])
    # an interface between equal permittivities changes C by discretisation only
    one = D.Stack([0, 0, 0], [4, 4, 3], [0, 3], [3.0], [D.GROUND] * 6)
    two = D.Stack([0, 0, 0], [4, 4, 3], [0, 1.5, 3], [3.0, 3.0], [D.GROUND] * 6)
    C1, _ = D.capacitance(D.mesh_stack(one, BOXES, 0.5, 1.0), one.eps)
    C2, _ = D.capacitance(D.mesh_stack(two, BOXES, 0.5, 1.0), two.eps)
    assert np.abs(C2 / C1 - 1.0).max() < 0.025


def test_stack_mesh_layout_and_guards():
    st = two_layer_stack(D.NEUMANN)
    m = D.mesh_stack(st, BOXES, 0.5, 1.0)
    rows, ucol, qcol, ids = D.layout(m)
    n_int = int(np.sum(m["kind"] == D.KIND_INTERFACE))
    # one row per (region, boundary panel): interfaces count twice
    assert len(rows) == len(m["axis"]) + n_int
    assert len(rows) == int(max(ucol.max(), qcol.max())) + 1
    assert np.all(ucol[m["cond"] == D.NEUMANN] >= 0) and np.all(qcol[m["cond"] == D.NEUMANN] < 0)
    assert np.all(qcol[m["cond"] >= 0] >= 0) and np.all(ucol[m["cond"] >= 0] < 0)
    # the panels tile every surface exactly
    area = O.areas(m["geo"])
    assert area[m["kind"] == D.KIND_INTERFACE].sum() == pytest.approx(16.0)
    assert area[m["kind"] == D.KIND_FACE].sum() == pytest.approx(2 * 16.0 + 4 * 12.0)
    with pytest.raises(ValueError):
        D.mesh_stack(st, [([1, 1, 1.5], [2, 2, 2.0], 0)], 0.5)   # bottom on the plane z = 1.5
    with pytest.raises(ValueError):
        D.mesh_stack(st, [([0, 1, 0.5], [2, 2, 1.0], 0)], 0.5)   # touches the enclosure


def test_via_through_an_interface():
    """A conductor crossing a layer plane (a via): its side faces are cut at
    the plane, the interface is holed along its footprint, every region's
    boundary stays closed (Gauss's theorem per region, as above), and C keeps
    the Maxwell pattern and near-symmetry."""
    st = D.Stack([0, 0, 0], [4, 4, 3], [0, 1.5, 3], [1.0, 3.0], [D.GROUND] * 6)
    boxes = [([1.5, 1.5, 0.8], [2.0, 2.0, 2.2], 0), ([0.5, 2.8, 0.5], [3.5, 3.3, 1.0], 1)]
    m = D.mesh_stack(st, boxes, 0.5, 1.0)
    ra, rb, sg, kind = m["region_a"], m["region_b"], m["sign"], m["kind"]
    area = O.areas(m["geo"])
    # the interface loses the via's footprint (0.25 um^2) and the via gains
    # side panels in both layers
    assert area[kind == D.KIND_INTERFACE].sum() == pytest.approx(16.0 - 0.25)
    via = (m["cond"] == 0) & (m["axis"] != 2)
    assert set(ra[via].tolist()) == {0, 1}
    for a in range(2):
        P = np.nonzero((ra == a) | (rb == a))[0]
        I, J = np.repeat(P, len(P)), np.tile(P, len(P))
        Dm = D.dlayer_entries(m["axis"], m["geo"], I, J).reshape(len(P), len(P))
        s = np.where(ra[P] == a, sg[P], -sg[P])
        assert np.abs(Dm @ s + 0.5 * area[P]).max() <= 1e-13 * area[P].max()
    C, _ = D.capacitance(m, st.eps)
    assert C[0, 0] > 0 and C[1, 1] > 0 and C[0, 1] < 0
    assert abs(C[0, 1] - C[1, 0]) < 0.03 * abs(C[0, 1])

