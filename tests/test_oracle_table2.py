"""The paper's own single-dielectric experiment (Sec. 5, Table 2) as a pin of
the oracle: two crossing 4 x 1 x 1 um bars inside a grounded 40 x 40 x 10 um
box.  The paper's capacitances converge to C11 = 226, C12 = -58.7 and
C22 = 179 aF (594 panels); Sun et al. (1997), quoted after the table, give
230 / -61 / 180.6 aF.  The permittivity is not stated; the magnitudes fit
eps_r = 1 (the reading recorded with the oracle).

The grounded box is the boundary of the domain (Sec. 3.1): its inner faces
carry unknown charges at potential 0.  The single-layer kernel does not
depend on panel orientation, so the faces are panels of a third conductor
held at 0 V in every solve, and C11, C12, C22 are the entries of the two
nets in the 3 x 3 Maxwell matrix.  The nets use uniform panels; the box
faces use tensor grids whose cells grow with the distance from the bars
(the charge on the walls spreads over microns, the bars' edges need tens of
nanometres only in their own faces).  Checked within the paper's 5 %
reading at two mesh levels.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

HERE = os.path.dirname(__file__)


def _graded(lo, hi, center, h0, growth, h_max):
    """1-D nodes on [lo, hi]: cells of h0 around `center`, growing by
    `growth` per cell away from it, capped at h_max."""
    def side(length):
        out, x, h = [0.0], 0.0, h0
        while x + h < length - 1e-9:
            x += h
            out.append(x)
            h = min(h * growth, h_max)
        if length - x < 0.3 * h and len(out) > 1:
            out.pop()
        out.append(length)
        return out
    left = [center - d for d in side(center - lo)][::-1]
    right = [center + d for d in side(hi - center)]
    return left[:-1] + right


def _face_panels(k, plane, n0, n1, cond):
    axis, geo, cid = [], [], []
    for a in range(len(n0) - 1):
        for b in range(len(n1) - 1):
            axis.append(k)
            geo.append((plane, n0[a], n0[a + 1], n1[b], n1[b + 1]))
            cid.append(cond)
    return axis, geo, cid


def table2_panels(h_net, h_wall, growth, h_max):
    nets, box = W.paper_two_bars()
    a, g, c = O.mesh_boxes(nets, h=h_net)
    axis, geo, cond = list(a), [tuple(r) for r in g], list(c)
    lo, hi, gid = box
    # x and y grids centred on the crossing; z grids from the bottom (the
    # bars sit 1 um above the bottom face and 6 um below the top)
    gx = _graded(lo[0], hi[0], 0.0, h_wall, growth, h_max)
    gy = _graded(lo[1], hi[1], 0.0, h_wall, growth, h_max)
    gz = _graded(lo[2], hi[2], 2.5, h_wall, growth, h_max)
    for k, (n0, n1) in enumerate(((gy, gz), (gx, gz), (gx, gy))):
        for plane in (lo[k], hi[k]):
            fa, fg, fc = _face_panels(k, plane, n0, n1, gid)
            axis += fa
            geo += fg
            cond += fc
    return np.array(axis, np.int32), np.array(geo, np.float64), np.array(cond, np.int32)


@pytest.fixture(scope="module")
def paper_values():
    ref = json.load(open(os.path.join(HERE, "golden", "reference_values.json")))
    t2 = ref["paper_table2_single_dielectric_aF"]
    return t2["C11"][-1], t2["C12"][-1], t2["C22"][-1]


@pytest.mark.slow
def test_table2_grounded_box_within_five_percent(paper_values):
    c11, c12, c22 = paper_values
    results = []
    for h_net, h_wall in ((0.25, 0.5), (0.2, 0.4)):
        a, g, c = table2_panels(h_net, h_wall, 1.35, 5.0)
        C = O.capacitance(a, g, c, 1.0) * 1e18   # aF; conductors 0, 1 = nets, 2 = box
        results.append((len(a), C))
        assert abs(C[0, 0] - c11) <= 0.05 * abs(c11), (len(a), C[0, 0])
        assert abs(C[0, 1] - c12) <= 0.05 * abs(c12), (len(a), C[0, 1])
        assert abs(C[1, 1] - c22) <= 0.05 * abs(c22), (len(a), C[1, 1])
        # reciprocity and the Maxwell pattern with the grounded box
        assert abs(C[0, 1] - C[1, 0]) <= 1e-9 * abs(C[0, 1])
        assert C[0, 0] > 0 and C[1, 1] > 0 and C[0, 1] < 0 and C[0, 2] < 0 and C[1, 2] < 0
    # refinement moves the values by well under the 5 % band
    (_, Ca), (_, Cb) = results
    assert np.max(np.abs(Ca[:2, :2] - Cb[:2, :2])) <= 0.02 * c11


def test_table2_with_the_papers_partition(paper_values):
    """Sec. 5's partition parameters (area 1.5 um^2 within 1 um of the main
    net, 1.5 d^3 beyond, four times that on faces turned away; Sec. 3.3) on
    the Table 2 geometry: with p1 scaled to give panel counts near the
    paper's 74 and 183, the oracle's C11, C12, C22 fall within 2 % of the
    values the paper prints for those counts, and within 5 % of its
    converged ones."""
    ref = json.load(open(os.path.join(HERE, "golden", "reference_values.json")))["paper_table2_single_dielectric_aF"]
    nets, box = W.paper_two_bars()
    for p1, n_paper_idx in ((3.0, 0), (0.75, 1)):
        a, g, c = O.mesh_graded(nets, 0, p1, 4.0, 1.0, 1.0, 0.0, enclosure=box)
        assert abs(len(a) - ref["panels"][n_paper_idx]) <= 0.15 * ref["panels"][n_paper_idx]
        C = O.capacitance(a, g, c, 1.0) * 1e18
        for got, key in ((C[0, 0], "C11"), (C[0, 1], "C12"), (C[1, 1], "C22")):
            printed = ref[key][n_paper_idx]
            assert abs(got - printed) <= 0.02 * abs(printed), (len(a), key, got, printed)
        c11, c12, c22 = paper_values
        assert abs(C[0, 0] - c11) <= 0.05 * c11 and abs(C[1, 1] - c22) <= 0.05 * c22
        assert abs(C[0, 1] - c12) <= 0.05 * abs(c12)
