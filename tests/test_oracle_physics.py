"""Physical pins for the oracle's capacitance chain (Sec. 3.1-3.2):
variational bounds and monotone convergence of the Galerkin solution, the
Maxwell sign pattern, the parallel-plate limit and the sphere."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

HERE = os.path.dirname(__file__)
GOLD = json.load(open(os.path.join(HERE, "golden", "reference_values.json")))
FOUR_PI_EPS0_UM = 4 * math.pi * O.EPS0 * 1e-6   # F per um


def _cap(boxes, params, eps_r=1.0):
    a, g, c = O.mesh_boxes(boxes, **params)
    return O.capacitance(a, g, c, eps_r), len(a)


def test_cube_converges_from_below():
    ref = GOLD["unit_cube_capacitance_over_4pi_eps_a"]["value"]
    vals = []
    for n in (2, 4, 8):
        C, _ = _cap(*W.cube(1.0, n))
        vals.append(C[0, 0] / FOUR_PI_EPS0_UM)
    # Galerkin on nested subspaces: monotone increase toward the exact value
    assert vals[0] < vals[1] < vals[2] < ref
    # convergence: successive differences shrink
    assert (vals[2] - vals[1]) < (vals[1] - vals[0])
    assert ref - vals[2] < 0.01 * ref


def test_maxwell_pattern_two_bars():
    C, n = _cap(*W.two_bars(), eps_r=3.9)
    assert n == 608
    assert C[0, 0] > 0 and C[1, 1] > 0
    assert C[0, 1] < 0 and C[1, 0] < 0
    assert abs(C[0, 1] - C[1, 0]) <= 1e-12 * abs(C[0, 1])
    # free space: every row sum (the charge with all conductors at 1 V) is positive
    assert np.all(C.sum(axis=1) > 0)
    # by symmetry of the geometry the two self capacitances agree
    assert C[0, 0] == pytest.approx(C[1, 1], rel=1e-10)
    # parallel-plate lower bound for the facing 1.0 x 0.2 faces at 0.1 um
    eps = 3.9 * O.EPS0 * 1e-6
    assert -C[0, 1] > eps * 1.0 * 0.2 / 0.1


def test_galerkin_loewner_monotone_under_nested_refinement():
    boxes, _ = W.two_bars()
    Ch, _ = _cap(boxes, dict(h=0.1, ratio=1.0, h_min=0.0))
    Ch2, _ = _cap(boxes, dict(h=0.05, ratio=1.0, h_min=0.0))
    ev = np.linalg.eigvalsh(Ch2 - Ch)
    assert ev.min() > -1e-12 * np.abs(Ch).max()
    assert ev.max() > 0


def test_parallel_plate_limit():
    ratios = []
    for g in (0.2, 0.1):
        C, _ = _cap(*W.parallel_plates(L=1.0, t=0.02, g=g, h=0.1))
        eps = O.EPS0 * 1e-6
        ratios.append(-C[0, 1] * g / (eps * 1.0))
    # fringing makes the coupling larger than the ideal plate value, and the
    # excess shrinks as the gap closes
    assert ratios[0] > ratios[1] > 1.0


def test_sphere_bracketed_by_staircases():
    """Capacitance grows with the conductor (set inclusion), so the staircase
    of voxels inside the ball and the one covering it bracket 4 pi eps R; the
    Galerkin value of the inner one lies further below.  The bracket narrows
    as the voxels shrink."""
    R = 1.0
    exact = FOUR_PI_EPS0_UM * R
    gaps = []
    for nv in (2, 4):
        vals = []
        for outer in (False, True):
            a, g, c = W.voxel_sphere_panels(R, nv, outer)
            C = O.capacitance(np.array(a), np.array(g), np.array(c), 1.0)
            vals.append(C[0, 0] / exact)
        assert vals[0] < 1.0 < vals[1]
        gaps.append(vals[1] - vals[0])
    assert gaps[1] < gaps[0]
