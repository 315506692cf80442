"""The paper's distance-graded partition (Sec. 3.3): the library's mesher
(host side, no GPU) against the oracle's separately written one, panel for
panel, and the rule itself checked on the panels it makes."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem, workloads as W


@pytest.fixture(scope="module")
def ctx():
    B.build()
    c = gbem.Context(device=-1, torch_alloc=False)
    yield c
    c.close()


def _key(a, g, c):
    return sorted((int(a[i]), int(c[i])) + tuple(np.round(g[i], 12)) for i in range(len(a)))


CASES = [
    # (structure, main net, p1, p2, p3, p5, h_max)
    ("two_bars", 0, 0.004, 4.0, 1.0, 0.1, 0.0),
    ("two_bars", 1, 0.002, 2.0, 1.5, 0.05, 0.08),
    ("crossing_bus_2x2", 2, 0.0009, 4.0, 1.0, 0.1, 0.0),
    ("bus_3layer_5x5x5", 7, 0.004, 4.0, 1.0, 0.15, 0.2),
]


@pytest.mark.parametrize("case", CASES)
def test_library_mesher_equals_oracle_mesher(ctx, case):
    name, main, p1, p2, p3, p5, hmax = case
    boxes, _ = getattr(W, name)()
    a, g, c = O.mesh_graded(boxes, main, p1, p2, p3, p5, hmax)
    mesh = gbem.gbem_mesh_graded(ctx, boxes, main, p1, p2, p3, p5, hmax)
    pa, pg, pc, _ = mesh.panels()
    assert mesh.n == len(a)
    assert _key(pa, pg, pc) == _key(a, g, c)
    mesh.close()


def test_paper_table2_partition_with_enclosure(ctx):
    """The Sec. 5 parameters (near 1.5 um^2 within 1 um, 1.5 d^3 beyond, four
    times that on back faces) on the Table 2 geometry with its grounded box."""
    nets, box = W.paper_two_bars()
    a, g, c = O.mesh_graded(nets, 0, 1.5, 4.0, 1.0, 1.0, 0.0, enclosure=box)
    mesh = gbem.gbem_mesh_graded(ctx, nets, 0, 1.5, 4.0, 1.0, 1.0, 0.0, enclosure=box)
    pa, pg, pc, _ = mesh.panels()
    assert _key(pa, pg, pc) == _key(a, g, c)
    assert set(np.unique(c)) == {0, 1, 2}
    mesh.close()


def test_rule_holds_and_is_tight():
    """Every panel meets its bound; its parent (twice as large across the
    split edge) would not, unless the panel is a whole face."""
    boxes, _ = W.crossing_bus_2x2()
    main, p1, p2, p3, p5 = 1, 0.0009, 4.0, 1.0, 0.1
    a, g, c = O.mesh_graded(boxes, main, p1, p2, p3, p5)
    mains = [(lo, hi) for lo, hi, cc in boxes if cc == main]
    mlo = [min(b[0][d] for b in mains) for d in range(3)]
    mhi = [max(b[1][d] for b in mains) for d in range(3)]

    def dist(lo, hi):
        return min(math.sqrt(sum(max(0.0, bl[d] - hi[d], lo[d] - bh[d]) ** 2 for d in range(3)))
                   for bl, bh in mains)

    n_tight = 0
    for i in range(len(a)):
        k = int(a[i])
        p, q = [x for x in range(3) if x != k]
        lo, hi = [0.0] * 3, [0.0] * 3
        lo[k] = hi[k] = g[i, 0]
        lo[p], hi[p], lo[q], hi[q] = g[i, 1], g[i, 2], g[i, 3], g[i, 4]
        d = dist(lo, hi)
        # the face the panel lies on, and whether it looks toward the main net
        face = [(blo, bhi, cc) for blo, bhi, cc in boxes
                if (blo[k] == g[i, 0] or bhi[k] == g[i, 0]) and blo[p] <= lo[p] and hi[p] <= bhi[p]
                and blo[q] <= lo[q] and hi[q] <= bhi[q]]
        assert face
        blo, bhi, cc = face[0]
        outward_plus = bhi[k] == g[i, 0]
        toward = cc == main or (mhi[k] > g[i, 0] if outward_plus else mlo[k] < g[i, 0])
        p4 = p1 if toward else p1 * p2
        limit = p4 if d < p5 else p4 * p3 * (d / p5) ** 3
        area = (g[i, 2] - g[i, 1]) * (g[i, 4] - g[i, 3])
        assert area <= limit * (1 + 1e-12)
        n_tight += area > limit / 2.5
    assert n_tight > len(a) // 4   # bisection leaves panels within a factor 2-4 of their bound


def test_grading_follows_distance():
    """Panels near the main net are small, far ones large: the mean panel area
    grows with the distance band."""
    boxes, _ = W.bus_3layer_5x5x5()
    a, g, c = O.mesh_graded(boxes, 7, 0.002, 4.0, 1.0, 0.15)
    main = [(lo, hi) for lo, hi, cc in boxes if cc == 7]
    cent = np.column_stack([np.zeros(len(a))] * 3)
    for i in range(len(a)):
        k = int(a[i])
        p, q = [x for x in range(3) if x != k]
        cent[i, k] = g[i, 0]
        cent[i, p] = 0.5 * (g[i, 1] + g[i, 2])
        cent[i, q] = 0.5 * (g[i, 3] + g[i, 4])
    lo, hi = np.array(main[0][0]), np.array(main[0][1])
    d = np.linalg.norm(np.maximum(0.0, np.maximum(lo - cent, cent - hi)), axis=1)
    area = (g[:, 2] - g[:, 1]) * (g[:, 4] - g[:, 3])
    near = area[d < 0.15].mean()
    far = area[d > 0.6].mean()
    assert far > 8 * near
