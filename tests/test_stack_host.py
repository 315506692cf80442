"""Host side of the multi-dielectric path (Sec. 4): the library's stack mesher
builds the same panels, regions and normals as the oracle's, in the same
order, and lays out a square system of the same size; malformed stacks are
refused.  No GPU is touched."""
import numpy as np
import pytest

from oracle import dielectric as D
from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem

CASES = [
    # (lo, hi, z, eps, face_bc, boxes, h, h_outer)
    ([0, 0, 0], [4, 4, 3], [0, 1.5, 3], [1.0, 3.0], [D.GROUND] * 6,
     [([1, 1, 0.5], [2, 3, 1], 0), ([2.5, 1, 1.8], [3, 3, 2.5], 1)], 0.5, 1.0),
    ([0, 0, 0], [2, 2, 2], [0, 1, 2], [1.0, 4.0], [D.NEUMANN] * 4 + [D.GROUND, 0], [], 0.25, 0.0),
    ([-3, -2, 0], [3, 2, 2.5], [0, 0.7, 1.6, 2.5], [3.9, 2.2, 7.0], [D.NEUMANN] * 4 + [D.GROUND, D.GROUND],
     [([-2, -1, 0.2], [-0.5, 1, 0.5], 4), ([0.5, -1.5, 0.9], [2.5, -1.0, 1.3], 2), ([0.5, 1.0, 0.9], [2.5, 1.5, 1.3], 7)],
     0.3, 0.8),
]


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gbem.load()


def _ctx():
    return gbem.Context(device=-1, torch_alloc=False)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_stack_mesh_matches_oracle(lib, case):
    lo, hi, z, eps, bc, boxes, h, ho = CASES[case]
    ctx = _ctx()
    S = gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, h, ho)
    got = S.panels()
    ref = D.mesh_stack(D.Stack(lo, hi, z, eps, bc), boxes, h, ho)
    for k in ("axis", "kind", "cond", "region_a", "region_b", "sign"):
        assert np.array_equal(got[k].astype(np.int64), ref[k].astype(np.int64)), k
    assert np.array_equal(got["geo"], ref["geo"])
    rows, ucol, qcol, ids = D.layout(ref)
    assert S.n_eq == len(rows)
    assert np.array_equal(got["cond_ids"], ids)
    S.close()
    ctx.close()


VIA_CASES = [
    ([0, 0, 0], [4, 4, 3], [0, 1.5, 3], [1.0, 3.0], [D.GROUND] * 6,
     [([1.5, 1.5, 0.8], [2.0, 2.0, 2.2], 0), ([0.5, 2.8, 0.5], [3.5, 3.3, 1.0], 1)], 0.5, 1.0, None),
    ([-3, -2, 0], [3, 2, 2.5], [0, 0.7, 1.6, 2.5], [3.9, 2.2, 7.0], [D.NEUMANN] * 4 + [D.GROUND, D.GROUND],
     [([-0.3, -0.3, 0.3], [0.3, 0.3, 2.2], 4), ([1.0, -1.5, 0.9], [2.5, -1.0, 1.3], 2)], 0.3, 0.8, None),
    ([-3, -2, 0], [3, 2, 2.5], [0, 0.7, 1.6, 2.5], [3.9, 2.2, 7.0], [D.NEUMANN] * 4 + [D.GROUND, D.GROUND],
     [([-0.3, -0.3, 0.3], [0.3, 0.3, 2.2], 4), ([1.0, -1.5, 0.9], [2.5, -1.0, 1.3], 2)], 0.3, 0.8,
     (4, 0.05, 4.0, 1.0, 0.5)),
]


@pytest.mark.parametrize("case", range(len(VIA_CASES)))
def test_vias_match_oracle(lib, case):
    """Conductors crossing layer planes: the same panels in the library and
    the oracle, uniform and graded."""
    lo, hi, z, eps, bc, boxes, h, ho, graded = VIA_CASES[case]
    ctx = _ctx()
    S = gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, h, ho, graded=graded)
    got = S.panels()
    ref = D.mesh_stack(D.Stack(lo, hi, z, eps, bc), boxes, h, ho, graded=graded)
    for k in ("axis", "kind", "cond", "region_a", "region_b", "sign"):
        assert np.array_equal(got[k].astype(np.int64), ref[k].astype(np.int64)), k
    assert np.array_equal(got["geo"], ref["geo"])
    assert S.n_eq == len(D.layout(ref)[0])
    S.close()
    ctx.close()


def test_stack_guards(lib):
    ctx = _ctx()
    lo, hi, z, eps, bc = [0, 0, 0], [4, 4, 3], [0, 1.5, 3], [1.0, 3.0], [D.GROUND] * 6
    bad_boxes = [
        [([1, 1, 1.5], [2, 2, 2.0], 0)],                              # bottom on a layer plane
        [([0, 1, 0.5], [2, 2, 1.0], 0)],                              # touches the enclosure
        [([1, 1, 0.5], [2, 2, 1.0], 0), ([2, 1, 0.5], [3, 2, 1.0], 1)],  # boxes touch
    ]
    for boxes in bad_boxes:
        with pytest.raises(gbem.GbemError) as e:
            gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, 0.5)
        assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:   # no conductor at all
        gbem.Stack(ctx, lo, hi, z, eps, bc, [], 0.5)
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:   # planes do not span the enclosure
        gbem.Stack(ctx, lo, hi, [0, 1.5, 2.9], eps, bc, [([1, 1, 0.5], [2, 3, 1], 0)], 0.5)
    assert e.value.status == -1
    with pytest.raises(gbem.GbemError) as e:   # non-positive permittivity
        gbem.Stack(ctx, lo, hi, z, [1.0, 0.0], bc, [([1, 1, 0.5], [2, 3, 1], 0)], 0.5)
    assert e.value.status == -1
    S = gbem.Stack(ctx, lo, hi, z, eps, bc, [([1, 1, 0.5], [2, 3, 1], 0)], 0.5)
    with pytest.raises(gbem.GbemError) as e:   # a host context cannot assemble
        S.assemble(gbem.GBEM_FP64, stream=0)
    assert e.value.status == -9
    with pytest.raises(gbem.GbemError) as e:   # nothing assembled to download
        S.system()
    assert e.value.status == -8
    with pytest.raises(gbem.GbemError) as e:   # no device to solve on
        S.capacitance(stream=0)
    assert e.value.status == -9
    with pytest.raises(gbem.GbemError) as e:   # a graded stack needs its main conductor
        gbem.Stack(ctx, lo, hi, z, eps, bc, [([1, 1, 0.5], [2, 3, 1], 0)], 0.5, graded=(5, 0.1, 4.0, 1.0, 1.0))
    assert e.value.status == -1
    S.close()
    ctx.close()


def test_graded_stack_matches_oracle_and_bounds(lib):
    """The paper's partition on a stack (Sec. 3.3 for conductors and the
    enclosure, Sec. 4 for interfaces): the library and the oracle build the
    same panels, and every panel meets its bound."""
    lo, hi, z, eps, bc = [-8, -8, 0], [8, 8, 4], [0, 1.5, 2.5, 4], [3.9, 2.5, 7.0], [D.NEUMANN] * 4 + [D.GROUND] * 2
    boxes = [([-1.5, -0.25, 1.75], [1.5, 0.25, 2.25], 0), ([-1.5, 0.75, 1.75], [1.5, 1.25, 2.25], 1),
             ([3.0, -3.0, 0.4], [3.5, 3.0, 0.9], 2)]
    main, p1, p2, p3, p5 = 0, 0.1, 4.0, 1.0, 1.0
    ctx = _ctx()
    S = gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, 0.5, 4.0, graded=(main, p1, p2, p3, p5))
    got = S.panels()
    ref = D.mesh_stack(D.Stack(lo, hi, z, eps, bc), boxes, 0.5, 4.0, graded=(main, p1, p2, p3, p5))
    for k in ("axis", "kind", "cond", "region_a", "region_b", "sign"):
        assert np.array_equal(got[k].astype(np.int64), ref[k].astype(np.int64)), k
    assert np.array_equal(got["geo"], ref["geo"])
    # bounds: distance to the main net's box, area limit by kind
    mlo, mhi = np.array(boxes[0][0], float), np.array(boxes[0][1], float)
    g, ax = ref["geo"], ref["axis"]
    for i in range(len(ax)):
        k = ax[i]
        p, q = [x for x in range(3) if x != k]
        plo, phi = np.zeros(3), np.zeros(3)
        plo[k] = phi[k] = g[i, 0]
        plo[p], phi[p], plo[q], phi[q] = g[i, 1], g[i, 2], g[i, 3], g[i, 4]
        d = np.linalg.norm(np.maximum(0.0, np.maximum(mlo - phi, plo - mhi)))
        area = (g[i, 2] - g[i, 1]) * (g[i, 4] - g[i, 3])
        power = 2 if ref["kind"][i] == D.KIND_INTERFACE else 3
        limit_far = p1 * p2 * p3 * max(1.0, d / p5) ** power   # the looser p4 of faces looking away
        assert area <= (p1 * p2 if d < p5 else limit_far) * (1 + 1e-12)
        assert max(g[i, 2] - g[i, 1], g[i, 4] - g[i, 3]) <= (0.5 if ref["kind"][i] == D.KIND_CONDUCTOR else 4.0) + 1e-12
    # the grading coarsens with distance: interface panels far from the net are larger
    itf = ref["kind"] == D.KIND_INTERFACE
    areas = (g[itf, 2] - g[itf, 1]) * (g[itf, 4] - g[itf, 3])
    assert areas.max() > 20 * areas.min()
    S.close()
    ctx.close()
