"""Host side of the flat-triangle path: a triangle mesh keeps its vertices
and conductor ids, and malformed triangles and rectangle-only calls are
refused.  No GPU is touched."""
import numpy as np
import pytest

from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem, workloads as W


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gbem.load()


def test_triangle_mesh_round_trip_and_guards(lib):
    ctx = gbem.Context(device=-1, torch_alloc=False)
    tris = W.icosphere(2.0, 1)
    cond = np.r_[np.full(40, 7), np.full(40, 3)].astype(np.int32)
    m = ctx.mesh_from_triangles(tris, cond)
    assert (m.n, m.n_cond) == (80, 2)
    t, c = m.triangles()
    assert np.array_equal(t, tris) and np.array_equal(c, cond)
    with pytest.raises(gbem.GbemError) as e:
        m.panels()                                     # no rectangles
    assert e.value.status == -8
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh_from_triangles([[0, 0, 0, 1, 0, 0, 2, 0, 0]], [0])   # collinear: zero area
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh_from_triangles([[0, 0, 0, 1, 0, 0, 0, np.nan, 0]], [0])
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:
        m.assemble(gbem.GBEM_FP64, stream=0)           # a host context cannot assemble
    assert e.value.status == -9
    m.close()
    ctx.close()


def test_icosphere_is_inscribed_and_closed():
    tris = W.icosphere(1.5, 2, centre=(1.0, -2.0, 0.5)).reshape(-1, 3, 3)
    assert len(tris) == 320
    r = np.linalg.norm(tris - np.array([1.0, -2.0, 0.5]), axis=2)
    assert np.allclose(r, 1.5, rtol=1e-14)
    # outward orientation, and every edge shared by exactly two triangles
    c = tris.mean(axis=1) - np.array([1.0, -2.0, 0.5])
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert np.all(np.einsum("ij,ij->i", n, c) > 0)
    edges = {}
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            key = tuple(sorted((tuple(np.round(t[a], 12)), tuple(np.round(t[b], 12)))))
            edges[key] = edges.get(key, 0) + 1
    assert set(edges.values()) == {2}


def test_trapezoid_bar_is_closed_and_outward():
    tris = W.trapezoid_bar(0.0, 4.0, 1.0, 0.6, 0.0, 0.5, n_len=8, n_w=3, n_h=2).reshape(-1, 3, 3)
    edges = {}
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            key = (tuple(t[a]), tuple(t[b]))
            edges[key] = edges.get(key, 0) + 1
    # every directed edge once, its reverse once: closed and consistently oriented
    assert all(v == 1 and edges.get((b, a), 0) == 1 for (a, b), v in edges.items())
    volume = sum(np.dot(t[0], np.cross(t[1] - t[0], t[2] - t[0])) / 6.0 for t in tris)
    assert volume == pytest.approx(4.0 * 0.5 * (1.0 + 0.6) / 2.0, rel=1e-12)
