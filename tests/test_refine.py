"""Error-driven refinement (Sec. 3.2, Proposition "error": a net's charge
error is bounded by C sup_j |I_j| sup |dq/dtau| on I_j).  The library's
refinement (host side, no GPU) against the oracle's separately written one on
seeded densities, its invariants, and a physical pin of the indicator: on a
cube the density is singular along the edges, so the panels it marks first
are the ones on the edges."""
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


def _density(geo, seed):
    """A seeded field: smooth (distance to a random point) plus noise."""
    rng = np.random.default_rng(seed)
    x0 = rng.uniform(-0.5, 1.0, 3)
    ctr = np.stack([geo[:, 0], 0.5 * (geo[:, 1] + geo[:, 2]), 0.5 * (geo[:, 3] + geo[:, 4])], axis=1)
    return 1.0 / (0.05 + np.linalg.norm(ctr - x0, axis=1)) + 0.1 * rng.standard_normal(len(geo))


@pytest.mark.parametrize("name", ["two_bars", "crossing_bus_2x2"])
@pytest.mark.parametrize("theta", [0.0, 0.35, 0.8, 1.0])
def test_library_refinement_equals_oracle(ctx, name, theta):
    boxes, params = getattr(W, name)()
    mesh = ctx.mesh(boxes, params)
    a, g, c, _ = mesh.panels()
    dens = _density(g, seed=len(a) + int(100 * theta))
    ref_a, ref_g, ref_c, ref_eta, ref_m = O.refine(a, g, c, dens, theta)
    new, eta, marked = gbem.gbem_mesh_refine(mesh, dens, theta)
    assert marked == ref_m
    assert np.allclose(eta, ref_eta, rtol=1e-12, atol=0.0)
    na, ng, nc, _ = new.panels()
    assert new.n == len(ref_a) == mesh.n + marked
    assert _key(na, ng, nc) == _key(ref_a, ref_g, ref_c)
    new.close()
    mesh.close()


def test_refinement_invariants(ctx):
    boxes, params = W.two_bars()
    mesh = ctx.mesh(boxes, params)
    a, g, c, _ = mesh.panels()
    area = lambda geo, cond, k: float(np.sum(((geo[:, 2] - geo[:, 1]) * (geo[:, 4] - geo[:, 3]))[cond == k]))
    # theta = 0: every panel halved, every conductor keeps its area
    d = _density(g, 3)
    new, eta, marked = gbem.gbem_mesh_refine(mesh, d, 0.0)
    na, ng, nc, _ = new.panels()
    assert marked == mesh.n and new.n == 2 * mesh.n
    for k in np.unique(c):
        assert abs(area(ng, nc, k) - area(g, c, k)) <= 1e-12 * area(g, c, k)
    new.close()
    # theta = 1: only the panels with the largest indicator
    new, eta, marked = gbem.gbem_mesh_refine(mesh, d, 1.0)
    assert marked == int(np.sum(eta == eta.max())) >= 1
    new.close()
    # a constant density has no derivative: nothing to refine
    new, eta, marked = gbem.gbem_mesh_refine(mesh, np.full(mesh.n, 2.5), 0.5)
    assert marked == 0 and new.n == mesh.n and np.all(eta == 0.0)
    new.close()
    with pytest.raises(gbem.GbemError):
        gbem.gbem_mesh_refine(mesh, d, 1.5)
    mesh.close()


def test_indicator_marks_the_edges_of_a_cube():
    """Unit cube, 4 x 4 panels a face, its own charge density from the
    oracle's solve: the density is singular along the edges, so every panel
    on an edge of the cube gets a larger indicator than every face-centre
    panel, and theta = 0.9 marks exactly the 72 edge panels, in both
    implementations."""
    boxes, params = W.cube(1.0, 4)
    a, g, c = O.mesh_boxes(boxes, **params)
    A = O.assemble(a, g)
    X = O.solve(A, O.rhs(c)[0])[:, 0]
    dens = X / O.areas(g)
    _, _, _, eta, marked = O.refine(a, g, c, dens, 0.9)
    on_edge = np.array([min(gi[1], 1 - gi[2], gi[3], 1 - gi[4]) < 1e-12 for gi in g])
    assert np.sum(on_edge) == 72 and np.sum(~on_edge) == 24
    assert eta[on_edge].min() > eta[~on_edge].max()
    assert marked == 72
