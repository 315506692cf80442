"""GPU path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 mode 1e-10 relative per matrix entry and 1e-9 relative on
capacitances; mixed mode (FP32 far field and factor, FP64 near field and
refinement) 1e-6 on both.  Capacitance errors are max |C - C_ref| / max |C_ref|.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(__file__)
ENTRY_TOL = {0: 1e-10, 1: 1e-6}
CAP_TOL = {0: 1e-9, 1: 1e-6}


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    B.build()
    c = gbem.Context(0)
    yield c
    c.close()


def _perm(mesh, oa, og, oc):
    pa, pg, pc, _ = mesh.panels()
    key = {}
    for i in range(len(oa)):
        key[(int(oa[i]), int(oc[i])) + tuple(np.round(og[i], 9))] = i
    return np.array([key[(int(pa[i]), int(pc[i])) + tuple(np.round(pg[i], 9))] for i in range(len(pa))])


def _rel(a, b):
    return np.abs(a - b) / np.abs(b)


def _cap_err(C, R):
    return float(np.max(np.abs(C - R)) / np.max(np.abs(R)))


@pytest.fixture(scope="module")
def two_bars_oracle():
    boxes, params = W.two_bars()
    a, g, c = O.mesh_boxes(boxes, **params)
    A = O.assemble(a, g)
    return boxes, params, (a, g, c), A


@pytest.mark.parametrize("prec", [0, 1])
def test_entries_two_bars(ctx, two_bars_oracle, prec):
    from paper_2203_11733_gb300 import gbem
    boxes, params, (a, g, c), A_ref = two_bars_oracle
    mesh = ctx.mesh(boxes, params)
    p = _perm(mesh, a, g, c)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    R = A_ref[np.ix_(p, p)]
    err = _rel(A, R)
    assert err.max() <= ENTRY_TOL[prec], (prec, err.max(), np.unravel_index(err.argmax(), err.shape))
    n, counts = mat.info()
    assert n == 608 and counts.sum() == 608 * 609 // 2 and counts[0] > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_capacitance_two_bars(ctx, two_bars_oracle, prec):
    from paper_2203_11733_gb300 import gbem
    boxes, params, (a, g, c), A_ref = two_bars_oracle
    C_ref = O.capacitance_from_matrix(A_ref, c, W.EPS_R_SIO2)
    C, resid = gbem.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)
    assert _cap_err(C, C_ref) <= CAP_TOL[prec]
    assert resid < 1e-10


@pytest.mark.parametrize("prec", [0, 1])
def test_ragged_panel_list_sphere(ctx, prec):
    """216 panels given in input order: 7 tiles of 32 with a ragged tail of 24,
    padded to 256 for the factor."""
    from paper_2203_11733_gb300 import gbem
    a, g, c = W.voxel_sphere_panels(1.0, 3, outer=True)
    a, g, c = np.array(a), np.array(g), np.array(c)
    mesh = ctx.mesh_from_panels(a, g, c)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    A_ref = O.assemble(a, g)
    assert _rel(A, A_ref).max() <= ENTRY_TOL[prec]
    C, _ = gbem.gbem_capacitance(mesh, mat, 1.0)
    C_ref = O.capacitance_from_matrix(A_ref, c, 1.0)
    assert _cap_err(C, C_ref) <= CAP_TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_graded_bus_entries_and_capacitance(ctx, prec):
    """Edge-graded 2x2 crossing bus at a coarser size (N = 1640): elongated
    panels of very different sizes, both panel orientations, four conductors."""
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.crossing_bus_2x2(h=0.08, h_min=0.015)
    a, g, c = O.mesh_boxes(boxes, **params)
    A_ref = O.assemble(a, g)
    mesh = ctx.mesh(boxes, params)
    p = _perm(mesh, a, g, c)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    assert _rel(A, A_ref[np.ix_(p, p)]).max() <= ENTRY_TOL[prec]
    C, _ = gbem.gbem_capacitance(mesh, mat, W.EPS_R_SIO2)
    C_ref = O.capacitance_from_matrix(A_ref, c, W.EPS_R_SIO2)
    assert _cap_err(C, C_ref) <= CAP_TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_bus_sampled_entries_and_capacitance(ctx, prec):
    """The 2x2 crossing bus at full size (N = 6264), the benchmark workload:
    sampled entries (random pairs plus whole rows, so every pair class is
    hit) against the oracle one by one, and the capacitance matrix against
    the stored oracle result."""
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.crossing_bus_2x2()
    a, g, c = O.mesh_boxes(boxes, **params)
    mesh = ctx.mesh(boxes, params)
    p = _perm(mesh, a, g, c)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    rng = np.random.default_rng(7)
    n = mesh.n
    I = rng.integers(0, n, 3000)
    J = rng.integers(0, n, 3000)
    rows = rng.integers(0, n, 2)
    I = np.concatenate([I, np.repeat(rows, n)])
    J = np.concatenate([J, np.tile(np.arange(n), len(rows))])
    ref = O.entries(a, g, p[I], p[J])
    err = _rel(A[I, J], ref)
    assert err.max() <= ENTRY_TOL[prec], err.max()
    gold = json.load(open(os.path.join(HERE, "golden", "crossing_bus_2x2_capacitance.json")))
    C_ref = np.array(gold["C"])
    C, _ = gbem.gbem_capacitance(mesh, mat, gold["eps_r"])
    assert _cap_err(C, C_ref) <= CAP_TOL[prec]


def test_solve_random_rhs(ctx):
    import torch
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.two_bars()
    mesh = ctx.mesh(boxes, params)
    for prec in (0, 1):
        mat = gbem.gbem_assemble(mesh, prec)
        A = mat.download()
        mat.factor()
        B = torch.randn(mesh.n, 20, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
        X, it = mat.solve(B)
        Xh, Bh = X.cpu().numpy(), B.cpu().numpy()
        r = np.abs(A @ Xh - Bh).max() / np.abs(Bh).max()
        assert r < 1e-11, (prec, r, it)
        if prec == 1:
            assert 1 <= it <= 10


def test_deterministic(ctx):
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.two_bars()
    for prec in (0, 1):
        C1, _ = gbem.extract(ctx, boxes, params, 3.9, precision=prec)
        C2, _ = gbem.extract(ctx, boxes, params, 3.9, precision=prec)
        assert np.array_equal(C1, C2)


def test_single_panel_per_conductor(ctx):
    """Degenerate case: one panel per conductor, N = 2, padded to 128."""
    from paper_2203_11733_gb300 import gbem
    a = np.array([2, 2])
    g = np.array([[0, 0, 1, 0, 1], [1, 0, 1, 0, 1]], dtype=float)
    c = np.array([5, 9])
    mesh = ctx.mesh_from_panels(a, g, c)
    C, _ = gbem.gbem_capacitance(mesh, gbem.gbem_assemble(mesh, 0), 1.0)
    C_ref = O.capacitance(a, g, c, 1.0)
    assert _cap_err(C, C_ref) <= 1e-9


def test_budget_refusal(ctx):
    from paper_2203_11733_gb300 import gbem
    small = gbem.Context(0, hbm_budget=1 << 20)
    mesh = small.mesh(*W.two_bars())
    with pytest.raises(gbem.GbemError) as e:
        gbem.gbem_assemble(mesh, 0)
    assert e.value.status == -2
    mesh.close()
    small.close()


def test_solve_before_factor_is_refused(ctx):
    import torch
    from paper_2203_11733_gb300 import gbem
    mesh = ctx.mesh(*W.cube(1.0, 2))
    mat = gbem.gbem_assemble(mesh, 0)
    with pytest.raises(gbem.GbemError) as e:
        mat.solve(torch.ones(mesh.n, 1, dtype=torch.float64, device="cuda"))
    assert e.value.status == -8


def test_kernel_trace_covers_the_mixed_path(ctx):
    """Level-2 tracing times every launch of the four traced kernels of a
    mixed extraction and reports their algorithmic work; the traced result
    is the untraced one."""
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.two_bars()
    C0, _ = gbem.extract(ctx, boxes, params, 3.9, precision=1)
    gbem.set_timing(ctx, 2)
    gbem.get_kernel_stats(ctx, reset=True)
    C1, _ = gbem.extract(ctx, boxes, params, 3.9, precision=1)
    k = gbem.get_kernel_stats(ctx, reset=True)
    gbem.set_timing(ctx, 0)
    assert np.array_equal(C0, C1)
    assert k["assemble"]["launches"] == 1
    # the FP32 factorisation is one traced span: its per-step launches and
    # the rest updates on the second stream overlap
    assert k["factor"]["launches"] == 1
    assert k["sweep"]["launches"] >= 2 and k["residual"]["launches"] >= 1
    for name, d in k.items():
        assert d["ms"] > 0 and d["bytes"] > 0, name
    assert k["factor"]["flops"] > 0 and k["residual"]["flops"] > 0
    empty = gbem.get_kernel_stats(ctx)
    assert all(d["launches"] == 0 for d in empty.values())


@pytest.mark.slow
@pytest.mark.parametrize("prec", [0, 1])
def test_three_layer_bus_sampled_entries_and_capacitance(ctx, prec):
    """The largest workload, the three-layer 5x5x5 crossing bus (N = 23172,
    15 conductors): 3000 random entries and two whole rows against the oracle
    one by one, and the 15 x 15 capacitance matrix against the stored oracle
    result of the full FP64 assembly and Cholesky solve."""
    from paper_2203_11733_gb300 import gbem
    gold = json.load(open(os.path.join(HERE, "golden", "bus_3layer_5x5x5_capacitance.json")))
    boxes, params = W.bus_3layer_5x5x5()
    assert gold["params"] == params
    a, g, c = O.mesh_boxes(boxes, **params)
    mesh = ctx.mesh(boxes, params)
    n = mesh.n
    assert n == gold["n_panels"] == 23172
    p = _perm(mesh, a, g, c)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    rng = np.random.default_rng(11)
    I = rng.integers(0, n, 3000)
    J = rng.integers(0, n, 3000)
    rows = rng.integers(0, n, 2)
    I = np.concatenate([I, np.repeat(rows, n)])
    J = np.concatenate([J, np.tile(np.arange(n), len(rows))])
    vals = A[I, J]
    del A
    ref = O.entries(a, g, p[I], p[J])
    err = _rel(vals, ref)
    assert err.max() <= ENTRY_TOL[prec], err.max()
    C, resid = gbem.gbem_capacitance(mesh, mat, gold["eps_r"])
    mat.close()
    mesh.close()
    C_ref = np.array(gold["C"])
    assert C.shape == (15, 15)
    assert _cap_err(C, C_ref) <= CAP_TOL[prec], _cap_err(C, C_ref)


@pytest.mark.slow
def test_mixed_refinement_converges_at_large_order(ctx):
    """The compensated FP32 residual must stay accurate enough for the FP64
    refinement to reach its 1e-11 tolerance at large N (the three-layer bus,
    N = 23172)."""
    from paper_2203_11733_gb300 import gbem
    boxes, params = W.bus_3layer_5x5x5()
    mesh = ctx.mesh(boxes, params)
    assert mesh.n == 23172
    mat = gbem.gbem_assemble(mesh, 1)
    C, res = gbem.gbem_capacitance(mesh, mat, W.EPS_R_SIO2)
    mat.close()
    mesh.close()
    assert res <= 1e-11
    assert np.all(np.diag(C) > 0) and np.all(C - np.diag(np.diag(C)) <= 0)
    assert np.all(C.sum(axis=1) > 0)
