"""Parity of the multi-dielectric path (Sec. 4) on the GPU with the oracle, in
FP64 and in mixed mode:
the assembled system entry by entry and the capacitance matrix after the LU
solve, on stacks of 184, 512 and 592 equations (ragged and whole 64-blocks);
at 5520 equations, sampled entries against the oracle's integrals and the
exact identity with the single-layer path when one dielectric fills the
enclosure."""
import numpy as np
import pytest
import torch

from oracle import dielectric as D
from oracle import oracle as O
from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem

from test_stack_host import CASES

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    gbem.load()
    torch.cuda.set_device(0)
    c = gbem.Context(0)
    yield c
    c.close()


def _stack(ctx, case):
    lo, hi, z, eps, bc, boxes, h, ho = case
    return gbem.Stack(ctx, lo, hi, z, eps, bc, boxes, h, ho), D.mesh_stack(D.Stack(lo, hi, z, eps, bc), boxes, h, ho)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_system_and_capacitance_match_oracle(ctx, case):
    S, ref = _stack(ctx, CASES[case])
    eps = CASES[case][3]
    stream = torch.cuda.Stream()
    S.assemble(gbem.GBEM_FP64, stream)
    M, Bg = S.system()
    M_ref, B_ref, ids = D.system(ref, eps)
    # every entry within 1e-10 of its row's largest entry
    scale = np.abs(M_ref).max(axis=1, keepdims=True)
    assert np.abs(M - M_ref).max(axis=1).max() <= 1e-10 * scale.max()
    assert np.all(np.abs(M - M_ref) <= 1e-10 * scale)
    assert np.abs(Bg - B_ref).max() <= 1e-10 * np.abs(B_ref).max()
    C, resid = S.capacitance(stream)
    import scipy.linalg as sla
    X = sla.lu_solve(sla.lu_factor(M_ref), B_ref)
    C_ref = D.charges(ref, eps, X, ids)
    assert resid < 1e-12
    assert np.abs(C - C_ref).max() <= 1e-9 * np.abs(C_ref).max()
    # a second solve reuses the factor
    C2, _ = S.capacitance(stream)
    assert np.array_equal(C, C2)
    S.close()


BENCH_STACK = ([-6, -6, 0], [6, 6, 4], [0, 1.0, 2.5, 4], [3.9, 2.5, 7.0], [D.NEUMANN] * 4 + [D.GROUND, D.GROUND],
               [([-4 + 2 * i, -5, 1.5], [-3 + 2 * i, 5, 2.0], i) for i in range(5)], 0.25, 0.6)


def test_full_size_sampled_entries(ctx):
    """Five wires in the middle of three layers, 5520 equations: 3000 sampled
    entries of every kind against the oracle's integrals."""
    S, ref = _stack(ctx, BENCH_STACK)
    assert S.n_eq == 5520
    S.assemble(gbem.GBEM_FP64, torch.cuda.Stream())
    M, Bg = S.system()
    rows, ucol, qcol, ids = D.layout(ref)
    eps = BENCH_STACK[3]
    rng = np.random.default_rng(7)
    ra, rb, sg = ref["region_a"], ref["region_b"], ref["sign"]
    area = O.areas(ref["geo"])
    picks = rng.integers(0, len(rows), 3000)
    I, K, R, A = [], [], [], []
    for r in picks:
        a, i = rows[r]
        P = np.nonzero((ra == a) | (rb == a))[0]
        k = int(P[rng.integers(0, len(P))])
        I.append(i)
        K.append(k)
        R.append(r)
        A.append(a)
    I, K = np.array(I), np.array(K)
    U = D.slayer_entries(ref["axis"], ref["geo"], I, K)
    Dl = D.dlayer_entries(ref["axis"], ref["geo"], I, K)
    for t in range(len(I)):
        i, k, r, a = I[t], K[t], R[t], A[t]
        own = ra[k] == a
        s = sg[k] if own else -sg[k]
        cu = (0.5 * area[i] if i == k else 0.0) + s * Dl[t]
        g = 1.0 if own else -eps[ra[k]] / eps[a]
        scale = np.abs(M[r]).max()
        if ucol[k] >= 0:
            assert abs(M[r, ucol[k]] - cu) <= 1e-10 * scale
        if qcol[k] >= 0:
            assert abs(M[r, qcol[k]] + U[t] * g) <= 1e-10 * scale
    C, resid = S.capacitance()
    assert resid < 1e-12
    # Maxwell pattern: positive diagonal, couplings negative up to the
    # discretisation level (the outer wires barely see each other past three
    # wires between grounded planes: |C_04| ~ 2e-5 C_00)
    assert np.all(np.diag(C) > 0)
    assert np.all(C - np.diag(np.diag(C)) < 1e-4 * np.diag(C).max())
    assert C[0, 1] < 0 and C[1, 2] < 0
    assert np.abs(C - C.T).max() < 0.02 * np.abs(C).max()
    S.close()


def test_single_dielectric_equals_single_layer_path(ctx):
    """One dielectric, grounded enclosure: the system of Sec. 4 gives the same
    C as the single-layer system of Sec. 3 on the same panels (the enclosure
    as a conductor held at 0 V), here at 2844 equations through both GPU
    paths."""
    lo, hi = [0, 0, 0], [6, 6, 3]
    boxes = [([1, 1, 1], [5, 1.5, 1.6], 0), ([1, 2.5, 1.2], [5, 3.0, 1.8], 1), ([2.5, 4, 0.5], [3, 5, 2.5], 2)]
    S = gbem.Stack(ctx, lo, hi, [0, 3], [2.0], [D.GROUND] * 6, boxes, 0.25, 0.5)
    C, resid = S.capacitance(torch.cuda.Stream())
    p = S.panels()
    cond = np.where(p["cond"] >= 0, p["cond"], 99).astype(np.int32)
    mesh = ctx.mesh_from_panels(p["axis"], p["geo"], cond)
    mat = mesh.assemble(gbem.GBEM_FP64)
    C1, _ = mat.capacitance(2.0)
    assert S.n_eq == len(cond)
    assert np.abs(C - C1[:3, :3]).max() <= 1e-9 * np.abs(C1).max()
    mat.close()
    mesh.close()
    S.close()


@pytest.mark.parametrize("case", range(len(CASES)))
def test_mixed_matches_oracle(ctx, case):
    """Mixed mode: FP32 far field and FP32 LU, refined against the FP64-stored
    system: entries within 2e-6 of their row's scale, C within 1e-6."""
    S, ref = _stack(ctx, CASES[case])
    eps = CASES[case][3]
    stream = torch.cuda.Stream()
    S.assemble(gbem.GBEM_MIXED, stream)
    M, Bg = S.system()
    M_ref, B_ref, ids = D.system(ref, eps)
    scale = np.abs(M_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(M - M_ref) <= 2e-6 * scale)
    assert np.abs(Bg - B_ref).max() <= 2e-6 * np.abs(B_ref).max()
    C, resid = S.capacitance(stream)
    import scipy.linalg as sla
    C_ref = D.charges(ref, eps, sla.lu_solve(sla.lu_factor(M_ref), B_ref), ids)
    assert resid <= 1e-11 and S.iterations() <= 6
    assert np.abs(C - C_ref).max() <= 1e-6 * np.abs(C_ref).max()
    S.close()


def test_mixed_full_size_against_fp64(ctx):
    """5520 equations: the mixed extraction against the FP64 one."""
    S, _ = _stack(ctx, BENCH_STACK)
    stream = torch.cuda.Stream()
    S.assemble(gbem.GBEM_FP64, stream)
    C64, r64 = S.capacitance(stream)
    assert S.iterations() == 1 and r64 <= 1e-12
    S.assemble(gbem.GBEM_MIXED, stream)
    C32, r32 = S.capacitance(stream)
    assert r32 <= 1e-11 and S.iterations() <= 6
    assert np.abs(C32 - C64).max() <= 1e-6 * np.abs(C64).max()
    S.close()
