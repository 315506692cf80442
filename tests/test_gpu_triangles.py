"""Parity of the flat-triangle path on the GPU with the triangle oracle: every
entry of a two-conductor mesh (a level-2 icosphere inside a level-1
icosphere shell, 400 triangles, a ragged last tile) and its capacitance in
FP64 and mixed precision; sampled entries of a 5120-triangle sphere,
including every pair that touches one triangle; and icospheres rising toward
the capacitance of the sphere, 4 pi eps R."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle import triangles as T
from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    B.build()
    gbem.load()
    torch.cuda.set_device(0)
    c = gbem.Context(0)
    yield c
    c.close()


def two_spheres():
    inner = W.icosphere(1.0, 2)
    outer = W.icosphere(2.5, 1, centre=(0.3, -0.2, 0.1))
    tris = np.vstack([inner, outer])
    cond = np.r_[np.zeros(len(inner)), np.ones(len(outer))].astype(np.int32)
    return tris, cond


def test_entries_and_capacitance_match_oracle(ctx):
    tris, cond = two_spheres()
    A_ref = T.tri_assemble(tris)
    mesh = ctx.mesh_from_triangles(tris, cond)
    mat = mesh.assemble(gbem.GBEM_FP64)
    A = mat.download()
    scale = np.abs(A_ref).max(axis=1, keepdims=True)
    assert np.all(np.abs(A - A_ref) <= 1e-10 * scale)
    C, resid = gbem.gbem_capacitance(mesh, mat, 1.0)
    C_ref = O.capacitance_from_matrix(A_ref, cond, 1.0)
    assert np.abs(C - C_ref).max() <= 1e-9 * np.abs(C_ref).max()
    mat.close()
    mat = mesh.assemble(gbem.GBEM_MIXED)
    Am = mat.download()   # float pairs hi + lo: FP64 closed forms near, FP32 far rules
    assert np.all(np.abs(Am - A_ref) <= 1e-6 * scale)
    Cm, resid = gbem.gbem_capacitance(mesh, mat, 1.0)
    assert resid <= 1e-10
    assert np.abs(Cm - C_ref).max() <= 1e-6 * np.abs(C_ref).max()
    mat.close()
    mesh.close()


def test_large_sphere_sampled_entries(ctx):
    tris = W.icosphere(1.0, 4)
    n = len(tris)
    mesh = ctx.mesh_from_triangles(tris, np.zeros(n, np.int32))
    mat = mesh.assemble(gbem.GBEM_FP64)
    A = mat.download()
    rng = np.random.default_rng(3)
    I = rng.integers(0, n, 1500)
    J = rng.integers(0, n, 1500)
    # every triangle touching triangle 17, and the self-term
    t = tris.reshape(-1, 3, 3)
    touch = [j for j in range(n) if any(np.array_equal(a, b) for a in t[17] for b in t[j])]
    I = np.r_[I, np.full(len(touch), 17)]
    J = np.r_[J, touch]
    ref = T.tri_entries(tris, I, J)
    assert len(touch) >= 10   # the triangle, 3 edge and 6-9 vertex neighbours
    assert np.all(np.abs(A[I, J] - ref) <= 1e-10 * np.abs(ref))
    mat.close()
    mesh.close()


def test_icospheres_approach_sphere_capacitance(ctx):
    vals = []
    for level in (2, 3, 4):
        tris = W.icosphere(1.0, level)
        mesh = ctx.mesh_from_triangles(tris, np.zeros(len(tris), np.int32))
        mat = mesh.assemble(gbem.GBEM_FP64)
        C, _ = gbem.gbem_capacitance(mesh, mat, 1.0)
        vals.append(C[0, 0] / (4 * math.pi * O.EPS0 * 1e-6))
        mat.close()
        mesh.close()
    assert vals[0] < vals[1] < vals[2] < 1.0
    assert vals[2] > 0.995
