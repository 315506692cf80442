"""The paper's distance-graded partition (Sec. 3.3) through the CUDA path:
meshes made by gbem_mesh_graded, with panels of very different sizes next to
each other (hanging nodes, enclosure walls of tens of microns beside
sub-micron panels), against the FP64 oracle on the identical panel set.

Tolerances as in the other parity tests: FP64 mode 1e-10 per entry and 1e-9
on capacitances, mixed mode 1e-6 on both."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu
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
    key = {(int(oa[i]), int(oc[i])) + tuple(np.round(og[i], 12)): i for i in range(len(oa))}
    return np.array([key[(int(pa[i]), int(pc[i])) + tuple(np.round(pg[i], 12))] for i in range(len(pa))])


def _cap_err(C, R):
    return float(np.max(np.abs(C - R)) / np.max(np.abs(R)))


CASES = [
    # the paper's Table 2 geometry with its grounded box and its Sec. 5 rule
    ("table2", dict(main=0, p1=0.75, p2=4.0, p3=1.0, p5=1.0), 1.0),
    # the 2x2 crossing bus graded for main net 0
    ("crossing_bus_2x2", dict(main=0, p1=0.0009, p2=4.0, p3=1.0, p5=0.1), 3.9),
]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_graded_mesh_entries_and_capacitance(ctx, case, prec):
    from paper_2203_11733_gb300 import gbem
    name, p, eps_r = case
    if name == "table2":
        boxes, encl = W.paper_two_bars()
    else:
        boxes, _ = getattr(W, name)()
        encl = None
    a, g, c = O.mesh_graded(boxes, p["main"], p["p1"], p["p2"], p["p3"], p["p5"], enclosure=encl)
    mesh = gbem.gbem_mesh_graded(ctx, boxes, p["main"], p["p1"], p["p2"], p["p3"], p["p5"], enclosure=encl)
    assert mesh.n == len(a)
    perm = _perm(mesh, a, g, c)
    A_ref = O.assemble(a, g)
    mat = gbem.gbem_assemble(mesh, prec)
    A = mat.download()
    err = np.abs(A - A_ref[np.ix_(perm, perm)]) / np.abs(A_ref[np.ix_(perm, perm)])
    assert err.max() <= ENTRY_TOL[prec], err.max()
    C, resid = gbem.gbem_capacitance(mesh, mat, eps_r)
    C_ref = O.capacitance_from_matrix(A_ref, c, eps_r)
    assert _cap_err(C, C_ref) <= CAP_TOL[prec]
    assert resid < 1e-10
    mat.close()
    mesh.close()
