"""Host-side checks of the C ABI: the library loads and exports every entry
point declared in include/gbem.h, and the host mesher (Sec. 3.1/3.3) builds
the same panels as the oracle's mesher.  No GPU is touched."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gbem.load()


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^\w[\w\s\*]*?\b(gbem_\w+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def test_header_declares_boundary(lib):
    names = _declared()
    for required in ("gbem_mesh", "gbem_assemble", "gbem_factor", "gbem_solve", "gbem_capacitance"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gbem_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing
    for n in _declared():
        assert hasattr(lib, n)


def _host_ctx():
    return gbem.Context(device=-1, torch_alloc=False)


def _match(pa, pg, pc, oa, og, oc):
    """Permutation p with product panel i == oracle panel p[i]."""
    key_o = {}
    for i in range(len(oa)):
        key_o[(int(oa[i]), int(oc[i])) + tuple(np.round(og[i], 9))] = i
    perm = np.empty(len(pa), dtype=np.int64)
    for i in range(len(pa)):
        k = (int(pa[i]), int(pc[i])) + tuple(np.round(pg[i], 9))
        perm[i] = key_o[k]
    return perm


@pytest.mark.parametrize("name", ["two_bars", "crossing_bus_2x2", "bus_3layer_5x5x5", "cube"])
def test_mesher_matches_oracle_mesher(lib, name):
    boxes, params = getattr(W, name)()
    ctx = _host_ctx()
    m = ctx.mesh(boxes, params)
    pa, pg, pc, ids = m.panels()
    oa, og, oc = O.mesh_boxes(boxes, **params)
    assert m.n == len(oa)
    perm = _match(pa, pg, pc, oa, og, oc)
    assert len(set(perm.tolist())) == len(perm)
    assert np.allclose(pg, og[perm], rtol=0, atol=1e-12)
    # ordered by conductor
    assert np.all(np.diff(pc) >= 0)
    assert list(ids) == sorted(set(int(b[2]) for b in boxes))


def test_expected_sizes(lib):
    ctx = _host_ctx()
    assert ctx.mesh(*W.two_bars()).n == 608
    assert ctx.mesh(*W.crossing_bus_2x2()).n == 6264
    assert ctx.mesh(*W.bus_3layer_5x5x5()).n == 23172


def test_mesh_errors(lib):
    ctx = _host_ctx()
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh([((0, 0, 0), (1, 1, 1), 0), ((0.5, 0.5, 0.5), (2, 2, 2), 1)], dict(h=0.5))
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh([((0, 0, 0), (1, 1, 1), 0), ((1, 0, 0), (2, 1, 1), 1)], dict(h=0.5))   # touching
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh([((0, 0, 0), (0, 1, 1), 0)], dict(h=0.5))   # empty box
    assert e.value.status == -7
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh([((0, 0, 0), (1, 1, 1), 0)], dict(h=0.0))
    assert e.value.status == -1
    with pytest.raises(gbem.GbemError) as e:
        ctx.mesh_from_panels([2], [[0, 0, 0, 0, 1]], [0])     # zero-area panel
    assert e.value.status == -7


def test_host_context_refuses_compute(lib):
    ctx = _host_ctx()
    m = ctx.mesh(*W.cube(1.0, 2))
    with pytest.raises(gbem.GbemError) as e:
        m.assemble(gbem.GBEM_FP64, stream=0)
    assert e.value.status == -9
    with pytest.raises(gbem.GbemError) as e:
        ctx.unit_rates(stream=0)
    assert e.value.status == -9
    out = (ctypes.c_double * 8)()
    assert lib.gbem_unit_rates(ctx.h, out, 0, None) == -1           # no rate asked for
    assert lib.gbem_unit_rates(ctx.h, out, 8, None) == -1           # more than GBEM_RATE_COUNT
    assert lib.gbem_unit_rates(None, out, 1, None) == -1


def test_graded_division_matches_definition(lib):
    # 0.1 um edge, h 30 nm, h_min 5 nm, ratio 1.5: 4 graded cells per side
    nodes = O.divide(0.0, 0.1, 0.03, 1.5, 0.005)
    sizes = np.diff(nodes)
    assert len(sizes) == 9
    assert np.allclose(sizes[:4], [0.005, 0.0075, 0.01125, 0.016875])
    assert np.allclose(sizes[-4:], sizes[:4][::-1])
