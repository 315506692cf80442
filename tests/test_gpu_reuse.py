"""A destroyed matrix's device buffers stay with the context (idle) and serve
the next matrix of the same size: a repeated extraction makes no allocation
and gives the same bits; a matrix of another size releases them; a budget
that cannot hold them next to a new matrix drops them instead of refusing."""
import numpy as np
import pytest

from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2203_11733_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()


def _extract(mesh, prec):
    from paper_2203_11733_gb300 import gbem
    mat = gbem.gbem_assemble(mesh, prec)
    C, res = gbem.gbem_capacitance(mesh, mat, W.EPS_R_SIO2)
    held = mesh.ctx.bytes_in_use()
    mat.close()
    return C, res, held


@pytest.mark.parametrize("prec", [0, 1])
def test_repeat_reuses_every_buffer_and_the_bits(lib, prec):
    from paper_2203_11733_gb300 import gbem
    ctx = gbem.Context(0)
    mesh = ctx.mesh(*W.two_bars())
    base = ctx.bytes_in_use()
    C1, r1, held1 = _extract(mesh, prec)
    assert held1 > base
    # the matrix's buffers are kept: nothing returned to the allocator
    assert ctx.bytes_in_use() == held1
    C2, r2, held2 = _extract(mesh, prec)
    assert held2 == held1          # every buffer of the second matrix was a spare
    assert np.array_equal(C1, C2) and r1 == r2
    # another size: the bus can take only the small spares of the bars (its
    # large buffers differ in size); when it goes, the bars' remaining spares
    # are released and the bus's are kept
    bus = ctx.mesh(*W.crossing_bus_2x2())
    bus_base = ctx.bytes_in_use()
    C3, _, held3 = _extract(bus, prec)
    assert held3 > bus_base
    kept = ctx.bytes_in_use()
    assert held3 - (held1 - base) <= kept < held3
    bus.close()
    mesh.close()
    ctx.close()


def test_budget_drops_spares_instead_of_refusing(lib):
    from paper_2203_11733_gb300 import gbem
    # sizes from a context without a budget
    probe = gbem.Context(0)
    bars = probe.mesh(*W.two_bars())
    base_b = probe.bytes_in_use()
    C_ref, _, held = _extract(bars, 1)
    m_b = held - base_b
    bars.close()
    probe.close()
    probe = gbem.Context(0)
    bus = probe.mesh(*W.crossing_bus_2x2())
    base_x = probe.bytes_in_use()
    _, _, held = _extract(bus, 1)
    m_x = held - base_x
    bus.close()
    probe.close()
    # room for both meshes, the bus's matrix and half of the bars': the bus
    # fits only once the bars' spares are dropped
    ctx = gbem.Context(0, hbm_budget=base_b + base_x + m_x + m_b // 2)
    bars = ctx.mesh(*W.two_bars())
    bus = ctx.mesh(*W.crossing_bus_2x2())
    C1, _, _ = _extract(bars, 1)
    assert ctx.bytes_in_use() == base_b + base_x + m_b   # the bars' buffers are kept
    _, res, _ = _extract(bus, 1)
    assert res <= 1e-11
    C2, _, _ = _extract(bars, 1)
    assert np.array_equal(C1, C_ref) and np.array_equal(C2, C_ref)
    bus.close()
    bars.close()
    ctx.close()
