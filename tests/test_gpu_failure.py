"""Failure paths, made on the host or by a withheld flag; none of them faults
or hangs the GPU.

* A bounded device wait whose dependency never arrives (a flag that nothing
  writes) gives up after its wall-clock limit, reports GBEM_ERR_TIMEOUT to
  the host, and leaves the context usable.
* An allocator callback that refuses (returns NULL) makes the call fail with
  GBEM_ERR_OOM, whichever allocation of the extraction it refuses; nothing
  leaks and the next extraction succeeds.
"""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gb():
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    B.build()
    return gbem


@pytest.fixture(scope="module")
def two_bars_ref():
    boxes, params = W.two_bars()
    a, g, c = O.mesh_boxes(boxes, **params)
    return boxes, params, O.capacitance(a, g, c, W.EPS_R_SIO2)


def _err(C, R):
    return float(np.max(np.abs(C - R)) / np.max(np.abs(R)))


def test_withheld_flag_times_out_and_context_survives(gb, two_bars_ref):
    boxes, params, C_ref = two_bars_ref
    ctx = gb.Context(0)
    assert ctx.selftest_wait(True, 50.0) == 0          # flag written: the wait ends at once
    t0 = time.perf_counter()
    st = ctx.selftest_wait(False, 50.0)                # flag withheld: the wait runs out
    dt = time.perf_counter() - t0
    assert st == -5, st                                # GBEM_ERR_TIMEOUT
    assert 0.04 <= dt < 5.0, dt
    assert b"gave up" in ctx.lib.gbem_last_error(ctx.h)
    for prec, tol in ((0, 1e-9), (1, 1e-6)):          # the context still computes
        C, _ = gb.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)
        assert _err(C, C_ref) <= tol
    with pytest.raises(gb.GbemError) as e:
        ctx.check(ctx.lib.gbem_selftest_wait(ctx.h, 0, 0.0, None))
    assert e.value.status == -1                        # limit out of range
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_allocator_refusal_at_every_allocation(gb, two_bars_ref, prec):
    boxes, params, C_ref = two_bars_ref
    probe = gb.Context(0)
    gb.extract(probe, boxes, params, W.EPS_R_SIO2, precision=prec)
    total = probe.alloc_calls                          # allocations of one extraction
    probe.close()
    assert total >= 5
    for k in range(total):
        ctx = gb.Context(0, refuse=lambda i, n, k=k: i == k)
        status = 0
        try:
            gb.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)
        except gb.GbemError as e:
            status = e.status
        assert status == -2, f"allocation {k} of {total} refused: status {status}"   # GBEM_ERR_OOM
        C, _ = gb.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=prec)   # refusals are over
        assert _err(C, C_ref) <= (1e-9 if prec == 0 else 1e-6)
        ctx.close()


def test_refused_context_releases_everything(gb, two_bars_ref):
    """After a refused assembly and the destruction of the mesh, the context
    holds no device memory (spare buffers are released with the context's
    next matrix destroy or its own destroy; none exist yet here)."""
    boxes, params, _ = two_bars_ref
    ctx = gb.Context(0, refuse=lambda i, n: i == 1)    # the mesh upload passes, the matrix is refused
    mesh = ctx.mesh(boxes, params)
    with pytest.raises(gb.GbemError) as e:
        gb.gbem_assemble(mesh, 1)
    assert e.value.status == -2
    mesh.close()
    assert ctx.bytes_in_use() == 0
    ctx.close()
