"""Extraction server (continuous batching): results in the mix equal the same
requests run alone; admission respects the HBM budget; requests overlap."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _err(C, R):
    return float(np.max(np.abs(C - R)) / np.max(np.abs(R)))


def _drain(srv, n, timeout_polls=2000):
    got = {}
    for _ in range(timeout_polls):
        for info, C in srv.poll(wait_ms=50):
            got[info["id"]] = (info, C)
        if len(got) >= n:
            break
    return got


def test_mix_equals_alone_and_overlaps():
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    torch.cuda.set_device(0)
    B.build()
    reqs = W.serving_requests(seed=31, count=10, rate_per_s=1000.0, n_lo=400, n_hi=2500)
    srv = gbem.Server(0, hbm_budget=8 << 30, slots=4)
    for k, (_, boxes, params) in enumerate(reqs):
        srv.submit(k, boxes, params, W.EPS_R_SIO2)
    got = _drain(srv, len(reqs))
    stats = srv.stats()
    srv.close()
    assert len(got) == len(reqs)
    assert stats["peak_reserved"] <= 8 << 30
    ctx = gbem.Context(0)
    for k, (_, boxes, params) in enumerate(reqs):
        info, C = got[k]
        assert info["status"] == 0 and info["residual"] < 1e-10
        C_alone, _ = gbem.extract(ctx, boxes, params, W.EPS_R_SIO2, precision=gbem.GBEM_MIXED)
        assert _err(C, C_alone) <= 1e-12
    # two small requests against the FP64 oracle
    for k in range(2):
        _, boxes, params = reqs[k]
        a, g, c = O.mesh_boxes(boxes, **params)
        if len(a) <= 900:
            assert _err(got[k][1], O.capacitance(a, g, c, W.EPS_R_SIO2)) <= 1e-6
    # work of different requests overlapped in time
    spans = sorted((got[k][0]["start_s"], got[k][0]["done_s"]) for k in got)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    ctx.close()


def test_budget_admission_and_rejection():
    from paper_2203_11733_gb300 import gbem
    rng = W.SplitMix64(8)
    small = W.bus_structure(rng, 600)
    big = W.bus_structure(rng, 6000)
    srv = gbem.Server(0, hbm_budget=200 << 20, slots=4)   # room for one small request at a time
    need_small = srv.submit(0, small[0], small[1], 1.0)
    srv.submit(1, small[0], small[1], 1.0)
    need_big = srv.submit(2, big[0], big[1], 1.0)
    assert need_small <= 200 << 20 < need_big
    got = _drain(srv, 3)
    stats = srv.stats()
    srv.close()
    assert got[2][0]["status"] == -2          # larger than the whole budget
    assert got[0][0]["status"] == 0 and got[1][0]["status"] == 0
    assert stats["peak_reserved"] <= 200 << 20
    assert np.array_equal(got[0][1], got[1][1])
    if 2 * need_small > 200 << 20:            # one at a time: no overlap possible
        s0, s1 = got[0][0], got[1][0]
        assert s1["start_s"] >= s0["done_s"] or s0["start_s"] >= s1["done_s"]
