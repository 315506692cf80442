"""Extraction server (continuous batching): results in the mix equal the same
requests run alone; admission respects the HBM budget; requests overlap."""
import json
import os

import numpy as np
import pytest

from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(__file__)


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
    # requests 0 and 1 (2304 and 1936 panels) against the stored FP64 oracle
    # results (tests/golden/make_golden.py serving_seed31)
    gold = json.load(open(os.path.join(HERE, "golden", "serving_seed31_capacitance.json")))["requests"]
    assert [g["request"] for g in gold] == [0, 1]
    for g in gold:
        k = g["request"]
        assert got[k][0]["n_panels"] == g["n_panels"]
        assert _err(got[k][1], np.array(g["C"])) <= 1e-6
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


def test_smaller_request_passes_a_blocked_head():
    """A request at the head of the queue that fits the budget but not the
    memory left next to the running requests does not hold back a smaller
    request behind it that fits: the small one is admitted at once, the
    large one when the memory frees up."""
    from paper_2203_11733_gb300 import gbem
    rng = W.SplitMix64(21)
    small = W.bus_structure(rng, 1500)
    big = W.bus_structure(rng, 6000)
    probe = gbem.Server(0, hbm_budget=1 << 40, slots=1)
    need_small = probe.submit(0, small[0], small[1], 1.0)
    need_big = probe.submit(1, big[0], big[1], 1.0)
    _drain(probe, 2)
    probe.close()
    budget = need_big + need_small // 2          # big alone fits, big + small does not
    assert 2 * need_small <= budget < need_big + need_small
    srv = gbem.Server(0, hbm_budget=budget, slots=3)
    srv.submit(0, small[0], small[1], 1.0)       # admitted at once
    srv.submit(1, big[0], big[1], 1.0)           # must wait for request 0
    srv.submit(2, small[0], small[1], 1.0)       # fits next to request 0
    got = _drain(srv, 3)
    stats = srv.stats()
    srv.close()
    assert all(got[k][0]["status"] == 0 for k in range(3))
    assert stats["peak_reserved"] <= budget
    i0, i1, i2 = (got[k][0] for k in range(3))
    assert i2["start_s"] < i1["start_s"]         # the small request passed the blocked head
    assert i1["start_s"] >= i0["done_s"] - 1e-6 and i1["start_s"] >= i2["done_s"] - 1e-6
    assert np.array_equal(got[0][1], got[2][1])
