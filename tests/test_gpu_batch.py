"""Batched extraction (one CUDA graph for many independent structures)
against the FP64 oracle and against single extractions."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_11733_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    from paper_2203_11733_gb300 import build as B
    from paper_2203_11733_gb300 import gbem
    torch.cuda.set_device(0)
    B.build()
    c = gbem.Context(0)
    yield c
    c.close()


def _err(C, R):
    return float(np.max(np.abs(C - R)) / np.max(np.abs(R)))


def test_batch_matches_oracle_and_single(ctx):
    from paper_2203_11733_gb300 import gbem
    structs = W.batch_small_structures(seed=99, count=6, n_lo=150, n_hi=450)
    meshes = [ctx.mesh(b, p) for b, p in structs]
    batch = gbem.Batch(ctx, meshes)
    Cs, res = batch.run(W.EPS_R_SIO2)
    assert np.all(res < 1e-9), res
    for (boxes, params), C, m in zip(structs, Cs, meshes):
        a, g, c = O.mesh_boxes(boxes, **params)
        C_ref = O.capacitance(a, g, c, W.EPS_R_SIO2)
        assert _err(C, C_ref) <= 1e-6
        C1, _ = gbem.gbem_capacitance(m, gbem.gbem_assemble(m, gbem.GBEM_MIXED), W.EPS_R_SIO2)
        assert _err(C, C1) <= 1e-6
    # the graph replays deterministically
    Cs2, res2 = batch.run(W.EPS_R_SIO2)
    for C, C2 in zip(Cs, Cs2):
        assert np.array_equal(C, C2)
    batch.close()


def test_batch_mixed_sizes_and_padding(ctx):
    """Structures of very different orders (one below a single tile) in one
    batch, including one with more than 8 conductors."""
    from paper_2203_11733_gb300 import gbem
    rng = W.SplitMix64(5)
    structs = [W.cube(1.0, 2), W.two_bars(), W.bus_structure(rng, 300)]
    while len(structs[-1][0]) <= 8:
        structs[-1] = W.bus_structure(rng, 300)
    meshes = [ctx.mesh(b, p) for b, p in structs]
    Cs, res = gbem.Batch(ctx, meshes).run(1.0)
    for (boxes, params), C in zip(structs, Cs):
        a, g, c = O.mesh_boxes(boxes, **params)
        assert _err(C, O.capacitance(a, g, c, 1.0)) <= 1e-6


def test_grouped_batch_equals_single_group(ctx):
    """Splitting a batch into groups (parts whose graphs run concurrently)
    changes no result: every structure's computation is its own."""
    from paper_2203_11733_gb300 import gbem
    structs = W.batch_small_structures(seed=321, count=9, n_lo=150, n_hi=900)
    meshes = [ctx.mesh(b, p) for b, p in structs]
    one = gbem.Batch(ctx, meshes, iters=3, groups=1)
    three = gbem.Batch(ctx, meshes, iters=3, groups=3)
    assert three.config == {"groups": 3, "iters": 3}
    C1, r1 = one.run(W.EPS_R_SIO2)
    C3, r3 = three.run(W.EPS_R_SIO2)
    for a, b in zip(C1, C3):
        assert np.array_equal(a, b)
    assert np.array_equal(r1, r3)
    one.close()
    three.close()


def test_autotune_picks_a_converging_configuration_and_caches_it(ctx, tmp_path):
    from paper_2203_11733_gb300 import gbem
    structs = W.batch_small_structures(seed=555, count=12, n_lo=150, n_hi=900)
    meshes = [ctx.mesh(b, p) for b, p in structs]
    cache = str(tmp_path / "batch_tuning.txt")
    batch, choice = gbem.Batch.autotune(ctx, meshes, max_iters=3, cache_path=cache)
    assert choice["groups"] in (1, 2, 4) and 1 <= choice["iters"] <= 3 and choice["ms"] > 0
    assert not choice["from_cache"]
    assert batch.config == {"groups": choice["groups"], "iters": choice["iters"]}
    Cs, res = batch.run(W.EPS_R_SIO2)
    assert np.all(res <= 1e-11), res
    ref = gbem.Batch(ctx, meshes, iters=3)
    Cr, _ = ref.run(W.EPS_R_SIO2)
    for a, b in zip(Cs, Cr):
        assert _err(a, b) <= 1e-9
    batch.close()
    ref.close()
    # the same batch again: the cached choice, without timing runs
    batch2, choice2 = gbem.Batch.autotune(ctx, meshes, max_iters=3, cache_path=cache)
    assert choice2["from_cache"]
    assert (choice2["groups"], choice2["iters"]) == (choice["groups"], choice["iters"])
    batch2.close()
