"""bench.py's multi-rank logic on CPU: two gloo ranks, as torchrun launches
them (RANK / WORLD_SIZE / LOCAL_RANK / MASTER_* in the environment).  The
extractions are independent per rank, so the ranks exchange only their
times: every rank must see the slowest rank's time, and the whole-job rate
is the units of all ranks over that time.  The reference arm runs on rank 0
alone; the other ranks leave without work."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, seconds, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_env()
    bench.dist_start(w, backend="gloo")
    t = bench.max_over_ranks(seconds[r], w, device="cpu")
    rate = bench.whole_job_rate(100.0, w, t)
    bench.dist_stop(w)
    q.put((r, local, w, t, rate))


@pytest.mark.parametrize("seconds", [(1.5, 4.0), (3.0, 0.5)])
def test_two_gloo_ranks_report_the_slowest_rank(seconds):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, seconds, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    slowest = max(seconds)
    for r, (rank, local, world, t, rate) in enumerate(got):
        assert (rank, local, world) == (r, r, 2)
        assert t == slowest
        assert rate == pytest.approx(2 * 100.0 / slowest, rel=1e-15)


def test_single_process_needs_no_process_group(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    bench.dist_start(1)   # no process group for one rank
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
    bench.dist_stop(1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    assert args.steps == 10
    bench.run_reference(args)   # returns at once: no oracle work, no line
    assert capsys.readouterr().out == ""


def test_headline_steps_default(monkeypatch):
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    assert (args.steps, args.warmup, args.gpus, args.impl, args.workload) == (20, 3, 1, "ours", "headline")
    json.dumps(vars(args))
