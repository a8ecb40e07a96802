"""Host logic of the multi-rank bench (N > 1) on CPU: two gloo ranks.

The filter's data path has no exchange step: every rank filters its own trajectories
(weak scaling), and the only collectives are the timing reductions. These tests run that
host logic as two spawned processes over gloo: the process group comes up from the
torchrun-style environment, ranks draw distinct inputs, timed regions reduce to the
slowest rank's time, and the whole-job rate counts every rank's units.
"""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, q) -> None:
    try:
        os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank),
                           "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
        sys.path.insert(0, ROOT)
        import bench
        from synth import simulate
        from synth.configs import batched_workloads
        r_, ws_, local, dist = bench._dist()
        assert (r_, ws_, local) == (rank, ws, rank)
        assert dist is not None and dist.get_backend() == "gloo"
        # each rank's "timed region" lasts a different time; all ranks see the largest
        t = 1.5 + 2.0 * rank
        t_max = bench.max_over_ranks(t, dist)
        # the same reduction on a value that only one rank holds large
        big = bench.max_over_ranks(7.0 if rank == ws - 1 else -3.0, dist)
        seed = bench.shard_seed(11, rank)
        tr = simulate("cubic", 4, 3, 0.01, seed=seed)
        members = batched_workloads(8, seed=bench.shard_seed(4, rank), steps=5)
        rate = bench.whole_job_rate(100, ws_, t_max)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, {"t_max": t_max, "big": big, "seed": seed, "dy0": tr.dy[0].tolist(),
                      "members": [(m.r, m.n, m.seed) for m in members], "rate": rate}))
    except BaseException as e:   # report to the parent instead of hanging it
        q.put((rank, {"error": repr(e)}))


def _run_ranks(ws: int = 2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(ws):
            rank, res = q.get(timeout=120)
            out[rank] = res
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return out


@pytest.fixture(scope="module")
def two_ranks():
    return _run_ranks(2)


def test_ranks_come_up_over_gloo(two_ranks):
    assert sorted(two_ranks) == [0, 1]
    for res in two_ranks.values():
        assert "error" not in res, res.get("error")


def test_timing_reduces_to_slowest_rank(two_ranks):
    # rank 0 timed 1.5 s, rank 1 timed 3.5 s: both report 3.5
    assert [two_ranks[r]["t_max"] for r in (0, 1)] == [3.5, 3.5]
    assert [two_ranks[r]["big"] for r in (0, 1)] == [7.0, 7.0]


def test_whole_job_rate_counts_every_rank(two_ranks):
    # 100 units per rank, 2 ranks, 3.5 s of the slowest rank
    for r in (0, 1):
        assert two_ranks[r]["rate"] == pytest.approx(200 / 3.5, rel=1e-15)


def test_ranks_filter_independent_inputs(two_ranks):
    a, b = two_ranks[0], two_ranks[1]
    assert a["seed"] != b["seed"]
    assert not np.allclose(a["dy0"], b["dy0"])
    assert a["members"] != b["members"]


def test_single_process_needs_no_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    assert bench._dist() == (0, 1, 0, None)
    assert bench.max_over_ranks(2.25, None) == 2.25
    assert bench.whole_job_rate(50, 1, 0.5) == 100.0
    assert bench.shard_seed(11, 0) == 11   # rank 0 keeps the workload's own trajectory
