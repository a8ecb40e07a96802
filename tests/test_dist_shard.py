"""The exchange and merge of a filter whose target rows are split across ranks, on the CPU:
two gloo ranks each hold one chunk of a seeded weighted node set, compute their chunk's
record (log-sum-exp, weight sums, weighted mean and second moment, written out here from
their definitions), exchange rows and records with the library's all-gather wiring
(sharded.exchange) and merge with the library's host merge (yy_merge_records_host, the same
code the device merge runs).  Both ranks must obtain the same result, equal to the FP64
oracle's normalisation and estimate of the whole node set."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
R_DIM, N_NODES = 5, 512


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _nodes():
    rng = np.random.default_rng(2024)
    u = rng.uniform(-0.3, 0.3, size=(N_NODES, R_DIM))
    lw = rng.normal(scale=4.0, size=N_NODES) + 30.0
    lw[rng.choice(N_NODES, 40, replace=False)] = -np.inf
    return u, lw


def _rank_main(rank: int, ws: int, port: int, q) -> None:
    try:
        os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        from paper_2509_16896_gb300 import binding, sharded
        dist.init_process_group("gloo", rank=rank, world_size=ws)
        u, lw = _nodes()
        chunk = N_NODES // ws
        rows = slice(rank * chunk, (rank + 1) * chunk)
        ul, ll = u[rows], lw[rows]
        # the chunk's record from its definition: lam_g = LSE of its rows, w = e^(l - lam_g)
        m = np.max(ll)
        lam = m + np.log(np.sum(np.exp(ll - m)))
        w = np.exp(ll - lam)
        W, Q = w.sum(), (w * w).sum()
        mean = w @ ul / W
        M2 = w @ ((ul - mean) ** 2)
        rec = np.concatenate([[lam, W, Q, 0.0], mean, M2])
        rows_all, recs = sharded.exchange(torch.tensor(ll - lam), torch.tensor(rec), dist)
        merged = binding.merge_records_host(recs.numpy(), R_DIM)
        dist.barrier()
        dist.destroy_process_group()
        q.put((rank, {"merged": merged.tolist(), "rows_all": rows_all.numpy().tolist(),
                      "recs": recs.numpy().tolist()}))
    except BaseException as e:   # report to the parent instead of hanging it
        q.put((rank, {"error": repr(e)}))


@pytest.fixture(scope="module")
def two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    try:
        for _ in range(2):
            rank, res = q.get(timeout=180)
            out[rank] = res
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.kill()
    return out


def test_ranks_agree_and_match_oracle(two_ranks):
    from oracle import filter as F
    for r in (0, 1):
        assert "error" not in two_ranks[r], two_ranks[r]
    a, b = np.array(two_ranks[0]["merged"]), np.array(two_ranks[1]["merged"])
    assert np.array_equal(a, b)                       # every rank merges the same buffers alike
    u, lw = _nodes()
    lam, lh = F.normalise(lw)
    mean, var, ess = F.estimate(u, lh)
    r = R_DIM
    assert abs(a[0] - lam) <= 1e-12 * abs(lam)
    assert abs(a[1] - 1.0) <= 1e-12
    assert abs(a[3] - ess) <= 1e-10 * ess
    assert np.max(np.abs(a[4:4 + r] - mean)) <= 1e-13
    assert np.max(np.abs(a[4 + r:] - var) / var) <= 1e-10
    # the gathered rows, shifted by each shard's lam_g - Lambda, are the normalised weights
    rows_all = np.array(two_ranks[0]["rows_all"])
    recs = np.array(two_ranks[0]["recs"])
    chunk = len(lw) // 2
    lam_g = np.repeat(recs[:, 0], chunk)
    norm = rows_all - (lam - lam_g)
    fin = np.isfinite(lh)
    assert np.array_equal(np.isfinite(norm), fin)
    assert np.max(np.abs(norm[fin] - lh[fin])) <= 1e-12


def test_merge_of_one_shard_is_its_record():
    from paper_2509_16896_gb300 import binding
    try:
        binding.load()
    except FileNotFoundError as e:
        pytest.skip(str(e))
    rec = np.array([[2.5, 1.0, 0.25, 0.0, 0.1, -0.2, 0.04, 0.09]])
    out = binding.merge_records_host(rec, 2)
    assert np.allclose(out, [2.5, 1.0, 0.25, 4.0, 0.1, -0.2, 0.04, 0.09], rtol=0, atol=1e-15)
