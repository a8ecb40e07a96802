"""The tensor-core prediction on CTA pairs (2-CTA clusters, tcgen05.mma.cta_group::2)
against the same prediction on single CTAs and against the FP64 oracle.

Each CTA of a pair screens its own 128 target rows exactly as a single CTA does; only the
staging of the source tiles (half per CTA) and the issue of the Gram products (one M = 256
instruction for both) differ.  With the first-pass length fixed, both forms therefore
take the same screening decisions: the exact-pair and tile counters must be equal, and
the predicted log-weights agree to float32 rounding (the column-direction terms of the
symmetric screen are added by compare-and-swap, in an order that is not deterministic
even between two runs of one form).  Cases: the self-term regime at high r (FP8 and BF16
operands), tens of millions of exact pairs with escalations to the second pass and split
source ranges, short rows (r <= 64), and ragged node counts."""
import os

import numpy as np
import pytest

from synth import simulate, sobol_poly_params, sobol_scramble_params

from ._helpers import rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # r, n, R, N, screen, first-pass stages (0: device-chosen, compared to the oracle only)
    (1000, 8192, 0.3, 3, "fp8", 4),
    (100, 16384, 0.3, 2, "bf16", 1),
    (80, 32768, 0.16, 2, "bf16", 1),
    (72, 40000, 0.17, 3, "fp8", 0),
    (8, 4096, 0.5, 2, "bf16", 0),
    (300, 5000, 0.3, 1, "bf16", 2),
]


def _filter(r, n, R, N, screen, prefix, seed):
    import torch
    from paper_2509_16896_gb300 import binding
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=R, n_scales=N, precision="bf16",
                              restart_interval=2, ess_frac=0.5, screen_type=screen, screen_prefix=prefix)
    flt = binding.Filter(cfg, stream=torch.cuda.Stream())
    flt.init_nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), np.zeros(r))
    return flt


@pytest.mark.parametrize("r,n,R,N,screen,prefix", CASES)
def test_pair_matches_single_cta_and_oracle(yy_lib, r, n, R, N, screen, prefix):
    import torch
    from oracle import filter as F
    seed = 23
    flt = _filter(r, n, R, N, screen, prefix, seed)
    assert flt.set_cta_pair(True) > 0                 # an unsplit filter runs on pairs
    tr = simulate("cubic", r, 3, 0.01, seed=seed)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(flt.stream):
        flt.run_steps(dy)
    torch.cuda.synchronize()
    centre, _, _ = flt.get_state()
    _, half = flt.get_box()
    logw, off = flt.get_log_weights()
    u, mask = flt.get_nodes()

    def predict(pair):
        active = flt.set_cta_pair(pair)
        assert (active > 0) == pair
        flt.predict()
        pred, poff = flt.get_log_weights()
        _, exact = flt.counters()          # exact pairs of this prediction
        last, _, tiles, resc = flt.screen()
        return pred.astype(np.float64) + poff, exact, (last, tiles, resc)

    p_pair, ex_pair, sc_pair = predict(True)
    p_one, ex_one, sc_one = predict(False)
    p_pair2, ex_pair2, sc_pair2 = predict(True)
    print(f"r={r} n={n} {screen}: exact pairs {ex_pair} / {ex_one}, screen {sc_pair} / {sc_one}")
    assert np.array_equal(np.isneginf(p_pair), mask) and np.array_equal(np.isneginf(p_one), mask)
    assert not np.any(np.isnan(p_pair))
    if prefix > 0:   # fixed first pass: identical screening decisions and Gram blocks
        assert ex_pair == ex_one == ex_pair2
        assert sc_pair[:2] == sc_one[:2] == sc_pair2[:2]
        # a pair rescreens a tile for both CTAs when either marked it
        assert sc_one[2] <= sc_pair[2] <= 2 * sc_one[2]
    fin = np.isfinite(p_one)
    d = np.abs(p_pair[fin] - p_one[fin]) / np.maximum(1.0, np.abs(p_one[fin]))
    assert d.max(initial=0.0) <= 2e-6, d.max()
    # and against the oracle, on row blocks at the start, the ragged end and inside
    p = F.Problem(model="cubic", r=r, n=n, dt=0.01, R=half.copy(), n_scales=N)
    prep = F.prepare(p, u, centre, half)
    lw = logw.astype(np.float64) + off
    rng = np.random.Generator(np.random.Philox(key=911 + r))
    starts = sorted(set([0, n - 16] + [int(s) for s in rng.integers(0, n - 16, size=3)]))
    threads = os.cpu_count() or 1
    worst = 0.0
    for s0 in starts:
        ref, _ = F.predict(p, prep, lw, s0, s0 + 16, n_threads=threads)
        worst = max(worst, rel_err(p_pair[s0:s0 + 16], ref))
    assert worst <= 1e-5, worst


def test_pair_schedule_for_shards_and_ragged_ends(yy_lib):
    """Whole filters and shards run on pairs, including a last shard whose rows end inside
    a 256-row block (its partner tile is padding); single CTAs are the default."""
    r, n = 96, 4096 + 384    # 35 target tiles of 128
    flt = _filter(r, n, 0.3, 2, "bf16", 1, 5)
    assert flt.set_cta_pair(False) == 0
    assert flt.set_cta_pair(True) > 0
    assert flt.set_cta_pair(False) == 0
    for rank in (0, 1):
        sh = _filter(r, n, 0.3, 2, "bf16", 1, 5)
        sh.set_shard(rank, 2)
        assert sh.set_cta_pair(True) > 0


def test_sharded_pairs_match_the_whole_filter(yy_lib):
    """Two shards on CTA pairs, merged, follow the whole filter (single CTAs) over steps with
    restarts, to float32 rounding."""
    import torch
    from paper_2509_16896_gb300 import binding
    r, n, seed, G = 130, 6000, 9, 2
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=0.3, n_scales=2, precision="bf16",
                              restart_interval=2, ess_frac=0.5, screen_prefix=1)

    def make():
        f = binding.Filter(cfg)
        f.init_nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), np.zeros(r))
        return f

    whole = make()
    shards = []
    for g in range(G):
        f = make()
        f.set_shard(g, G)
        assert f.set_cta_pair(True) > 0
        shards.append(f)
    chunk = shards[0].shard_rows()[1]
    tr = simulate("cubic", r, 4, 0.01, seed=seed)
    dys = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    tol = 1e-5
    for k in range(4):
        whole.predict()
        whole.update(dys[k])
        mw, vw, ew, zw = whole.estimate()
        rows = [torch.empty(chunk, dtype=torch.float32, device="cuda") for _ in range(G)]
        recs = torch.empty((G, 2 * r + 4), dtype=torch.float64, device="cuda")
        for g, s in enumerate(shards):
            s.predict()
            s.update_shard(dys[k], rows[g], recs[g])
        torch.cuda.synchronize()
        rows_all = torch.cat(rows)
        for s in shards:
            s.merge_shards(rows_all, recs, G)
        for g, s in enumerate(shards):
            m, v, e, z = s.estimate()
            assert np.max(np.abs(m - mw) / np.maximum(1.0, np.abs(mw))) <= tol, (k, g)
            assert np.all(np.abs(v - vw) <= tol * np.abs(vw) + 1e-12), (k, g)
            assert abs(e - ew) <= tol * ew, (k, g)
            assert abs(z - zw) <= tol * max(1.0, abs(zw)), (k, g)
        did = whole.restart(mode=0, report=True)
        for s in shards:
            assert s.restart(mode=0, report=True) == did
