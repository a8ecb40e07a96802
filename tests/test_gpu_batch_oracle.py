"""Batches of ragged filters against the FP64 oracle (not only against the library's own
single-filter runs): step-local parity of every member on both prediction paths (tensor-core
screen and FP32 form), whole runs with interval restarts, and the linear-Gaussian members
against the exact discrete Kalman filter.

Bars: 1e-5 relative for the step-local outputs (the float32 bar of the single-filter
parity tests); over whole runs every step's posterior mean within 1e-3 x state scale (the
RMS of the true trajectory) of the oracle's, and the RMSE likewise; for the Kalman
comparison, the batch's RMS deviation from the Kalman mean within 1e-3 sqrt(P_inf) of the
oracle's own deviation (the method's quadrature error is the oracle's; the batch must
reproduce it); in absolute terms below 0.005 sqrt(P_inf) at n = 4096, the size the oracle
itself is pinned at (measured 4.2e-4), and reported at node counts that are not powers of
two, whose scrambled Sobol sets are not complete nets and integrate less evenly (measured
9.5e-3 at n = 3001 and 1.9e-2 at n = 5000, the oracle's values to four digits)."""
import math

import numpy as np
import pytest

from synth import simulate

from ._helpers import oracle_problem, rel_err, sobol_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5
P_INF = math.sqrt(1.25) - 0.5   # steady Kalman-Bucy variance at a = -0.5 (dP/dt = 2aP + 1 - P^2)

# (model, r, n, R, seed, path): path 0 = tensor-core screen, 1 = FP32 form
STEP_MEMBERS = [("cubic", 10, 1500, 0.3, 71, 0), ("linear", 40, 2100, 0.3, 72, 0), ("cubic", 130, 1000, 0.3, 73, 0),
                ("linear", 8, 777, 0.3, 74, 1), ("cubic", 64, 2600, 0.3, 75, 1), ("cubic", 100, 2048, 0.3, 76, 0)]


def _batch(members, N, restart_interval=0, ess_frac=0.0, paths=None):
    from paper_2509_16896_gb300 import binding
    cfgs = [binding.make_config(model=m, r=r, n=n, dt=0.01, R=R, n_scales=N, precision="bf16",
                                restart_interval=restart_interval, ess_frac=ess_frac)
            for (m, r, n, R, s, *_) in members]
    bt = binding.Batch(cfgs)
    for b, (m, r, n, R, s, *_) in enumerate(members):
        poly, scr = sobol_inputs(r, s)
        bt.filters[b].init_nodes(poly, scr, np.zeros(r))
    if paths is not None:
        bt.set_routing(paths)
    return bt


def _oracle_state(p, u, steps, seed):
    from oracle import filter as F
    tr = simulate(p.model, p.r, steps + 1, p.dt, seed=seed + 100)
    st = F.init_state(p, u, np.zeros(p.r))
    for k in range(steps):
        _, st = F.step(p, st, tr.dy[k])
    return st, tr.dy[steps]


def test_batch_step_local_parity_both_paths(yy_lib):
    import torch
    from oracle import filter as F
    members = STEP_MEMBERS
    N = 2
    bt = _batch(members, N, paths=[m[5] for m in members])
    assert list(bt.routing()) == [m[5] for m in members]
    probs, states, dys, nodes = [], [], [], []
    for b, (m, r, n, R, s, _) in enumerate(members):
        p = oracle_problem(m, r, n, 0.01, R, N)
        u, _ = bt.filters[b].get_nodes()
        st, dy = _oracle_state(p, u, 2, s)
        probs.append(p); states.append(st); dys.append(dy); nodes.append(u)
        bt.filters[b].set_state(st.centre, st.logw.astype(np.float32), st.lognorm, st.k)
    # prediction of every member in one batched launch
    bt.predict()
    for b, p in enumerate(probs):
        lw_pred, off = bt.filters[b].get_log_weights()
        prep = F.prepare(p, nodes[b], states[b].centre)
        ref, _ = F.predict(p, prep, states[b].logw.astype(np.float32).astype(np.float64))
        assert rel_err(lw_pred.astype(np.float64) + off, ref) <= TOL, b
    # one whole batched step (prediction, correction, estimate) from the same states
    for b, st in enumerate(states):
        bt.filters[b].set_state(st.centre, st.logw.astype(np.float32), st.lognorm, st.k)
    dy_all = torch.tensor(np.concatenate(dys)[None, :], dtype=torch.float64, device="cuda")
    hist = torch.zeros((1, bt.H), dtype=torch.float64, device="cuda")
    bt.run_steps(dy_all, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()[0]
    for b, (p, st) in enumerate(zip(probs, states)):
        r = p.r
        st_in = F.State(u=nodes[b], centre=st.centre, logw=st.logw.astype(np.float32).astype(np.float64),
                        lognorm=st.lognorm, k=st.k)
        rec, _ = F.step(p, st_in, dys[b], keep_logw=True)
        row = h[bt.hist_off[b]:bt.hist_off[b + 1]]
        mean, var, ess, lam, z = row[:r], row[r:2 * r], row[2 * r], row[2 * r + 1], row[2 * r + 2]
        assert np.max(np.abs(mean - rec.mean) / np.maximum(1.0, np.abs(rec.mean))) <= TOL, b
        assert np.all(np.abs(var - rec.var) <= TOL * np.abs(rec.var) + 1e-12), b
        assert abs(ess - rec.ess) <= TOL * rec.ess, b
        assert abs(lam - rec.lam) <= TOL * max(1.0, abs(rec.lam)), b
        assert abs(z - rec.lognorm) <= TOL * max(1.0, abs(rec.lognorm)), b
        lw_hat, off = bt.filters[b].get_log_weights()
        assert off == 0.0
        assert rel_err(lw_hat, rec.logw_hat) <= TOL, b


def _whole_runs(members, N, K, restart_interval, paths):
    """GPU batch histories and oracle runs of every member on the same seeded inputs."""
    import torch
    from oracle import filter as F
    bt = _batch(members, N, restart_interval=restart_interval, paths=paths)
    trs = [simulate(m, r, K, 0.01, seed=s) for (m, r, n, R, s, *_) in members]
    dy_all = torch.tensor(np.concatenate([t.dy for t in trs], axis=1), dtype=torch.float64, device="cuda")
    hist = torch.zeros((K, bt.H), dtype=torch.float64, device="cuda")
    bt.run_steps(dy_all, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    out = []
    for b, (m, r, n, R, s, *_) in enumerate(members):
        p = oracle_problem(m, r, n, 0.01, R, N, restart_interval=restart_interval)
        u, _ = bt.filters[b].get_nodes()
        recs = F.run(p, F.init_state(p, u, np.zeros(r)), trs[b].dy)
        gpu = h[:, bt.hist_off[b]:bt.hist_off[b] + r]
        ref = np.array([q.mean for q in recs])
        flags_gpu = h[:, bt.hist_off[b] + 2 * r + 3]
        flags_ref = np.array([1.0 if q.restarted else 0.0 for q in recs])
        out.append((trs[b], gpu, ref, flags_gpu, flags_ref))
    return out


def _assert_whole_run(tr, gpu, ref, b):
    scale = float(np.sqrt(np.mean(tr.x ** 2)))
    err = float(np.max(np.abs(gpu - ref)))
    rm_g = float(np.sqrt(np.mean((gpu - tr.x) ** 2)))
    rm_o = float(np.sqrt(np.mean((ref - tr.x) ** 2)))
    print(f"member {b}: max |x_hat - oracle| {err:.2e}, RMSE gpu {rm_g:.6f} oracle {rm_o:.6f} (scale {scale:.3f})")
    assert err <= 1e-3 * scale, b
    assert abs(rm_g - rm_o) <= 1e-3 * scale, b


def test_batch_linear_members_follow_the_kalman_filter(yy_lib):
    """Global box (R = 6), first-order kernel, no restart: the linear-Gaussian members track
    the exact discrete Kalman filter as the oracle does (reading A4: the Kalman pin uses
    N = 1), and a cubic member rides along in the same launches."""
    from oracle import kalman
    K = 100
    members = [("linear", 1, 4096, 6.0, 81), ("linear", 1, 3001, 6.0, 82), ("linear", 1, 5000, 6.0, 83),
               ("cubic", 2, 1024, 4.0, 84)]
    res = _whole_runs(members, 1, K, 0, paths=[0, 1, 0, 1])
    for b, (tr, gpu, ref, fg, fr) in enumerate(res):
        _assert_whole_run(tr, gpu, ref, b)
        if members[b][0] != "linear":
            continue
        km, _ = kalman.kalman_filter(tr.dy, -0.5, 0.01)
        dev_gpu = float(np.sqrt(np.mean((gpu - km) ** 2)))
        dev_ref = float(np.sqrt(np.mean((ref - km) ** 2)))
        print(f"member {b}: RMS |x_hat - KF| gpu {dev_gpu:.3e} oracle {dev_ref:.3e} (sqrt P_inf {math.sqrt(P_INF):.3f})")
        assert abs(dev_gpu - dev_ref) <= 1e-3 * math.sqrt(P_INF), b
        if members[b][2] == 4096:
            assert dev_gpu <= 0.005 * math.sqrt(P_INF), b


def test_batch_local_box_members_match_oracle_runs(yy_lib):
    """The batched workload's shape: local boxes R = 0.3 re-centred every second step,
    N = 2, half cubic and half linear, ragged r and n, both prediction paths.  Posterior
    means follow the oracle's run; the linear members' deviation from the Kalman filter is
    the oracle's (reported)."""
    from oracle import kalman
    K = 30
    members = [("cubic", 12, 2048, 0.3, 91), ("linear", 10, 2048, 0.3, 92), ("cubic", 70, 1500, 0.3, 93),
               ("linear", 33, 3000, 0.3, 94)]
    res = _whole_runs(members, 2, K, 2, paths=[1, 0, 0, 1])
    for b, (tr, gpu, ref, fg, fr) in enumerate(res):
        assert np.array_equal(fg, fr), b
        _assert_whole_run(tr, gpu, ref, b)
        if members[b][0] == "linear":
            km, _ = kalman.kalman_filter(tr.dy, -0.5, 0.01)
            dev_gpu = float(np.sqrt(np.mean((gpu - km) ** 2)))
            dev_ref = float(np.sqrt(np.mean((ref - km) ** 2)))
            print(f"member {b} (r={members[b][1]}): RMS |x_hat - KF| gpu {dev_gpu:.4f} oracle {dev_ref:.4f}")
            assert abs(dev_gpu - dev_ref) <= 1e-3 * math.sqrt(P_INF), b
