"""Learned restart proposal: data from plain runs, training and evaluation on the GPU.

The proposal network (include/yy.h, network section) maps the estimate's moments and the
latest observation increment to a shift and scale of the next local box.  It learns from
the restarts of the plain method: at every restart of a plain run on training
trajectories the features [x_hat - c; sqrt(v_hat); dy / sqrt(dt)] (c the centre of the box
the estimate was computed in: the estimate at the previous restart, or the initial centre)
and the offset of the true state from the estimate, x_true - x_hat, are recorded.  Everything runs through the
library: the plain runs are one batch (all trajectories advance together), training uses
the library's forward/backward/Adam kernels, and the evaluation runs the learned rule
inside the filter's restart on the device, against the plain rule on the same data.
"""
from __future__ import annotations

import numpy as np

from . import binding


def collect_restarts(workload, seeds, precision: str = "bf16", device: str = "cuda:0"):
    """Runs the plain filter on every seed (as one batch) and returns (X [M][3r], T [M][r])
    float32 arrays of the restarts, plus the batch's plain RMSE per seed."""
    import torch

    from synth import simulate, sobol_poly_params, sobol_scramble_params
    w = workload.with_(restart_rule="plain")
    cfgs = [binding.config_from_workload(w, precision=precision) for _ in seeds]
    bt = binding.Batch(cfgs, device=device)
    trs = []
    for b, s in enumerate(seeds):
        bt.filters[b].init_nodes(sobol_poly_params(w.r, s), sobol_scramble_params(w.r, s), np.zeros(w.r))
        trs.append(simulate(w.model, w.r, w.steps, w.dt, seed=s, model_a=w.model_a))
    dy = torch.tensor(np.concatenate([t.dy for t in trs], axis=1), dtype=torch.float64, device=device)
    hist = torch.zeros((w.steps, bt.H), dtype=torch.float64, device=device)
    with torch.cuda.stream(bt.stream):
        bt.run_steps(dy, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    xs, ts, rmses = [], [], []
    r = w.r
    for b, t in enumerate(trs):
        row = h[:, bt.hist_off[b]:bt.hist_off[b + 1]]
        mean, var, flag = row[:, :r], row[:, r:2 * r], row[:, 2 * r + 3]
        rmses.append(float(np.sqrt(np.mean((mean - t.x) ** 2))))
        k = np.where(flag > 0.5)[0]
        # box centre in force at step j: the plain rule re-centres at x_hat of every restart step
        centre = np.zeros_like(mean)
        last = np.zeros(r)
        for j in range(mean.shape[0]):
            centre[j] = last
            if flag[j] > 0.5:
                last = mean[j]
        feats = np.concatenate([mean[k] - centre[k], np.sqrt(np.maximum(var[k], 0.0)), t.dy[k] / np.sqrt(w.dt)],
                               axis=1)
        xs.append(feats)
        ts.append(t.x[k] - mean[k])
    bt.close()
    return (np.concatenate(xs).astype(np.float32), np.concatenate(ts).astype(np.float32),
            np.array(rmses))


def train_proposal(r: int, X: np.ndarray, T: np.ndarray, R: float, hidden: int = 256, epochs: int = 20,
                   batch: int = 256, lr: float = 1e-3, seed: int = 0, init_params: np.ndarray | None = None,
                   clip: float | None = None, device: str = "cuda:0"):
    """Trains a fresh network on (X, T); returns (network, last mini-batch loss).

    clip (default R): the targets are clipped to [-clip, clip] first.  A box can only be
    moved within its own scale (the proposal must contain the estimate), and offsets far
    beyond it -- frequent when the plain filter has lost track -- otherwise dominate the
    loss and make training diverge."""
    import torch
    clip = R if clip is None else clip
    T = np.clip(T, -clip, clip) if clip > 0 else T
    net = binding.MLP(r, hidden, max_batch=batch, device=device)
    if init_params is not None:
        net.set_params(init_params)
    # per-feature statistics of the training set, applied (and clamped) before layer 1
    net.set_input_norm(X.mean(axis=0), np.maximum(X.std(axis=0), 1e-3))
    xd = torch.tensor(X, device=device)
    td = torch.tensor(T, device=device)
    loss = net.train(xd, td, R, epochs, batch, lr, seed)
    return net, loss


def run_filter(workload, seed: int, rule: str, net=None, precision: str = "bf16", device: str = "cuda:0"):
    """One trajectory with the given restart rule; returns (RMSE, steps/s, restarts)."""
    import torch

    from synth import simulate, sobol_poly_params, sobol_scramble_params
    w = workload.with_(restart_rule=rule)
    cfg = binding.config_from_workload(w, precision=precision)
    stream = torch.cuda.Stream(device)
    f = binding.Filter(cfg, device=device, stream=stream)
    f.init_nodes(sobol_poly_params(w.r, seed), sobol_scramble_params(w.r, seed), np.zeros(w.r))
    if rule == "learned":
        f.set_restart_mlp(net)
    tr = simulate(w.model, w.r, w.steps, w.dt, seed=seed, model_a=w.model_a)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device=device)
    hist = torch.zeros((w.steps, 2 * w.r + 4), dtype=torch.float64, device=device)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        f.run_steps(dy, hist)
    e1.record(stream)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    rmse = float(np.sqrt(np.mean((h[:, :w.r] - tr.x) ** 2)))
    return rmse, w.steps / (e0.elapsed_time(e1) / 1e3), int(h[:, 2 * w.r + 3].sum())


def constant_box_network(r: int, lam: float, hidden: int = 256, device: str = "cuda:0"):
    """A network whose output is the constant [0; lam] (no shift, every half-width R e^lam):
    the plain rule with a wider or narrower fixed box, the ablation of a trained network
    whose output does not depend on its input."""
    p = {"W1": np.zeros((hidden, 3 * r)), "b1": np.zeros(hidden), "W2": np.zeros((hidden, hidden)),
         "b2": np.zeros(hidden), "W3": np.zeros((2 * r, hidden)), "b3": np.concatenate([np.zeros(r), np.full(r, lam)])}
    net = binding.MLP(r, hidden, max_batch=8, device=device)
    net.set_params(binding.pack_mlp_params(p))
    return net


def output_spread(net, X: np.ndarray, r: int, device: str = "cuda:0"):
    """(mean over coordinates of the row-to-row standard deviation of delta, of lambda, and the
    mean lambda) of the network's proposals on rows X: how much the proposal depends on its
    input."""
    import torch
    out = net.forward(torch.tensor(X, device=device)).cpu().numpy()
    return float(out[:, :r].std(axis=0).mean()), float(out[:, r:].std(axis=0).mean()), float(out[:, r:].mean())


def judge(workload, candidates: dict, seeds, device: str = "cuda:0"):
    """Mean RMSE of each candidate rule over the seeds; candidates maps a name to None (the
    plain rule) or a network (the learned rule with it).  The plain rule is the judge: the
    selection is the candidate with the smallest mean, the plain rule on a tie."""
    res = {}
    for name, net in candidates.items():
        rule = "plain" if net is None else "learned"
        res[name] = float(np.mean([run_filter(workload, s, rule, net=net, device=device)[0] for s in seeds]))
    best = min(res, key=lambda k: (res[k], 0 if candidates[k] is None else 1))
    return best, res
