"""FP64 reference of the restart-proposal network (a library addition; the paper's
restart, "Local Resampling-Restart Mechanism", re-centres the box at the estimate with a fixed
half-width).

Network: features z = [x_hat - c; sqrt(v_hat); dy / sqrt(dt)] in R^{3r} (c the centre of the box the
estimate was computed in, so the first block is how far the posterior moved inside it), normalised per
feature and clamped, zn = clip((z - mu) / s, -4, 4) (mu, s from the training set), ->
    h1 = relu(W1 zn + b1),  h2 = relu(W2 h1 + b2),  o = W3 h2 + b3,  o = [delta; lambda] in R^{2r}.
Proposed box: centre x_hat + delta, half-widths R exp(lambda); it falls back to the plain
rule when a value is not finite, a half-width leaves [R/8, 8R], or the box would not
contain the current estimate (|delta_d| > R exp(lambda_d)).

Training target: the true state's offset t = x_true - x_hat at each restart of a plain run.
Loss (Gaussian negative log-likelihood with sigma = (R/3) exp(lambda), so that the box
half-width is 3 sigma), averaged over rows and coordinates:
    L = mean_{b,d} [ (t - delta)^2 / (2 sigma^2) + log sigma ].

Everything here is plain numpy in float64: forward, the hand-derived backward pass, and
Adam (Kingma & Ba, 2015).  forward and backward take an optional operand rounding `rnd`
applied to both operands of every matrix product (identity by default); with a rounding
to bfloat16 they give the exact products of the rounded operands that a BF16 tensor-core
implementation accumulates, which separates its accumulation error from its operand
rounding.
"""
from __future__ import annotations

import numpy as np


def init_params(r: int, hidden: int, seed: int) -> dict:
    """He-uniform initialisation (the CUDA path receives these values as inputs)."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(seed) ^ np.uint64(0x3A11)))
    dims = [(hidden, 3 * r), (hidden, hidden), (2 * r, hidden)]
    p = {}
    for i, (o, n_in) in enumerate(dims, start=1):
        lim = np.sqrt(6.0 / n_in)
        p[f"W{i}"] = rng.uniform(-lim, lim, size=(o, n_in))
        p[f"b{i}"] = np.zeros(o)
    p["W3"] *= 0.01   # start near the plain rule: delta ~ 0, lambda ~ 0
    p["mu"] = np.zeros(3 * r)
    p["s"] = np.ones(3 * r)
    return p


TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3")


def normalise(p: dict, z: np.ndarray) -> np.ndarray:
    mu = p.get("mu", np.zeros(z.shape[-1]))
    s = p.get("s", np.ones(z.shape[-1]))
    return np.clip((z - mu) / s, -4.0, 4.0)


def _identity(a: np.ndarray) -> np.ndarray:
    return a


def forward(p: dict, z_raw: np.ndarray, rnd=None) -> tuple[np.ndarray, dict]:
    q = rnd or _identity
    z = normalise(p, z_raw)
    a1 = q(z) @ q(p["W1"]).T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = q(h1) @ q(p["W2"]).T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    o = q(h2) @ q(p["W3"]).T + p["b3"]
    return o, {"z": z, "a1": a1, "h1": h1, "a2": a2, "h2": h2}


def loss_and_grad_out(o: np.ndarray, t: np.ndarray, R: float) -> tuple[float, np.ndarray]:
    """NLL of the module docstring and its gradient with respect to o = [delta; lambda]."""
    B, two_r = o.shape
    r = two_r // 2
    delta, lam = o[:, :r], o[:, r:]
    sigma = (R / 3.0) * np.exp(lam)
    e = t - delta
    L = float(np.mean(e * e / (2.0 * sigma * sigma) + np.log(sigma)))
    g = np.empty_like(o)
    scale = 1.0 / (B * r)
    g[:, :r] = -e / (sigma * sigma) * scale
    g[:, r:] = (1.0 - e * e / (sigma * sigma)) * scale
    return L, g


def backward(p: dict, cache: dict, g_o: np.ndarray, rnd=None) -> dict:
    q = rnd or _identity
    g = {}
    g["W3"] = q(g_o).T @ q(cache["h2"])
    g["b3"] = g_o.sum(axis=0)
    g_h2 = q(g_o) @ q(p["W3"])
    g_a2 = g_h2 * (cache["a2"] > 0)
    g["W2"] = q(g_a2).T @ q(cache["h1"])
    g["b2"] = g_a2.sum(axis=0)
    g_h1 = q(g_a2) @ q(p["W2"])
    g_a1 = g_h1 * (cache["a1"] > 0)
    g["W1"] = q(g_a1).T @ q(cache["z"])
    g["b1"] = g_a1.sum(axis=0)
    return g


def adam_step(p: dict, g: dict, m: dict, v: dict, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    for k in g:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def features(mean: np.ndarray, var: np.ndarray, dy: np.ndarray, dt: float, centre: np.ndarray) -> np.ndarray:
    return np.concatenate([mean - centre, np.sqrt(np.maximum(var, 0.0)), dy / np.sqrt(dt)])


def proposal(p: dict, mean: np.ndarray, var: np.ndarray, dy: np.ndarray, dt: float, R: np.ndarray,
             centre: np.ndarray):
    """(centre, half-widths, accepted) of the learned box; plain box when rejected.  centre:
    the current box's centre."""
    r = mean.shape[0]
    o, _ = forward(p, features(mean, var, dy, dt, centre)[None, :])
    delta, lam = o[0, :r], o[0, r:]
    half = R * np.exp(lam)
    ok = bool(np.all(np.isfinite(delta)) and np.all(np.isfinite(half))
              and np.all(half >= R / 8) and np.all(half <= 8 * R) and np.all(np.abs(delta) <= half))
    if not ok:
        return mean.copy(), R.copy(), False
    return mean + delta, half, True
