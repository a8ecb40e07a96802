"""FP64 reference of the restart-proposal network (a library addition; the paper's
restart, Section 5, re-centres the box at the estimate with a fixed half-width).

Network: features z = [x_hat; sqrt(v_hat); dy / sqrt(dt)] in R^{3r}, normalised per
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
Adam (Kingma & Ba, 2015).
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


def forward(p: dict, z_raw: np.ndarray) -> tuple[np.ndarray, dict]:
    z = normalise(p, z_raw)
    a1 = z @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    o = h2 @ p["W3"].T + p["b3"]
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


def backward(p: dict, cache: dict, g_o: np.ndarray) -> dict:
    g = {}
    g["W3"] = g_o.T @ cache["h2"]
    g["b3"] = g_o.sum(axis=0)
    g_h2 = g_o @ p["W3"]
    g_a2 = g_h2 * (cache["a2"] > 0)
    g["W2"] = g_a2.T @ cache["h1"]
    g["b2"] = g_a2.sum(axis=0)
    g_h1 = g_a2 @ p["W2"]
    g_a1 = g_h1 * (cache["a1"] > 0)
    g["W1"] = g_a1.T @ cache["z"]
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


def features(mean: np.ndarray, var: np.ndarray, dy: np.ndarray, dt: float) -> np.ndarray:
    return np.concatenate([mean, np.sqrt(np.maximum(var, 0.0)), dy / np.sqrt(dt)])


def proposal(p: dict, mean: np.ndarray, var: np.ndarray, dy: np.ndarray, dt: float, R: np.ndarray):
    """(centre, half-widths, accepted) of the learned box; plain box when rejected."""
    r = mean.shape[0]
    o, _ = forward(p, features(mean, var, dy, dt)[None, :])
    delta, lam = o[0, :r], o[0, r:]
    half = R * np.exp(lam)
    ok = bool(np.all(np.isfinite(delta)) and np.all(np.isfinite(half))
              and np.all(half >= R / 8) and np.all(half <= 8 * R) and np.all(np.abs(delta) <= half))
    if not ok:
        return mean.copy(), R.copy(), False
    return mean + delta, half, True
