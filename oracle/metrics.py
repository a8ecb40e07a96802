"""Error metrics of "Numerical Experiments" (error metrics):
RMSE = sqrt( sum_k |x_hat_k - x_k|^2 / (K r) ),  ME = (1/K) sum_k sqrt(|x_hat_k - x_k|^2 / r)."""
from __future__ import annotations

import numpy as np


def rmse(est: np.ndarray, truth: np.ndarray) -> float:
    K, r = truth.shape
    return float(np.sqrt(np.sum((est - truth) ** 2) / (K * r)))


def me(est: np.ndarray, truth: np.ndarray) -> float:
    K, r = truth.shape
    return float(np.mean(np.sqrt(np.sum((est - truth) ** 2, axis=1) / r)))
