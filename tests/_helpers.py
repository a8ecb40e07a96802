"""Shared set-up for the parity tests: the same seeded inputs for the oracle and the
CUDA library (nothing here does filter arithmetic)."""
from __future__ import annotations

import numpy as np

from synth import sobol_poly_params, sobol_scramble_params


def sobol_inputs(r: int, seed: int, scrambled: bool = True):
    poly = sobol_poly_params(r, seed)
    scr = sobol_scramble_params(r, seed) if scrambled else None
    return poly, scr


def oracle_problem(model, r, n, dt, R, N, restart_interval=0, ess_frac=0.0, a=-0.5,
                   restart_init="gauss", prior_mean=0.0, prior_var=1.0, noise=None):
    from oracle import filter as F
    return F.Problem(model=model, r=r, n=n, dt=dt, R=np.full(r, float(R)), n_scales=N, model_a=a,
                     restart_interval=restart_interval, ess_frac=ess_frac, prior_mean=prior_mean,
                     prior_var=prior_var, restart_init=restart_init, noise=noise)


def rel_err(a, b, floor=1.0):
    """max |a - b| / max(floor, |b|) over finite entries; -inf must match exactly."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ia, ib = np.isneginf(a), np.isneginf(b)
    assert np.array_equal(ia, ib), f"-inf pattern differs at {np.where(ia != ib)[0][:10]}"
    fin = ~ib
    if not np.any(fin):
        return 0.0
    return float(np.max(np.abs(a[fin] - b[fin]) / np.maximum(floor, np.abs(b[fin]))))


def combination_err_ok(gpu, ref, Lj, coef, logw, tol, eps=2.0 ** -24):
    """True if every finite predicted log-weight is within tol max(1, |ref|) plus the
    float32 error the multi-scale combination amplifies: its condition number
    kappa_i = sum_j |c_j e^{L_j}| / |sum_j c_j e^{L_j}| (identity term included) times a few
    ulps of the largest |L_j(i)| (the per-scale sums carry that much float32 error).
    -inf must match exactly."""
    gpu = np.asarray(gpu, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert np.array_equal(np.isneginf(gpu), np.isneginf(ref))
    N = Lj.shape[1]
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        terms = np.concatenate([np.exp(Lj - ref[:, None]) * coef[:N], (coef[N] * np.exp(logw - ref))[:, None]],
                               axis=1)
        kappa = np.abs(terms).sum(1) / np.abs(terms.sum(1))
    fin = np.isfinite(ref)
    big = np.max(np.abs(np.where(np.isfinite(Lj), Lj, 0.0)), axis=1)
    bound = tol * np.maximum(1.0, np.abs(ref)) + 8 * eps * kappa * np.maximum(big, np.abs(ref))
    return bool(np.all(np.abs(gpu[fin] - ref[fin]) <= bound[fin])), float(np.nanmax(kappa[fin]))
