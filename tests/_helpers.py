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
                   restart_init="gauss", prior_mean=0.0, prior_var=1.0):
    from oracle import filter as F
    return F.Problem(model=model, r=r, n=n, dt=dt, R=np.full(r, float(R)), n_scales=N, model_a=a,
                     restart_interval=restart_interval, ess_frac=ess_frac, prior_mean=prior_mean,
                     prior_var=prior_var, restart_init=restart_init)


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
