"""Whole runs of the mixed-precision path (Gram screen on BF16 or FP8 operands, exact
float32 survivors, float32 log-sum-exp, float64 normaliser and moment merges) against the
FP64 oracle on the same seeded inputs, at the shapes of the r = 100 and r = 50 workloads:
the cubic sensor with local boxes R = 0.3 re-centred by the interval rule and by the ESS
test.

Bars: |RMSE_gpu - RMSE_oracle| <= 1e-3 x state scale (the RMS of the true trajectory), and
every step's posterior mean within 1e-3 x state scale of the oracle's.  Restart decisions
must agree except at a tie (|ESS - rho n| < 1e-3 n, reading A12), where the comparison
stops.  The measured error of every output (posterior mean and variance, ESS, Lambda_k,
Z_k) is printed for the record."""
import os

import numpy as np
import pytest

from synth import simulate, sobol_poly_params, sobol_scramble_params

pytestmark = pytest.mark.gpu

_ORACLE_RUNS = {}


def _oracle_run(model, r, n, R, N, K, seed, u):
    from oracle import filter as F
    key = (model, r, n, R, N, K, seed)
    if key not in _ORACLE_RUNS:
        p = F.Problem(model=model, r=r, n=n, dt=0.01, R=np.full(r, R), n_scales=N, restart_interval=2,
                      ess_frac=0.5)
        tr = simulate(model, r, K, 0.01, seed=seed)
        recs = F.run(p, F.init_state(p, u, np.zeros(r)), tr.dy, n_threads=os.cpu_count() or 1)
        _ORACLE_RUNS[key] = (p, tr, recs)
    return _ORACLE_RUNS[key]


@pytest.mark.parametrize("r,n,N,K,screen", [(100, 16384, 2, 24, "bf16"), (100, 16384, 2, 24, "fp8"),
                                            (50, 8192, 2, 100, "bf16")])
def test_mixed_precision_whole_run_matches_oracle(yy_lib, r, n, N, K, screen):
    import torch
    from paper_2509_16896_gb300 import binding
    model, R, seed = "cubic", 0.3, 2 if r == 100 else 5
    cfg = binding.make_config(model=model, r=r, n=n, dt=0.01, R=R, n_scales=N, precision="bf16",
                              restart_interval=2, ess_frac=0.5, screen_type=screen)
    stream = torch.cuda.Stream()
    flt = binding.Filter(cfg, stream=stream)
    flt.init_nodes(sobol_poly_params(r, seed), sobol_scramble_params(r, seed), np.zeros(r))
    u, _ = flt.get_nodes()
    p, tr, recs = _oracle_run(model, r, n, R, N, K, seed, u)
    dy = torch.tensor(tr.dy, dtype=torch.float64, device="cuda")
    hist = torch.zeros((K, 2 * r + 4), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        flt.run_steps(dy, hist)
    torch.cuda.synchronize()
    h = hist.cpu().numpy()
    g_mean, g_var, g_ess, g_lam, g_z, g_flag = (h[:, :r], h[:, r:2 * r], h[:, 2 * r], h[:, 2 * r + 1],
                                                h[:, 2 * r + 2], h[:, 2 * r + 3])
    o_mean = np.array([q.mean for q in recs])
    o_var = np.array([q.var for q in recs])
    o_ess = np.array([q.ess for q in recs])
    o_lam = np.array([q.lam for q in recs])
    o_z = np.array([q.lognorm for q in recs])
    o_flag = np.array([1.0 if q.restarted else 0.0 for q in recs])
    # compare up to the first restart decision that differs; it must be a tie
    Kc = K
    diff = np.nonzero(g_flag != o_flag)[0]
    if diff.size:
        k = int(diff[0])
        assert abs(o_ess[k] - 0.5 * n) < 1e-3 * n, f"restart decisions fork at step {k} without a tie"
        Kc = k + 1
    scale = float(np.sqrt(np.mean(tr.x[:Kc] ** 2)))
    rm_g = float(np.sqrt(np.mean((g_mean[:Kc] - tr.x[:Kc]) ** 2)))
    rm_o = float(np.sqrt(np.mean((o_mean[:Kc] - tr.x[:Kc]) ** 2)))
    err = {
        "mean_abs": float(np.max(np.abs(g_mean[:Kc] - o_mean[:Kc]))),
        "var_rel": float(np.max(np.abs(g_var[:Kc] - o_var[:Kc]) / np.maximum(o_var[:Kc], 1e-300))),
        "ess_rel": float(np.max(np.abs(g_ess[:Kc] - o_ess[:Kc]) / o_ess[:Kc])),
        "lam_abs": float(np.max(np.abs(g_lam[:Kc] - o_lam[:Kc]))),
        "z_rel": float(np.max(np.abs(g_z[:Kc] - o_z[:Kc]) / np.maximum(1.0, np.abs(o_z[:Kc])))),
    }
    print(f"r={r} n={n} N={N} {screen} steps {Kc}/{K} restarts {int(g_flag[:Kc].sum())}: "
          f"RMSE gpu {rm_g:.6f} oracle {rm_o:.6f} |diff| {abs(rm_g - rm_o):.2e} (scale {scale:.3f}); "
          + " ".join(f"{k} {v:.2e}" for k, v in err.items()))
    assert Kc >= min(K, 10)
    assert abs(rm_g - rm_o) <= 1e-3 * scale
    assert err["mean_abs"] <= 1e-3 * scale
