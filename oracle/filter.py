"""One step of the improved Yau--Yau filter in float64, in the paper's order.

Per step k ("Procedure for the Improved Yau-Yau Algorithm"; log-domain forms of "Log-Domain
Computation"):
  1. prediction  ell_pred(i) = log( sum_j c_j e^{L_j(i)} + c_{N+1} e^{ell(i)} ), the N-scale
     kernel of eq. general_kernel applied to the weights ("Solving Kolmogorov Equations
     via Low-Discrepancy Sampling and Kernel Approximation"), with
     L_j(i) = LSE over unmasked sources of log K_{dt/s_j}(x_i, x_s) + log w_q + ell(s)
     (computed by the C core, see csrc/yyo_kernel.c); the identity term carries no
     quadrature factor.  Targets on the Dirichlet boundary get -inf ("Algorithm for Kolmogorov
     Equation", step 3).
     Negative coefficients are handled by a signed log-sum-exp; a non-positive total
     gives -inf and is counted.
  2. correction  ell'(i) = ell_pred(i) + h(x_i).dy_k - dt/2 |h(x_i)|^2 (online stage of
     "Procedure for the Improved Yau-Yau Algorithm"; observation update of "Log-Domain
     Computation").
  3. normalisation  Lambda_k = LSE_i ell'(i), ell_hat = ell' - Lambda_k (normalisation in
     "Log-Domain Computation"); running log-normaliser Z_k = Z_{k-1} + Lambda_k, Z_0 = 0 (the prior
     weights are normalised at initialisation).
  4. estimate  x_hat = sum w_hat x ("Procedure for the Improved Yau-Yau Algorithm", step 4);
     variance v_hat = sum w_hat (x - x_hat)^2; ESS = 1 / sum w_hat^2.
  5. restart  ("Local Resampling-Restart Mechanism"): when ESS < rho n, or iota >= 2 and
     k mod iota == 0, the box is re-centred at x_hat, the reference nodes are translated (the same u), and the
     weights are re-initialised from N(c, diag(max(v_hat, v_min))), v_min = (R/4)^2,
     c the new centre, or uniformly.  Z is left unchanged by a restart.  With the learned
     rule (a library addition, see oracle/mlp.py) the centre is x_hat + delta and the
     half-widths R exp(lambda); the reference nodes are re-mapped from their Sobol
     integers to the new half-widths.

Nodes are held as float32 box coordinates u (what both implementations store) and
float64 centre c; positions are x = c + u in float64.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib, coeffs, model as mdl


@dataclass
class Problem:
    model: str
    r: int
    n: int
    dt: float
    R: np.ndarray                 # [r] half-widths
    n_scales: int
    model_a: float = -0.5
    restart_interval: int = 0
    ess_frac: float = 0.0
    prior_mean: float = 0.0
    prior_var: float = 1.0
    restart_init: str = "gauss"   # "gauss" | "uniform"
    restart_rule: str = "plain"   # "plain" | "learned"
    mlp_params: dict | None = None
    noise: dict | None = None     # diagonal noise coefficients (model.state_noise); None: unit

    @property
    def taus(self) -> np.ndarray:
        return self.dt / coeffs.scales(self.n_scales)

    @property
    def log_wq(self) -> float:
        return log_wq(self.R, self.n)

    @property
    def coef(self) -> np.ndarray:
        return coeffs.kernel_coefficients(self.n_scales)


@dataclass
class Prepared:
    x: np.ndarray      # [n][r] float64
    f: np.ndarray      # [n][r]
    divf: np.ndarray   # [n]
    mask: np.ndarray   # [n] bool
    minv: np.ndarray | None = None   # [n][r] a(x)^+ (diagonal) with noise coefficients
    hld: np.ndarray | None = None    # [n] 1/2 log det_+ a(x)


def log_wq(half: np.ndarray, n: int) -> float:
    """Quadrature volume per node of the box with these half-widths ("Discrete Solution-Mapping
    Operator Construction", remark)."""
    return float(np.sum(np.log(2.0 * half)) - np.log(n))


def boundary_mask(u: np.ndarray, R: np.ndarray) -> np.ndarray:
    """Nodes within omega = 1e-12 R of a face of [-R, R]^r ("Algorithm for Kolmogorov
    Equation", step 3)."""
    uu = np.abs(u.astype(np.float64))
    return np.any(uu >= R[None, :] - 1e-12 * R[None, :], axis=1)


def prepare(p: Problem, u: np.ndarray, centre: np.ndarray, half: np.ndarray | None = None) -> Prepared:
    x = centre[None, :].astype(np.float64) + u.astype(np.float64)
    minv, hld = mdl.kernel_metric(p.noise, x) if p.noise is not None else (None, None)
    return Prepared(x=x, f=mdl.drift(p.model, x, p.model_a),
                    divf=mdl.divergence(p.model, x, p.model_a),
                    mask=boundary_mask(u, p.R if half is None else half), minv=minv, hld=hld)


def log_sum_exp(a: np.ndarray) -> float:
    m = np.max(a)
    if np.isinf(m):
        return float(m)
    return float(m + np.log(np.sum(np.exp(a - m))))


def normalise(logw: np.ndarray) -> tuple[float, np.ndarray]:
    lam = log_sum_exp(logw)
    return lam, logw - lam


def prior_logw(p: Problem, x: np.ndarray) -> np.ndarray:
    """log sigma_0(x_i) for x_0 ~ N(mu0, s0^2 I) ("Algorithm for Kolmogorov Equation", step 4)."""
    d = x - p.prior_mean
    return -0.5 * np.sum(d * d, axis=1) / p.prior_var - 0.5 * p.r * np.log(2 * np.pi * p.prior_var)


def kernel_lse(p: Problem, prep: Prepared, logw: np.ndarray, t0: int = 0, t1: int | None = None,
               n_threads: int = 0, half: np.ndarray | None = None) -> np.ndarray:
    """L_j(i) for targets t0 <= i < t1 and every scale j: [(t1 - t0)][N]."""
    t1 = p.n if t1 is None else t1
    lwq = p.log_wq if half is None else log_wq(half, p.n)
    L = _lib.lib()
    x = np.ascontiguousarray(prep.x, dtype=np.float64)
    f = np.ascontiguousarray(prep.f, dtype=np.float64)
    dv = np.ascontiguousarray(prep.divf, dtype=np.float64)
    lw = np.ascontiguousarray(logw, dtype=np.float64)
    mk = np.ascontiguousarray(prep.mask, dtype=np.uint8)
    tau = np.ascontiguousarray(p.taus, dtype=np.float64)
    out = np.empty((t1 - t0, p.n_scales), dtype=np.float64)
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    mi = None if prep.minv is None else np.ascontiguousarray(prep.minv, dtype=np.float64)
    hl = None if prep.hld is None else np.ascontiguousarray(prep.hld, dtype=np.float64)
    L.yyo_kernel_lse(p.n, p.r, ptr(x), ptr(f), ptr(dv), ptr(lw), ptr(mk), p.n_scales,
                     ptr(tau), lwq, t0, t1, ptr(out), n_threads,
                     None if mi is None else ptr(mi), None if hl is None else ptr(hl))
    return out


def combine(p: Problem, Lj: np.ndarray, logw_t: np.ndarray, mask_t: np.ndarray) -> tuple[np.ndarray, int]:
    """Signed log-sum-exp of sum_j c_j e^{L_j} + c_{N+1} e^{ell}; returns (ell_pred, clamps)."""
    c = p.coef
    n_t = Lj.shape[0]
    out = np.empty(n_t)
    clamps = 0
    for i in range(n_t):
        if mask_t[i]:
            out[i] = -np.inf
            continue
        terms, signs = [], []
        for j in range(p.n_scales + 1):
            if c[j] == 0.0:
                continue
            val = Lj[i, j] if j < p.n_scales else logw_t[i]
            if np.isinf(val) and val < 0:
                continue
            terms.append(np.log(abs(c[j])) + val)
            signs.append(1.0 if c[j] > 0 else -1.0)
        if not terms:
            out[i] = -np.inf
            continue
        m = max(terms)
        s = sum(sg * np.exp(t - m) for sg, t in zip(signs, terms))
        if s > 0.0:
            out[i] = m + np.log(s)
        else:
            out[i] = -np.inf
            clamps += 1
    return out, clamps


def predict(p: Problem, prep: Prepared, logw: np.ndarray, t0: int = 0, t1: int | None = None,
            n_threads: int = 0, half: np.ndarray | None = None) -> tuple[np.ndarray, int]:
    t1 = p.n if t1 is None else t1
    Lj = kernel_lse(p, prep, logw, t0, t1, n_threads, half)
    return combine(p, Lj, logw[t0:t1], prep.mask[t0:t1])


def log_likelihood(p: Problem, x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """h(x_i).dy - dt/2 |h(x_i)|^2, the Ito-corrected log update factor; with noise
    coefficients h^T b^-1 dy - dt/2 h^T b^-1 h, b = V V^T (table of the section on noise
    coefficients, online update row)."""
    h = mdl.sensor(p.model, x)
    if p.noise is None:
        return h @ dy - 0.5 * p.dt * np.sum(h * h, axis=1)
    ib = 1.0 / mdl.obs_noise(p.noise, x) ** 2
    return np.sum(ib * (h * dy[None, :] - 0.5 * p.dt * h * h), axis=1)


def estimate(x: np.ndarray, logw_hat: np.ndarray) -> tuple[np.ndarray, np.ndarray, float]:
    w = np.exp(logw_hat)
    mean = w @ x
    d = x - mean[None, :]
    var = w @ (d * d)
    ess = 1.0 / float(np.sum(w * w))
    return mean, var, ess


def restart_due(p: Problem, ess: float, k: int) -> bool:
    by_ess = p.ess_frac > 0.0 and ess < p.ess_frac * p.n
    by_interval = p.restart_interval >= 2 and k % p.restart_interval == 0
    return bool(by_ess or by_interval)


def restart_logw(p: Problem, x: np.ndarray, centre: np.ndarray, var: np.ndarray,
                 half: np.ndarray | None = None) -> np.ndarray:
    """Fresh normalised log-weights after a restart: N(centre, diag(max(var, (R/4)^2)))."""
    if p.restart_init == "uniform":
        return np.full(p.n, -np.log(p.n))
    R = p.R if half is None else half
    v = np.maximum(var, (R / 4.0) ** 2)
    d = x - centre[None, :]
    lw = -0.5 * np.sum(d * d / v[None, :], axis=1) - 0.5 * np.sum(np.log(2 * np.pi * v))
    return normalise(lw)[1]


@dataclass
class State:
    u: np.ndarray          # [n][r] float32 reference nodes (box coordinates)
    centre: np.ndarray     # [r] float64
    logw: np.ndarray       # [n] float64, normalised
    lognorm: float = 0.0   # Z
    k: int = 0
    half: np.ndarray | None = None   # [r] current half-widths (None: the problem's R)
    y: np.ndarray | None = None      # [n][r] Sobol integers of the nodes (learned rule)


@dataclass
class StepRecord:
    mean: np.ndarray
    var: np.ndarray
    ess: float
    lam: float
    lognorm: float
    restarted: bool
    clamps: int
    learned: bool = False
    logw_pred: np.ndarray = field(repr=False, default=None)
    logw_hat: np.ndarray = field(repr=False, default=None)


def init_state(p: Problem, u: np.ndarray, centre: np.ndarray) -> State:
    prep = prepare(p, u, centre)
    lw = prior_logw(p, prep.x)
    lw[prep.mask] = -np.inf
    _, lw_hat = normalise(lw)
    return State(u=u, centre=centre.astype(np.float64).copy(), logw=lw_hat, lognorm=0.0, k=0)


def step(p: Problem, st: State, dy: np.ndarray, n_threads: int = 0,
         keep_logw: bool = False) -> tuple[StepRecord, State]:
    half = p.R if st.half is None else st.half
    prep = prepare(p, st.u, st.centre, half)
    lw_pred, clamps = predict(p, prep, st.logw, n_threads=n_threads, half=half)
    lw_upd = lw_pred + log_likelihood(p, prep.x, dy)
    lam, lw_hat = normalise(lw_upd)
    if np.isinf(lam):
        raise FloatingPointError("all weights vanished")
    mean, var, ess = estimate(prep.x, lw_hat)
    k = st.k + 1
    Z = st.lognorm + lam
    rec = StepRecord(mean=mean, var=var, ess=ess, lam=lam, lognorm=Z, restarted=False,
                     clamps=clamps, logw_pred=lw_pred if keep_logw else None,
                     logw_hat=lw_hat if keep_logw else None)
    new = State(u=st.u, centre=st.centre, logw=lw_hat, lognorm=Z, k=k, half=st.half, y=st.y)
    if restart_due(p, ess, k):
        rec.restarted = True
        centre, new_half, u = mean.copy(), half, st.u
        if p.restart_rule == "learned":
            from . import mlp, sobol
            centre, new_half, ok = mlp.proposal(p.mlp_params, mean, var, dy, p.dt, p.R, st.centre)
            rec.learned = ok
            if ok:
                u = sobol.to_box(st.y, new_half)
        prep2 = prepare(p, u, centre, new_half)
        lw0 = restart_logw(p, prep2.x, centre, var, new_half)
        lw0[prep2.mask] = -np.inf
        new = State(u=u, centre=centre, logw=lw0, lognorm=Z, k=k, half=np.array(new_half, dtype=np.float64),
                    y=st.y)
    return rec, new


def run(p: Problem, st: State, dys: np.ndarray, n_threads: int = 0) -> list[StepRecord]:
    recs = []
    for k in range(dys.shape[0]):
        rec, st = step(p, st, dys[k], n_threads=n_threads)
        recs.append(rec)
    return recs
