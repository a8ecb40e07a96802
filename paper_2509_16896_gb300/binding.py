"""Thin Python binding of libyy (include/yy.h): argument marshalling only.

Every step of the filter runs in the library's CUDA kernels.  PyTorch provides the
device workspace, the device buffers of the observation increments and the CUDA stream.
There is no fallback: if the library cannot be loaded the binding raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "lib", "libyy.so")
_lock = threading.Lock()
_lib = None

YY_OK = 0
STATUS_NAMES = {0: "YY_OK", 1: "YY_ERR_ARG", 2: "YY_ERR_CUDA", 3: "YY_ERR_WORKSPACE",
                4: "YY_ERR_NONFINITE", 5: "YY_ERR_DEGENERATE", 6: "YY_ERR_TIMEOUT",
                7: "YY_ERR_STATE", 8: "YY_ERR_UNSUPPORTED"}
MODELS = {"cubic": 0, "linear": 1, "paper_e1": 2}
PRECISIONS = {"f64": 0, "f32": 1, "bf16": 2, "f32s": 3}
RESTART_INIT = {"gauss": 0, "uniform": 1}
RESTART_RULE = {"plain": 0, "learned": 1}
SCREEN_TYPE = {"bf16": 0, "fp8": 1}
NODES = {"sobol": 0, "halton": 1, "faure": 2}
RESTART_AUTO, RESTART_FORCE, RESTART_NEVER = 0, 1, 2
SOBOL_POLY_WORDS = 16
SOBOL_SCRAMBLE_WORDS = 33

# every symbol include/yy.h declares
EXPORTS = ("yy_workspace_bytes", "yy_create", "yy_destroy", "yy_init_nodes", "yy_sobol_bits",
           "yy_predict", "yy_update", "yy_estimate", "yy_restart", "yy_get_nodes",
           "yy_get_log_weights", "yy_set_state", "yy_get_state", "yy_get_clamps",
           "yy_launch_count", "yy_status_str", "yy_weighted_moments_static",
           "yy_run_steps", "yy_graph_capture", "yy_graph_launch", "yy_graph_kernel_count",
           "yy_batch_workspace_bytes", "yy_batch_create", "yy_batch_destroy", "yy_batch_filter",
           "yy_batch_run_steps", "yy_batch_predict", "yy_batch_graph_capture", "yy_batch_graph_launch",
           "yy_batch_set_schedule", "yy_batch_get_schedule", "yy_batch_autotune",
           "yy_batch_launch_count", "yy_batch_graph_kernel_count", "yy_get_counters",
           "yy_batch_get_routing", "yy_get_box", "yy_set_restart_mlp", "yy_mlp_param_count",
           "yy_mlp_workspace_bytes", "yy_mlp_create", "yy_mlp_destroy", "yy_mlp_set_params",
           "yy_mlp_get_params", "yy_mlp_forward", "yy_mlp_loss_grad", "yy_mlp_train",
           "yy_mlp_set_input_norm", "yy_get_screen", "yy_batch_set_routing",
           "yy_set_wait_limit", "yy_set_shard", "yy_shard_rows", "yy_update_shard", "yy_merge_shards",
           "yy_merge_records_host", "yy_init_nodes_lds", "yy_tune_materialise", "yy_set_cta_pair",
           "yy_set_route", "yy_tune_route")


class YYError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} failed: {STATUS_NAMES.get(code, code)}")
        self.code = code


class YYConfig(ctypes.Structure):
    _fields_ = [("r", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_int64),
                ("dt", ctypes.c_double), ("R", ctypes.c_double), ("n_scales", ctypes.c_int32),
                ("model", ctypes.c_int32), ("model_a", ctypes.c_double),
                ("precision", ctypes.c_int32), ("restart_interval", ctypes.c_int32),
                ("ess_frac", ctypes.c_double), ("restart_init", ctypes.c_int32),
                ("prior_mean", ctypes.c_double), ("prior_var", ctypes.c_double),
                ("restart_rule", ctypes.c_int32), ("screen_prefix", ctypes.c_int32),
                ("screen_type", ctypes.c_int32), ("noise", ctypes.c_int32), ("noise_u_zero", ctypes.c_int32),
                ("noise_u", ctypes.c_double), ("noise_u_kappa", ctypes.c_double),
                ("noise_v", ctypes.c_double), ("noise_v_kappa", ctypes.c_double),
                ("materialise", ctypes.c_int32)]


def _declare(L: ctypes.CDLL) -> None:
    P, I32, I64, D, S = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
    sig = {
        "yy_workspace_bytes": (S, [P]),
        "yy_create": (I32, [P, P, S, P, P]),
        "yy_destroy": (I32, [P]),
        "yy_init_nodes": (I32, [P, P, P, P, P]),
        "yy_sobol_bits": (I32, [P, P, I64, I64]),
        "yy_predict": (I32, [P]),
        "yy_update": (I32, [P, P]),
        "yy_estimate": (I32, [P, P, P, P, P]),
        "yy_restart": (I32, [P, I32, P]),
        "yy_get_nodes": (I32, [P, P, P]),
        "yy_get_log_weights": (I32, [P, P, P]),
        "yy_set_state": (I32, [P, P, P, D, I64]),
        "yy_get_state": (I32, [P, P, P, P]),
        "yy_get_screen": (I32, [P, P, P, P, P]),
        "yy_get_clamps": (I32, [P, P]),
        "yy_launch_count": (I64, [P]),
        "yy_status_str": (ctypes.c_char_p, [I32]),
        "yy_weighted_moments_static": (I32, [P, I64, I32, I64, P, P, P]),
        "yy_run_steps": (I32, [P, P, I64, P]),
        "yy_graph_capture": (I32, [P, P, I64, P]),
        "yy_graph_launch": (I32, [P]),
        "yy_graph_kernel_count": (I64, [P]),
        "yy_batch_workspace_bytes": (S, [P, I32]),
        "yy_batch_create": (I32, [P, I32, P, S, P, P]),
        "yy_batch_destroy": (I32, [P]),
        "yy_batch_filter": (I32, [P, I32, P]),
        "yy_batch_run_steps": (I32, [P, P, I64, P]),
        "yy_batch_predict": (I32, [P]),
        "yy_batch_graph_capture": (I32, [P, P, I64, P]),
        "yy_batch_graph_launch": (I32, [P]),
        "yy_batch_set_schedule": (I32, [P, I32, I32]),
        "yy_batch_get_schedule": (I32, [P, P, P]),
        "yy_batch_autotune": (I32, [P, ctypes.c_char_p, I32, P, P]),
        "yy_batch_launch_count": (I64, [P]),
        "yy_batch_graph_kernel_count": (I64, [P]),
        "yy_get_counters": (I32, [P, P, P]),
        "yy_batch_get_routing": (I32, [P, P]),
        "yy_batch_set_routing": (I32, [P, P]),
        "yy_set_wait_limit": (I32, [P, D]),
        "yy_set_shard": (I32, [P, I32, I32]),
        "yy_shard_rows": (I32, [P, P, P]),
        "yy_update_shard": (I32, [P, P, P, P]),
        "yy_merge_shards": (I32, [P, P, P, I32]),
        "yy_merge_records_host": (I32, [P, I32, I32, P]),
        "yy_init_nodes_lds": (I32, [P, I32, P, P]),
        "yy_tune_materialise": (I32, [P, I32, I32, P, P]),
        "yy_set_route": (I32, [P, I32]),
        "yy_tune_route": (I32, [P, I32, P, P]),
        "yy_set_cta_pair": (I32, [P, I32, P]),
        "yy_get_box": (I32, [P, P, P]),
        "yy_set_restart_mlp": (I32, [P, P]),
        "yy_mlp_param_count": (I64, [I32, I32]),
        "yy_mlp_workspace_bytes": (S, [I32, I32, I32]),
        "yy_mlp_create": (I32, [I32, I32, I32, P, S, P, P]),
        "yy_mlp_destroy": (I32, [P]),
        "yy_mlp_set_params": (I32, [P, P]),
        "yy_mlp_get_params": (I32, [P, P]),
        "yy_mlp_forward": (I32, [P, P, I32, P]),
        "yy_mlp_loss_grad": (I32, [P, P, P, I32, D, P, P]),
        "yy_mlp_train": (I32, [P, P, P, I64, D, I32, I32, ctypes.c_float, ctypes.c_uint64, P]),
        "yy_mlp_set_input_norm": (I32, [P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads lib/libyy.so, compiling it first if it is missing; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                if not build_if_missing:
                    raise FileNotFoundError(f"{_LIB_PATH} is missing; run build()")
                from . import build as _b
                _b.build()
            L = ctypes.CDLL(_LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(fn: str, code: int) -> None:
    if code != YY_OK:
        raise YYError(fn, code)


def make_config(model: str, r: int, n: int, dt: float, R: float, n_scales: int,
                precision: str, restart_interval: int = 0, ess_frac: float = 0.0,
                model_a: float = -0.5, restart_init: str = "gauss", prior_mean: float = 0.0,
                prior_var: float = 1.0, restart_rule: str = "plain", screen_prefix: int = 0,
                screen_type: str = "bf16", noise: dict | None = None, materialise: int = 0) -> YYConfig:
    """noise: None (unit noise) or diagonal noise coefficients {u, u_kappa, u_zero, v, v_kappa}
    (include/yy.h, yy_noise)."""
    nz = noise or {}
    return YYConfig(r=r, m=r, n=n, dt=dt, R=R, n_scales=n_scales, model=MODELS[model],
                    model_a=model_a, precision=PRECISIONS[precision],
                    restart_interval=restart_interval, ess_frac=ess_frac,
                    restart_init=RESTART_INIT[restart_init], prior_mean=prior_mean,
                    prior_var=prior_var, restart_rule=RESTART_RULE[restart_rule],
                    screen_prefix=screen_prefix, screen_type=SCREEN_TYPE[screen_type],
                    noise=1 if noise else 0, noise_u_zero=int(nz.get("u_zero", 0)),
                    noise_u=float(nz.get("u", 1.0)), noise_u_kappa=float(nz.get("u_kappa", 0.0)),
                    noise_v=float(nz.get("v", 1.0)), noise_v_kappa=float(nz.get("v_kappa", 0.0)),
                    materialise=materialise)


def config_from_workload(w, precision: str | None = None, **over) -> YYConfig:
    kw = dict(model=w.model, r=w.r, n=w.n, dt=w.dt, R=w.R, n_scales=w.n_scales,
              precision=precision or w.precision, restart_interval=w.restart_interval,
              ess_frac=w.ess_frac, model_a=w.model_a, prior_mean=w.prior_mean,
              prior_var=w.prior_var, restart_rule=w.restart_rule,
              screen_type=getattr(w, "screen_type", "bf16"))
    kw.update(over)
    return make_config(**kw)


class Filter:
    """One filter handle on one CUDA device (torch allocates its workspace)."""

    def __init__(self, cfg: YYConfig, device: str = "cuda:0", stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.cfg = cfg
        self.device = torch.device(device)
        nbytes = self.lib.yy_workspace_bytes(ctypes.byref(cfg))
        if nbytes == 0:
            raise YYError("yy_workspace_bytes", 1)
        self.ws_bytes = int(nbytes)
        self.ws = torch.empty(self.ws_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        self.ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        # the workspace is used on self.stream: the caching allocator must not hand it out
        # again before that stream's work has finished
        self.ws.record_stream(self.stream)
        h = ctypes.c_void_p()
        _check("yy_create", self.lib.yy_create(ctypes.byref(cfg), ctypes.c_void_p(self.ws_ptr),
                                               self.ws_bytes, ctypes.c_void_p(self.stream.cuda_stream),
                                               ctypes.byref(h)))
        self.h = h
        self.r, self.n = cfg.r, cfg.n
        self.fp64 = cfg.precision == PRECISIONS["f64"]

    def close(self) -> None:
        if getattr(self, "h", None):
            self.stream.synchronize()   # no kernel of this handle may outlive its workspace
            self.lib.yy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- calls -------------------------------------------------------------------
    def init_nodes(self, poly: np.ndarray, scramble: np.ndarray | None, center: np.ndarray,
                   halfwidth: np.ndarray | None = None) -> None:
        poly = np.ascontiguousarray(poly, dtype=np.uint32)
        scr = None if scramble is None else np.ascontiguousarray(scramble, dtype=np.uint32)
        cen = np.ascontiguousarray(center, dtype=np.float64)
        hw = None if halfwidth is None else np.ascontiguousarray(halfwidth, dtype=np.float64)
        assert poly.shape == (self.r, SOBOL_POLY_WORDS) and cen.shape == (self.r,)
        _check("yy_init_nodes", self.lib.yy_init_nodes(
            self.h, _ptr(poly), None if scr is None else _ptr(scr), _ptr(cen),
            None if hw is None else _ptr(hw)))

    def init_nodes_lds(self, kind: str, center: np.ndarray, halfwidth: np.ndarray | None = None) -> None:
        """Halton ("halton") or Faure ("faure") nodes instead of Sobol nodes."""
        cen = np.ascontiguousarray(center, dtype=np.float64)
        hw = None if halfwidth is None else np.ascontiguousarray(halfwidth, dtype=np.float64)
        assert cen.shape == (self.r,)
        _check("yy_init_nodes_lds", self.lib.yy_init_nodes_lds(self.h, NODES[kind], _ptr(cen),
                                                               None if hw is None else _ptr(hw)))

    def sobol_bits(self, first: int, count: int):
        out = self.torch.empty((count, self.r), dtype=self.torch.int32, device=self.device)
        _order_after_torch(self.stream, self.device)
        _check("yy_sobol_bits", self.lib.yy_sobol_bits(self.h, ctypes.c_void_p(out.data_ptr()),
                                                       first, count))
        self.stream.synchronize()
        return out

    def predict(self) -> None:
        _check("yy_predict", self.lib.yy_predict(self.h))

    def update(self, dy_dev) -> None:
        """dy_dev: torch float64 tensor [r] on the device."""
        assert dy_dev.dtype == self.torch.float64 and dy_dev.is_cuda and dy_dev.numel() == self.r
        _order_after_torch(self.stream, self.device)
        _check("yy_update", self.lib.yy_update(self.h, ctypes.c_void_p(dy_dev.data_ptr())))

    def estimate(self):
        mean = np.empty(self.r)
        var = np.empty(self.r)
        ess = ctypes.c_double()
        z = ctypes.c_double()
        _check("yy_estimate", self.lib.yy_estimate(self.h, _ptr(mean), _ptr(var), ctypes.byref(ess),
                                                   ctypes.byref(z)))
        return mean, var, ess.value, z.value

    def restart(self, mode: int = RESTART_AUTO, report: bool = False):
        did = ctypes.c_int32(0)
        _check("yy_restart", self.lib.yy_restart(self.h, mode, ctypes.byref(did) if report else None))
        return bool(did.value) if report else None

    def get_nodes(self):
        u = np.empty((self.n, self.r), dtype=np.float32)
        mask = np.empty(self.n, dtype=np.uint8)
        _check("yy_get_nodes", self.lib.yy_get_nodes(self.h, _ptr(u), _ptr(mask)))
        return u, mask.astype(bool)

    def get_log_weights(self):
        out = np.empty(self.n, dtype=np.float64 if self.fp64 else np.float32)
        off = ctypes.c_double()
        _check("yy_get_log_weights", self.lib.yy_get_log_weights(self.h, _ptr(out), ctypes.byref(off)))
        return out, off.value

    def set_state(self, center: np.ndarray, logw: np.ndarray, lognorm: float = 0.0, step: int = 0):
        cen = np.ascontiguousarray(center, dtype=np.float64)
        lw = np.ascontiguousarray(logw, dtype=np.float64 if self.fp64 else np.float32)
        _check("yy_set_state", self.lib.yy_set_state(self.h, _ptr(cen), _ptr(lw), lognorm, step))

    def get_box(self):
        cen = np.empty(self.r)
        half = np.empty(self.r)
        _check("yy_get_box", self.lib.yy_get_box(self.h, _ptr(cen), _ptr(half)))
        return cen, half

    def set_restart_mlp(self, net) -> None:
        _check("yy_set_restart_mlp", self.lib.yy_set_restart_mlp(self.h, None if net is None else net.h))
        self._mlp = net   # keep the network alive while attached

    def get_state(self):
        cen = np.empty(self.r)
        z = ctypes.c_double()
        k = ctypes.c_int64()
        _check("yy_get_state", self.lib.yy_get_state(self.h, _ptr(cen), ctypes.byref(z), ctypes.byref(k)))
        return cen, z.value, k.value

    def clamps(self) -> int:
        c = ctypes.c_int64()
        _check("yy_get_clamps", self.lib.yy_get_clamps(self.h, ctypes.byref(c)))
        return c.value

    def launches(self) -> int:
        return int(self.lib.yy_launch_count(self.h))

    def tune_materialise(self, predicts_per_build: int, reps: int = 3):
        """Times recompute, build and apply; returns (choice 0/1, (ms recompute, build, apply))."""
        ms = np.zeros(3)
        ch = ctypes.c_int32()
        _check("yy_tune_materialise", self.lib.yy_tune_materialise(self.h, predicts_per_build, reps, _ptr(ms),
                                                                   ctypes.byref(ch)))
        return ch.value, tuple(ms)

    def set_route(self, plain: bool) -> None:
        """BF16 filters: predictions on the plain float32 form (True) or the screen (False)."""
        _check("yy_set_route", self.lib.yy_set_route(self.h, 1 if plain else 0))

    def tune_route(self, reps: int = 3):
        """Times the screened and the plain prediction and keeps the faster; returns
        (route 0 screen / 1 plain, (ms screened, ms plain))."""
        ms = np.zeros(2)
        rt = ctypes.c_int32()
        _check("yy_tune_route", self.lib.yy_tune_route(self.h, reps, _ptr(ms), ctypes.byref(rt)))
        return rt.value, tuple(ms)

    def set_wait_limit(self, seconds: float) -> None:
        _check("yy_set_wait_limit", self.lib.yy_set_wait_limit(self.h, float(seconds)))

    def set_cta_pair(self, on: bool) -> int:
        """Allow (True) or forbid the tensor-core prediction on 2-CTA clusters; returns
        the number of CTA pairs of the current schedule (0: single CTAs)."""
        pairs = ctypes.c_int32(0)
        _check("yy_set_cta_pair", self.lib.yy_set_cta_pair(self.h, 1 if on else 0, ctypes.byref(pairs)))
        return pairs.value

    # ---- one filter across devices (target rows split) ------------------------------
    def set_shard(self, rank: int, count: int) -> None:
        _check("yy_set_shard", self.lib.yy_set_shard(self.h, rank, count))

    def shard_rows(self):
        """(first row of this shard's chunk, chunk length)."""
        r0, ch = ctypes.c_int64(), ctypes.c_int64()
        _check("yy_shard_rows", self.lib.yy_shard_rows(self.h, ctypes.byref(r0), ctypes.byref(ch)))
        return r0.value, ch.value

    def update_shard(self, dy_dev, rows_out, record_out) -> None:
        """rows_out: device tensor [chunk] (float32, float64 for FP64); record_out: float64 [2r + 4]."""
        t = self.torch
        assert dy_dev.dtype == t.float64 and dy_dev.numel() == self.r
        assert rows_out.dtype == (t.float64 if self.fp64 else t.float32) and rows_out.is_contiguous()
        assert record_out.dtype == t.float64 and record_out.numel() == 2 * self.r + 4 and record_out.is_contiguous()
        assert rows_out.numel() == self.shard_rows()[1]
        _order_after_torch(self.stream, self.device)
        _check("yy_update_shard", self.lib.yy_update_shard(self.h, ctypes.c_void_p(dy_dev.data_ptr()),
                                                           ctypes.c_void_p(rows_out.data_ptr()),
                                                           ctypes.c_void_p(record_out.data_ptr())))
        _order_torch_after(self.stream, self.device)

    def merge_shards(self, rows_all, records, count: int) -> None:
        """rows_all: device [n_pad] (every shard's chunk in shard order); records: float64
        [count][2r + 4] in shard order."""
        assert rows_all.is_contiguous() and records.is_contiguous() and records.dtype == self.torch.float64
        _order_after_torch(self.stream, self.device)
        _check("yy_merge_shards", self.lib.yy_merge_shards(self.h, ctypes.c_void_p(rows_all.data_ptr()),
                                                           ctypes.c_void_p(records.data_ptr()), count))

    def screen(self):
        """(first-pass chunks of the last prediction, of the next one, tiles, tiles
        rescreened) of the last BF16 prediction."""
        last, nxt, t, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check("yy_get_screen", self.lib.yy_get_screen(self.h, ctypes.byref(last), ctypes.byref(nxt),
                                                       ctypes.byref(t), ctypes.byref(e)))
        return last.value, nxt.value, t.value, e.value

    def counters(self):
        """(clamps, pairs evaluated exactly) of the last prediction."""
        c, p = ctypes.c_int64(), ctypes.c_int64()
        _check("yy_get_counters", self.lib.yy_get_counters(self.h, ctypes.byref(c), ctypes.byref(p)))
        return c.value, p.value

    def run_steps(self, dy_all_dev, hist_dev=None) -> None:
        """dy_all_dev: float64 [K][r] device tensor; hist_dev: float64 [K][2r + 4] or None."""
        K = dy_all_dev.shape[0]
        _order_after_torch(self.stream, self.device)
        _check("yy_run_steps", self.lib.yy_run_steps(
            self.h, ctypes.c_void_p(dy_all_dev.data_ptr()), K,
            None if hist_dev is None else ctypes.c_void_p(hist_dev.data_ptr())))
        _order_torch_after(self.stream, self.device)

    def graph_capture(self, dy_all_dev, hist_dev=None) -> None:
        K = dy_all_dev.shape[0]
        _check("yy_graph_capture", self.lib.yy_graph_capture(
            self.h, ctypes.c_void_p(dy_all_dev.data_ptr()), K,
            None if hist_dev is None else ctypes.c_void_p(hist_dev.data_ptr())))

    def graph_launch(self) -> None:
        _order_after_torch(self.stream, self.device)
        _check("yy_graph_launch", self.lib.yy_graph_launch(self.h))
        _order_torch_after(self.stream, self.device)

    def graph_kernels(self) -> int:
        return int(self.lib.yy_graph_kernel_count(self.h))


class MLP:
    """Restart-proposal network (include/yy.h, network section)."""

    def __init__(self, r: int, hidden: int = 256, max_batch: int = 256, device: str = "cuda:0", stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.r, self.hidden, self.max_batch = r, hidden, max_batch
        self.device = torch.device(device)
        self.n_params = int(self.lib.yy_mlp_param_count(r, hidden))
        nbytes = int(self.lib.yy_mlp_workspace_bytes(r, hidden, max_batch))
        if nbytes == 0:
            raise YYError("yy_mlp_workspace_bytes", 1)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ws.record_stream(self.stream)
        h = ctypes.c_void_p()
        _check("yy_mlp_create", self.lib.yy_mlp_create(r, hidden, max_batch, ctypes.c_void_p(ptr), nbytes,
                                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.stream.synchronize()
            self.lib.yy_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat: np.ndarray) -> None:
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.n_params
        _check("yy_mlp_set_params", self.lib.yy_mlp_set_params(self.h, _ptr(flat)))

    def set_input_norm(self, mean: np.ndarray, std: np.ndarray) -> None:
        mean = np.ascontiguousarray(mean, dtype=np.float32)
        std = np.ascontiguousarray(std, dtype=np.float32)
        _check("yy_mlp_set_input_norm", self.lib.yy_mlp_set_input_norm(self.h, _ptr(mean), _ptr(std)))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        _check("yy_mlp_get_params", self.lib.yy_mlp_get_params(self.h, _ptr(out)))
        return out

    def forward(self, x_dev):
        B = x_dev.shape[0]
        out = self.torch.empty((B, 2 * self.r), dtype=self.torch.float32, device=self.device)
        _order_after_torch(self.stream, self.device)
        _check("yy_mlp_forward", self.lib.yy_mlp_forward(self.h, ctypes.c_void_p(x_dev.data_ptr()), B,
                                                         ctypes.c_void_p(out.data_ptr())))
        _order_torch_after(self.stream, self.device)
        return out

    def loss_grad(self, x_dev, t_dev, R: float):
        loss = ctypes.c_float()
        g = np.empty(self.n_params, dtype=np.float32)
        _order_after_torch(self.stream, self.device)
        _check("yy_mlp_loss_grad", self.lib.yy_mlp_loss_grad(
            self.h, ctypes.c_void_p(x_dev.data_ptr()), ctypes.c_void_p(t_dev.data_ptr()), x_dev.shape[0], R,
            ctypes.byref(loss), _ptr(g)))
        return loss.value, g

    def train(self, x_dev, t_dev, R: float, epochs: int, batch: int, lr: float, seed: int = 0) -> float:
        loss = ctypes.c_float()
        _order_after_torch(self.stream, self.device)
        _check("yy_mlp_train", self.lib.yy_mlp_train(
            self.h, ctypes.c_void_p(x_dev.data_ptr()), ctypes.c_void_p(t_dev.data_ptr()), x_dev.shape[0], R,
            epochs, batch, ctypes.c_float(lr), ctypes.c_uint64(seed), ctypes.byref(loss)))
        return loss.value


def _order_after_torch(stream, device) -> None:
    """Makes `stream` wait for the work already queued on torch's current and default
    streams (buffers filled there, e.g. torch.zeros, must be ready before the library
    reads or writes them on its own stream)."""
    import torch
    for other in (torch.cuda.current_stream(device), torch.cuda.default_stream(device)):
        if other.cuda_stream != stream.cuda_stream:
            stream.wait_stream(other)


def _order_torch_after(stream, device) -> None:
    """Makes torch's current and default streams wait for the library's stream, so that
    device outputs (histories, network outputs) are ready for torch work queued next."""
    import torch
    for other in (torch.cuda.current_stream(device), torch.cuda.default_stream(device)):
        if other.cuda_stream != stream.cuda_stream:
            other.wait_stream(stream)


def merge_records_host(records: np.ndarray, r: int) -> np.ndarray:
    """The shard merge on the host: records float64 [count][2r + 4] -> [Lambda, W, Q, ESS,
    mean of u [r], variance [r]] (yy_merge_records_host; no device needed)."""
    L = load()
    rec = np.ascontiguousarray(records, dtype=np.float64)
    out = np.empty(2 * r + 4)
    _check("yy_merge_records_host", L.yy_merge_records_host(_ptr(rec), rec.shape[0], r, _ptr(out)))
    return out


def pack_mlp_params(p: dict) -> np.ndarray:
    """Packs {W1, b1, W2, b2, W3, b3} in the layout of yy_mlp_set_params."""
    return np.concatenate([p[k].ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)


def unpack_mlp_params(flat: np.ndarray, r: int, hidden: int) -> dict:
    shapes = [("W1", (hidden, 3 * r)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
              ("W3", (2 * r, hidden)), ("b3", (2 * r,))]
    out, o = {}, 0
    for k, shp in shapes:
        n = int(np.prod(shp))
        out[k] = np.asarray(flat[o:o + n], dtype=np.float64).reshape(shp)
        o += n
    return out


class _BorrowedFilter(Filter):
    """A filter handle owned by a Batch (no workspace of its own)."""

    def __init__(self, batch, b, cfg):
        self.torch = batch.torch
        self.lib = batch.lib
        self.cfg = cfg
        self.device = batch.device
        self.stream = batch.stream
        h = ctypes.c_void_p()
        _check("yy_batch_filter", self.lib.yy_batch_filter(batch.h, b, ctypes.byref(h)))
        self.h = h
        self.r, self.n = cfg.r, cfg.n
        self.fp64 = False

    def close(self) -> None:   # owned by the batch
        self.h = None


class Batch:
    """B independent filters advanced together (include/yy.h, batch section)."""

    def __init__(self, cfgs, device: str = "cuda:0", stream=None):
        import torch
        self.torch = torch
        self.lib = load()
        self.device = torch.device(device)
        self.cfgs = list(cfgs)
        self.B = len(self.cfgs)
        arr = (YYConfig * self.B)(*self.cfgs)
        self._arr = arr
        nbytes = self.lib.yy_batch_workspace_bytes(arr, self.B)
        if nbytes == 0:
            raise YYError("yy_batch_workspace_bytes", 1)
        self.ws = torch.empty(int(nbytes) + 256, dtype=torch.uint8, device=self.device)
        ptr = (self.ws.data_ptr() + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.ws.record_stream(self.stream)
        h = ctypes.c_void_p()
        _check("yy_batch_create", self.lib.yy_batch_create(arr, self.B, ctypes.c_void_p(ptr), int(nbytes),
                                                           ctypes.c_void_p(self.stream.cuda_stream),
                                                           ctypes.byref(h)))
        self.h = h
        self.filters = [_BorrowedFilter(self, b, self.cfgs[b]) for b in range(self.B)]
        self.dy_off = np.cumsum([0] + [c.m for c in self.cfgs])
        self.hist_off = np.cumsum([0] + [2 * c.r + 4 for c in self.cfgs])

    @property
    def M(self) -> int:
        return int(self.dy_off[-1])

    @property
    def H(self) -> int:
        return int(self.hist_off[-1])

    def close(self) -> None:
        if getattr(self, "h", None):
            self.stream.synchronize()   # no kernel of the batch may outlive its workspace
            self.lib.yy_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run_steps(self, dy_all_dev, hist_dev=None) -> None:
        K = dy_all_dev.shape[0]
        _order_after_torch(self.stream, self.device)
        _check("yy_batch_run_steps", self.lib.yy_batch_run_steps(
            self.h, ctypes.c_void_p(dy_all_dev.data_ptr()), K,
            None if hist_dev is None else ctypes.c_void_p(hist_dev.data_ptr())))
        _order_torch_after(self.stream, self.device)

    def predict(self) -> None:
        _check("yy_batch_predict", self.lib.yy_batch_predict(self.h))

    def graph_capture(self, dy_all_dev, hist_dev=None) -> None:
        K = dy_all_dev.shape[0]
        _check("yy_batch_graph_capture", self.lib.yy_batch_graph_capture(
            self.h, ctypes.c_void_p(dy_all_dev.data_ptr()), K,
            None if hist_dev is None else ctypes.c_void_p(hist_dev.data_ptr())))

    def graph_launch(self) -> None:
        _order_after_torch(self.stream, self.device)
        _check("yy_batch_graph_launch", self.lib.yy_batch_graph_launch(self.h))
        _order_torch_after(self.stream, self.device)

    def set_schedule(self, bn: int, grid: int) -> None:
        _check("yy_batch_set_schedule", self.lib.yy_batch_set_schedule(self.h, bn, grid))

    def schedule(self):
        bn, grid = ctypes.c_int32(), ctypes.c_int32()
        _check("yy_batch_get_schedule", self.lib.yy_batch_get_schedule(self.h, ctypes.byref(bn), ctypes.byref(grid)))
        return bn.value, grid.value

    def autotune(self, cache_path: str | None = None, reps: int = 3):
        bn, grid = ctypes.c_int32(), ctypes.c_int32()
        _check("yy_batch_autotune", self.lib.yy_batch_autotune(
            self.h, None if cache_path is None else cache_path.encode(), reps, ctypes.byref(bn), ctypes.byref(grid)))
        return bn.value, grid.value

    def routing(self):
        out = np.zeros(self.B, dtype=np.int32)
        _check("yy_batch_get_routing", self.lib.yy_batch_get_routing(self.h, _ptr(out)))
        return out

    def set_routing(self, path) -> None:
        """Per-filter prediction path: 0 = tensor-core screen, 1 = FP32 form."""
        arr = np.ascontiguousarray(path, dtype=np.int32)
        assert arr.shape == (self.B,)
        _check("yy_batch_set_routing", self.lib.yy_batch_set_routing(self.h, _ptr(arr)))

    def launches(self) -> int:
        return int(self.lib.yy_batch_launch_count(self.h))

    def graph_kernels(self) -> int:
        return int(self.lib.yy_batch_graph_kernel_count(self.h))


def weighted_moments_static(u_dev, logw_dev, out_dev, stream=None) -> None:
    """Calls yy_weighted_moments_static, which allocates no device memory: u_dev is a
    float32 [n][ld] device tensor (row stride ld >= r = u_dev.shape[1] when 2-D), logw_dev
    float32 [n], out_dev float64 [2r + 3] (mean, var, ESS, LSE, weight sum).  All three
    tensors must be on one device; the call runs with that device current."""
    import torch
    L = load()
    n, r = u_dev.shape
    ld = u_dev.stride(0)
    assert u_dev.dtype == torch.float32 and u_dev.stride(1) == 1
    assert logw_dev.dtype == torch.float32 and logw_dev.numel() == n and logw_dev.is_contiguous()
    assert out_dev.dtype == torch.float64 and out_dev.numel() >= 2 * r + 3 and out_dev.is_contiguous()
    assert u_dev.is_cuda and logw_dev.device == u_dev.device and out_dev.device == u_dev.device
    with torch.cuda.device(u_dev.device):
        s = stream if stream is not None else torch.cuda.current_stream(u_dev.device)
        _check("yy_weighted_moments_static", L.yy_weighted_moments_static(
            ctypes.c_void_p(u_dev.data_ptr()), n, r, ld, ctypes.c_void_p(logw_dev.data_ptr()),
            ctypes.c_void_p(out_dev.data_ptr()), ctypes.c_void_p(s.cuda_stream)))
