"""Restart-proposal network on the GPU: forward and gradients against the FP64 oracle,
training, the learned restart inside the filter against the oracle's learned restart, and
what the trained network gains over the plain rule."""
import numpy as np
import pytest

from synth import simulate

from ._helpers import oracle_problem, rel_err, sobol_inputs

pytestmark = pytest.mark.gpu


def _rand_params(r, H, seed):
    from oracle import mlp
    p = mlp.init_params(r, H, seed)
    rng = np.random.default_rng(seed)
    for k in mlp.TRAINED:
        p[k] = p[k] + 0.1 * rng.normal(size=p[k].shape)
    p["mu"] = 0.2 * rng.normal(size=3 * r)
    p["s"] = 1.0 + 0.3 * rng.random(3 * r)
    return p


def _bf16(a):
    """Round float64 values to bfloat16 (round to nearest even), as the kernels' operands."""
    f = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounded = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_and_gradients_match_oracle(yy_lib):
    import torch
    from oracle import mlp
    from paper_2509_16896_gb300 import binding
    r, H, B, R = 5, 32, 64, 0.3
    p = _rand_params(r, H, 1)
    rng = np.random.default_rng(2)
    X = rng.normal(size=(B, 3 * r)).astype(np.float32)
    T = (0.2 * rng.normal(size=(B, r))).astype(np.float32)
    net = binding.MLP(r, H, max_batch=B)
    net.set_params(binding.pack_mlp_params(p))
    net.set_input_norm(p["mu"], p["s"])
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    o_gpu = net.forward(xd).cpu().numpy().astype(np.float64)
    o_ref, cache = mlp.forward(p, X.astype(np.float64))
    assert np.linalg.norm(o_gpu - o_ref) <= 1e-2 * np.linalg.norm(o_ref)
    loss, g = net.loss_grad(xd, td, R)
    L_ref, g_o = mlp.loss_and_grad_out(o_ref, T.astype(np.float64), R)
    g_ref = mlp.backward(p, cache, g_o)
    assert loss == pytest.approx(L_ref, rel=1e-2)
    g_gpu = binding.unpack_mlp_params(g, r, H)
    # Every product rounds both operands to bfloat16 (unit roundoff u = 2^-8), so a gradient
    # that passes through d products (3 forward + 1..3 backward) is within 2 u d of the
    # exact one, norm-wise, to first order: W3 d = 4, W2 d = 5, W1 d = 6.
    u = 2.0 ** -8
    depth = {"W3": 4, "b3": 3, "W2": 5, "b2": 4, "W1": 6, "b1": 5}
    for k in mlp.TRAINED:
        err = np.linalg.norm(g_gpu[k] - g_ref[k]) / np.linalg.norm(g_ref[k])
        assert err <= 2 * u * depth[k], (k, err)


def test_training_reduces_the_loss(yy_lib):
    import torch
    from oracle import mlp
    from paper_2509_16896_gb300 import binding
    r, H, R = 4, 64, 0.3
    rng = np.random.default_rng(3)
    X = rng.normal(size=(2048, 3 * r)).astype(np.float32)
    A = rng.normal(size=(3 * r, r)) * 0.05
    T = (X @ A + 0.02 * rng.normal(size=(2048, r))).astype(np.float32)
    net = binding.MLP(r, H, max_batch=128)
    net.set_params(binding.pack_mlp_params(mlp.init_params(r, H, 4)))
    xd, td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    l0, _ = net.loss_grad(xd[:128], td[:128], R)
    net.train(xd, td, R, epochs=15, batch=128, lr=2e-3, seed=5)
    l1, _ = net.loss_grad(xd[:128], td[:128], R)
    assert l1 < l0 - 0.5, (l0, l1)


@pytest.mark.parametrize("lam0,accepted", [(np.log(1.5), True), (3.0, False)])
def test_learned_restart_matches_oracle(yy_lib, lam0, accepted):
    """A network whose output is a known constant (W3 = 0, b3 = [delta0; lambda0]): the
    device restart must build the oracle's box, re-map the nodes bit for bit, set the
    oracle's weights, and predict with the new box volume."""
    import torch
    from oracle import filter as F, mlp, sobol
    from paper_2509_16896_gb300 import binding
    r, n, H, R = 6, 777, 16, 0.3
    p = mlp.init_params(r, H, 0)
    p["W3"][:] = 0.0
    delta0 = np.linspace(-0.05, 0.07, r).astype(np.float32).astype(np.float64)
    p["b3"][:r] = delta0
    p["b3"][r:] = np.float32(lam0)
    p["b3"] = p["b3"].astype(np.float32).astype(np.float64)
    cfg = binding.make_config(model="cubic", r=r, n=n, dt=0.01, R=R, n_scales=2, precision="f32",
                              restart_rule="learned")
    flt = binding.Filter(cfg)
    poly, scr = sobol_inputs(r, 61)
    flt.init_nodes(poly, scr, np.zeros(r))
    net = binding.MLP(r, H, max_batch=8)
    net.set_params(binding.pack_mlp_params(p))
    flt.set_restart_mlp(net)
    tr = simulate("cubic", r, 2, 0.01, seed=61)
    flt.predict()
    flt.update(torch.tensor(tr.dy[0], dtype=torch.float64, device="cuda"))
    mean, var, ess, z = flt.estimate()
    assert flt.restart(mode=1, report=True)
    cen, half = flt.get_box()
    prob = oracle_problem("cubic", r, n, 0.01, R, 2)
    prob.restart_rule, prob.mlp_params = "learned", p
    c_ref, h_ref, ok = mlp.proposal(p, mean, var, tr.dy[0], 0.01, prob.R)
    assert ok == accepted
    assert np.allclose(cen, c_ref, rtol=0, atol=1e-12) and np.allclose(half, h_ref, rtol=1e-12, atol=0)
    y, _ = sobol.nodes(poly, scr, n, R)
    u_ref = sobol.to_box(y, half)
    u_gpu, mask = flt.get_nodes()
    assert np.array_equal(u_gpu.view(np.uint32), u_ref.view(np.uint32))
    assert np.array_equal(mask, F.boundary_mask(u_ref, half))
    lw, _ = flt.get_log_weights()
    prep = F.prepare(prob, u_ref, cen, half)
    ref = F.restart_logw(prob, prep.x, cen, var, half)
    ref[prep.mask] = -np.inf
    assert rel_err(lw, ref) <= 1e-5
    # the next prediction uses the new box volume (quadrature factor and offset)
    flt.predict()
    pred, off = flt.get_log_weights()
    ref_pred, _ = F.predict(prob, prep, lw.astype(np.float64), half=half)
    assert rel_err(pred.astype(np.float64) + off, ref_pred) <= 1e-5


def test_trained_proposal_against_plain_rule(yy_lib):
    """Trains the network on restarts of plain runs (16 training trajectories) and runs
    both rules on held-out trajectories.  Reports the RMSE of each; the learned rule must
    run and stay finite, and its gain (or loss) is printed."""
    from paper_2509_16896_gb300 import learned_restart as LR
    from synth import WORKLOADS
    w = WORKLOADS["cubic_r50_n8192"].with_(n=4096, steps=150)
    X, T, _ = LR.collect_restarts(w, seeds=list(range(100, 116)))
    assert X.shape[0] > 500 and np.all(np.isfinite(X)) and np.all(np.isfinite(T))
    net, loss = LR.train_proposal(w.r, X, T, w.R, hidden=256, epochs=10, batch=256, lr=1e-3, seed=1)
    assert np.isfinite(loss)
    res = {}
    for rule in ("plain", "learned"):
        res[rule] = [LR.run_filter(w, s, rule, net=net)[0] for s in (5, 6)]
    print("RMSE plain", res["plain"], "learned", res["learned"])
    assert np.all(np.isfinite(res["learned"]))
