"""Pins for the oracle's restart-proposal network (oracle/mlp.py)."""
import numpy as np
import pytest

from oracle import filter as F, mlp, sobol
from synth import simulate, sobol_poly_params, sobol_scramble_params


def _setup(r=3, hidden=8, B=5, seed=0):
    p = mlp.init_params(r, hidden, seed)
    rng = np.random.default_rng(seed)
    for k in mlp.TRAINED:   # non-trivial values everywhere (the init has zero biases and tiny W3)
        p[k] = p[k] + 0.3 * rng.normal(size=p[k].shape)
    p["mu"] = 0.1 * rng.normal(size=3 * r)
    p["s"] = 1.0 + 0.2 * rng.random(3 * r)
    z = rng.normal(size=(B, 3 * r))
    t = 0.2 * rng.normal(size=(B, r))
    return p, z, t


def test_backward_matches_central_differences():
    p, z, t = _setup()
    R = 0.3
    o, cache = mlp.forward(p, z)
    L, g_o = mlp.loss_and_grad_out(o, t, R)
    g = mlp.backward(p, cache, g_o)
    rng = np.random.default_rng(1)
    h = 1e-6
    for k in mlp.TRAINED:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[k].shape)
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            Lp, _ = mlp.loss_and_grad_out(mlp.forward(q, z)[0], t, R)
            q[k][idx] -= 2 * h
            Lm, _ = mlp.loss_and_grad_out(mlp.forward(q, z)[0], t, R)
            fd = (Lp - Lm) / (2 * h)
            assert g[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (k, idx)


def test_loss_hand_value():
    # one row, r = 1: delta = 0.1, lambda = 0 -> sigma = R/3 = 0.1 ; t = 0.3: e = 0.2
    o = np.array([[0.1, 0.0]])
    L, g = mlp.loss_and_grad_out(o, np.array([[0.3]]), 0.3)
    assert L == pytest.approx(0.04 / (2 * 0.01) + np.log(0.1))
    assert g[0, 0] == pytest.approx(-0.2 / 0.01)
    assert g[0, 1] == pytest.approx(1.0 - 0.04 / 0.01)


def test_adam_first_step_is_signed_lr():
    p = {"w": np.array([1.0, -2.0])}
    g = {"w": np.array([0.5, -3.0])}
    m = {"w": np.zeros(2)}
    v = {"w": np.zeros(2)}
    mlp.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01], atol=1e-7)


def test_proposal_falls_back_to_plain_rule():
    r = 2
    p = mlp.init_params(r, 4, 0)
    R = np.full(r, 0.3)
    mean, var, dy = np.array([0.5, -0.1]), np.array([0.01, 0.02]), np.array([0.03, 0.0])
    p["b3"][r:] = 5.0   # half-width R e^5 > 8R: rejected
    c, h, ok = mlp.proposal(p, mean, var, dy, 0.01, R, np.zeros(r))
    assert not ok and np.array_equal(c, mean) and np.array_equal(h, R)
    p["b3"][r:] = np.log(2.0)
    p["b3"][:r] = [0.05, -0.02]
    p["W3"][:] = 0.0
    c, h, ok = mlp.proposal(p, mean, var, dy, 0.01, R, np.zeros(r))
    assert ok and np.allclose(c, mean + [0.05, -0.02]) and np.allclose(h, 2 * R)


def test_zero_output_network_reproduces_plain_restarts():
    """delta = 0, lambda = 0: the learned rule is the plain rule, step for step."""
    r, n = 4, 256
    poly, scr = sobol_poly_params(r, 3), sobol_scramble_params(r, 3)
    y, u = sobol.nodes(poly, scr, n, 0.3)
    params = mlp.init_params(r, 8, 0)
    params["W3"][:] = 0.0
    tr = simulate("cubic", r, 6, 0.01, seed=3)
    out = []
    for rule in ("plain", "learned"):
        p = F.Problem(model="cubic", r=r, n=n, dt=0.01, R=np.full(r, 0.3), n_scales=2, restart_interval=2,
                      restart_rule=rule, mlp_params=params)
        st = F.init_state(p, u, np.zeros(r))
        st.y = y
        recs = F.run(p, st, tr.dy)
        out.append(np.array([q.mean for q in recs]))
    assert np.array_equal(out[0], out[1])


def test_normalisation_clamps_out_of_range_features():
    p = mlp.init_params(2, 4, 0)
    p["mu"] = np.array([1.0, 0, 0, 0, 0, 0])
    p["s"] = np.full(6, 0.5)
    zn = mlp.normalise(p, np.array([[1.5, 10.0, -10.0, 0.0, 0.5, 2.1]]))
    assert np.allclose(zn, [[1.0, 4.0, -4.0, 0.0, 1.0, 4.0]])


def test_box_must_contain_the_estimate():
    r = 2
    p = mlp.init_params(r, 4, 0)
    p["W3"][:] = 0.0
    p["b3"][:r] = [0.5, 0.0]      # shift beyond the half-width R = 0.3
    R = np.full(r, 0.3)
    c, h, ok = mlp.proposal(p, np.zeros(r), np.full(r, 0.01), np.zeros(r), 0.01, R, np.zeros(r))
    assert not ok
