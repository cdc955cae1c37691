"""Pins of the oracle's policy network, loss gradient, features and learned
rollout (no GPU)."""
import os

import numpy as np

import oracle
from paper_1802_06215_b300 import inputs as I

G32 = float(np.float32(0.95))


def rand_weights(seed, scale=0.2):
    rng = np.random.default_rng(seed)
    return {"W1": rng.normal(0, scale, (64, 256)), "b1": rng.normal(0, 0.1, 256),
            "W2": rng.normal(0, scale / 2, (256, 256)), "b2": rng.normal(0, 0.1, 256),
            "W3": rng.normal(0, scale, (256, 32)), "b3": rng.normal(0, 0.1, 32)}


def test_gradient_matches_finite_differences():
    w = rand_weights(1)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (6, 64))
    y = rng.integers(0, 20, 6)
    loss, g = oracle.mlp_loss_grad(w, X, y, 20)
    eps = 1e-6
    for name, idx in [("W1", (3, 7)), ("W1", (60, 200)), ("b1", (11,)), ("W2", (5, 9)), ("W2", (255, 0)),
                      ("b2", (100,)), ("W3", (17, 4)), ("b3", (19,)), ("b3", (0,))]:
        wp = {k: v.copy() for k, v in w.items()}
        wm = {k: v.copy() for k, v in w.items()}
        wp[name][idx] += eps
        wm[name][idx] -= eps
        lp, _ = oracle.mlp_loss_grad(wp, X, y, 20)
        lm, _ = oracle.mlp_loss_grad(wm, X, y, 20)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[name][idx]) <= 1e-4 * max(1e-3, abs(fd)) + 1e-9, (name, idx, fd, g[name][idx])
    # logits beyond the action count carry no gradient
    assert np.all(g["b3"][20:] == 0) and np.all(g["W3"][:, 20:] == 0)


def test_zero_weights_reduce_to_softmax_of_bias():
    """All weights zero: logits = b3 and the loss is -log softmax(b3)[y]."""
    w = rand_weights(3)
    for k in ("W1", "W2", "W3", "b1", "b2"):
        w[k][:] = 0
    X = np.random.default_rng(4).normal(0, 1, (3, 64))
    lg = oracle.mlp_forward(w, X)
    assert np.allclose(lg, w["b3"][None, :])
    y = np.array([0, 5, 12])
    loss, _ = oracle.mlp_loss_grad(w, X, y, 13)
    z = w["b3"][:13]
    ref = np.mean([-(z[k] - np.log(np.exp(z).sum())) for k in y])
    assert abs(loss - ref) < 1e-12


def test_bf16_forward_close_to_exact():
    w = rand_weights(5)
    X = np.random.default_rng(6).normal(0, 1, (16, 64))
    a = oracle.mlp_forward(w, X)
    b = oracle.mlp_forward(w, X, bf16=True)
    assert np.max(np.abs(a - b)) <= 3e-2 * np.max(np.abs(a))


def test_features_golden():
    cfg = I.Config(kind=I.GRID, n=5, m=2, K=4, D=10, seed=0, rock_cells=np.array([1 | (2 << 8), 4], np.int32))
    m = oracle.Model(cfg)
    b = np.zeros((5, 1), np.uint32)
    b[0] = 2 | (3 << 8)
    b[3] = 2
    h = np.zeros((1, 32), np.int8)
    h[0, 0], h[0, 1] = 5, -1
    f = oracle.features_rs(m, b, h)[0]
    vals = [float(x) for x in open(os.path.join(os.path.dirname(__file__), "golden", "rs_features.txt")).read()
            .split("\n")[-2].split()]
    assert np.allclose(f[:10], vals, atol=1e-7)
    assert np.all(f[10:] == 0)


def test_learned_rollout_constant_east_is_closed_form():
    """A network whose logits are its bias, largest for E: the learned rollout
    walks east, worth 10 * gamma^(n-1-x) (the fixed-sequence closed form)."""
    w = rand_weights(7)
    for k in ("W1", "W2", "W3", "b1", "b2"):
        w[k][:] = 0
    w["b3"][:] = 0
    w["b3"][1] = 5.0
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    rng = np.random.default_rng(0)
    for x in (0, 7, 14):
        b = I.rs_block(cfg, 3, rng, pos=[(x, 4)])
        v, bad, steps = oracle.rollout_learned(m, b, None, 3, w)
        assert np.allclose(v, 10 * G32 ** (14 - x), rtol=1e-6)
        assert steps == 3 * (15 - x)
        # replaying the same actions agrees everywhere
        logged = np.full((3, cfg.D), 1, np.int32)
        v2, bad2, _ = oracle.rollout_learned(m, b, None, 3, w, logged=logged)
        assert np.array_equal(v, v2) and np.all(bad2 == 0)
