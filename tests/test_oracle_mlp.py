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


def bias_net(prefs):
    """A network whose logits are its output bias: prefs maps action -> logit."""
    w = rand_weights(7)
    for k in w:
        w[k][:] = 0
    for a, v in prefs.items():
        w["b3"][a] = v
    return w


def test_learned_rollout_masks_border_moves():
    """N preferred, then E: the robot climbs to the top row, where N is not
    allowed (it would cost -100 and stay), then walks east along it:
    10 * gamma^((n-1-y) + (n-1-x))."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    w = bias_net({0: 5.0, 1: 1.0})
    rng = np.random.default_rng(1)
    for x, y in ((0, 0), (3, 14), (14, 9), (6, 6)):
        b = I.rs_block(cfg, 2, rng, pos=[(x, y)])
        v, _, steps = oracle.rollout_learned(m, b, None, 0, w)
        assert np.allclose(v, 10 * G32 ** ((14 - y) + (14 - x)), rtol=1e-6)
        assert steps == 2 * ((14 - y) + (15 - x))
        # a logged border move is reported as a disagreement
        logged = np.full((2, cfg.D), 1, np.int32)
        logged[:, 0] = 3 if x == 0 else 0
        _, bad, _ = oracle.rollout_learned(m, b, None, 0, w, logged=logged)
        if x == 0 or y == 14:
            assert np.all(bad >= 1)


def test_learned_rollout_samples_only_unsampled_rocks():
    """Sample preferred, then E: along a row the robot samples each unsampled
    rock it stands on once (+-10 by its hidden state) and exits."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    w = bias_net({4: 5.0, 1: 1.0})
    cells = cfg.rock_cells
    rx, ry = cells & 0xFF, cells >> 8
    rng = np.random.default_rng(2)
    for y in range(cfg.n):
        on_row = [i for i in range(cfg.m) if ry[i] == y]
        for pre in (0, 1):
            b = I.rs_block(cfg, 4, rng, pos=[(0, y)])
            if pre and on_row:
                b[3] |= np.uint32(1 << on_row[0])
                b[2] &= ~b[3]
            v, _, _ = oracle.rollout_learned(m, b, None, 0, w)
            for s in range(4):
                t, expect = 0, 0.0
                for xx in range(cfg.n):
                    for i in on_row:
                        if rx[i] == xx and not (int(b[3, s]) >> i) & 1:
                            expect += G32 ** t * (10.0 if (int(b[2, s]) >> i) & 1 else -10.0)
                            t += 1
                    t += 1
                expect += 10.0 * G32 ** (t - 1) - 0.0
                assert np.isclose(v[s], expect, rtol=1e-5), (y, pre, s, v[s], expect)


def test_learned_rollout_sensing_is_bounded():
    """Sense rock 0 preferred, then E: the robot senses until the counter
    reads +-3 (an odd number k >= 3 of readings) and walks east, so the value
    is 10 * gamma^(k + n-1-x); with rock 0 sampled it walks east at once."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    w = bias_net({5: 5.0, 1: 1.0})
    rng = np.random.default_rng(3)
    b = I.rs_block(cfg, 200, rng, pos=[(4, 2)])
    v, _, _ = oracle.rollout_learned(m, b, None, 0, w)
    k = np.log(v / 10.0) / np.log(G32) - 10
    kr = np.round(k)
    assert np.allclose(k, kr, atol=1e-3)
    assert np.all(kr >= 3) and np.all(kr % 2 == 1)
    b[3] |= 1
    b[2] &= ~b[3]
    v2, _, _ = oracle.rollout_learned(m, b, None, 0, w)
    assert np.allclose(v2, 10 * G32 ** 10, rtol=1e-6)


def test_learned_rollout_never_pays_illegal_penalties():
    """Whatever the network, the allowed-action rule keeps every reward at
    least -10 (a bad rock), so a rollout is worth more than -10 per rock."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    rng = np.random.default_rng(4)
    for seed in range(3):
        w = rand_weights(seed)
        w["b3"] = rng.normal(0, 3, 32)
        b = I.rs_block(cfg, 40, rng)
        b[2] &= ~b[3]
        hist = rng.integers(-4, 5, (40, 32)).astype(np.int8)
        v, _, _ = oracle.rollout_learned(m, b, hist, 0, w)
        assert np.all(v >= -10.0 * cfg.m)


def test_learned_rollout_defer_is_the_heuristic():
    """A network whose largest logit is column |A| ("defer") takes the
    heuristic policy's action at every step: its rollouts equal the heuristic
    rollouts (Eq. lb with the hand-written default policy) value for value."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    w = bias_net({20: 5.0, 1: 1.0, 4: 2.0})
    rng = np.random.default_rng(6)
    b = I.rs_block(cfg, 300, rng)
    b[3] = rng.integers(0, 1 << 15, 300).astype(np.uint32)
    b[2] &= ~b[3]
    hist = rng.integers(-2, 4, (300, 32)).astype(np.int8)
    for d0 in (0, 7):
        v, bad, steps = oracle.rollout_learned(m, b, hist, d0, w)
        vh, steps_h = m.rollout(b, hist, d0)
        assert np.array_equal(v.astype(np.float32), vh.astype(np.float32)) and steps == steps_h
    # the same network one logit lower on defer: the East/Sample preferences take over
    w2 = bias_net({20: 0.5, 1: 1.0, 4: 2.0})
    v2, _, _ = oracle.rollout_learned(m, b, hist, 0, w2)
    assert not np.array_equal(v2, oracle.rollout_learned(m, b, hist, 0, w)[0])


def car_state(cfg, s, v, peds):
    b = np.zeros((I.words(cfg), 1), np.uint32)
    b[0, 0] = np.float32(s).view(np.uint32)
    b[1, 0] = v
    for j, (x, y, g) in enumerate(peds):
        b[4 + j, 0] = np.float32(x).view(np.uint32)
        b[4 + cfg.P + j, 0] = np.float32(y).view(np.uint32)
        b[4 + 2 * cfg.P + j // 4, 0] |= np.uint32(g << (8 * (j % 4)))
    return b


def test_car_features_golden():
    cfg = I.car_config(P=3, K=4, D=10, seed=0)
    b = car_state(cfg, 5.0, 2, [(-2.0, 20.5, 0), (-5.0, 26.0, 0), (0.0, 19.0, 0)])
    f = oracle.features_car(oracle.Model(cfg), b)[0]
    vals = [float(x) for x in open(os.path.join(os.path.dirname(__file__), "golden", "car_features.txt")).read()
            .split("\n")[-2].split()]
    assert np.allclose(f[:11], vals, atol=1e-6)
    assert np.all(f[11:] == 0)


def test_car_learned_defer_is_the_heuristic():
    """A network whose largest logit is column 3 ("defer") takes the car
    heuristic's action at every step: value for value the heuristic rollout."""
    cfg = I.car50()
    m = oracle.Model(cfg)
    w = bias_net({3: 5.0, 0: 1.0})
    rng = np.random.default_rng(8)
    b = I.car_block(cfg, 24, rng)
    for d0 in (0, 20):
        v, _, steps = oracle.rollout_learned(m, b, None, d0, w)
        vh, sh = m.rollout(b, None, d0)
        assert np.array_equal(v.astype(np.float32), vh.astype(np.float32)) and steps == sh


def test_car_learned_constant_actions_closed_form():
    """With action failures off and one pedestrian standing far away:
    always Accelerate reaches s = 60 m after T steps (speeds 1, 2, 3, 3, ...
    m/s, 0.33 s per step), worth 1000 gamma^(T-1); always Decelerate stays at
    rest and pays 0.1 per step, -0.1 (1 - gamma^n) / (1 - gamma)."""
    cfg = I.car_config(P=1, K=4, D=100, seed=0).with_(fail_p=0.0)
    m = oracle.Model(cfg)
    b = car_state(cfg, 0.0, 0, [(0.0, 0.0, 0)])
    s, v, T = np.float32(0), 0, None
    for t in range(cfg.D):
        v = min(v + 1, 3)
        s = np.float32(s + np.float32(v) * np.float32(0.33))
        if s >= 60:
            T = t + 1
            break
    va, _, steps = oracle.rollout_learned(m, b, None, 0, bias_net({0: 5.0}))
    assert np.isclose(va[0], 1000 * 0.95 ** (T - 1), rtol=1e-5) and steps == T
    vd, _, steps = oracle.rollout_learned(m, b, None, 0, bias_net({2: 5.0}))
    n = cfg.D
    assert np.isclose(vd[0], -0.1 * (1 - 0.95 ** n) / (1 - 0.95), rtol=1e-5) and steps == n
