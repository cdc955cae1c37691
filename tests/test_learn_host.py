"""Host-side logic of the learned-policy pipeline (no GPU): the label
generator's copy of the heuristic policy, the allowed-action mask, and the
belief update of the planner episodes."""
import math

import numpy as np

import oracle
from paper_1802_06215_b300 import inputs as I
from paper_1802_06215_b300 import learn


def test_heuristic_action_matches_oracle_policy():
    cfg = I.rs15_15()
    om = oracle.Model(cfg)
    rng = np.random.default_rng(0)
    pos, s, h, _ = learn.random_states(cfg, 4000, rng)
    h[:, :cfg.m] = rng.integers(-2, 3, (4000, cfg.m))
    b = np.zeros((5, 4000), np.uint32)
    b[0], b[3] = pos, s
    assert np.array_equal(np.asarray(om.policy(b, h)).ravel(), learn.heuristic_action(cfg, pos, s, h))


def test_allowed_mask_rules():
    cfg = I.rs15_15()
    rx, ry = cfg.rock_cells[0] & 0xFF, cfg.rock_cells[0] >> 8
    pos = np.array([0 | (0 << 8), 14 | (14 << 8), rx | (ry << 8), rx | (ry << 8)], np.uint32)
    sampled = np.array([0, 0, 0, 1], np.uint32)
    hist = np.zeros((4, 32), np.int8)
    hist[:, 1] = 3
    al = learn.allowed_mask(cfg, pos, sampled, hist)
    assert al.shape == (4, 21) and al[:, 20].all() and al[:, 1].all()
    assert not al[0, 2] and not al[0, 3] and al[0, 0]      # bottom-left corner: no S, no W
    assert not al[1, 0] and al[1, 2] and al[1, 3]          # top-right: no N
    assert al[2, 4] and not al[3, 4]                       # Sample only on an unsampled rock
    assert not al[:, 5 + 1].any()                          # counter at +3: no more Sense of rock 1
    assert al[2, 5] and not al[3, 5]                       # no Sense of a sampled rock


def test_belief_update_is_bayes():
    cfg = I.rs15_15()
    b = learn.Belief(cfg, learn.start_word(cfg))
    c = int(cfg.rock_cells[2])
    d = math.hypot((c & 0xFF) - 0, (c >> 8) - 7)
    q = 0.5 + 0.5 * 2 ** (-d / 20)
    b.update(7, 1, b.pos, 0)       # Sense rock 2, reading good
    assert math.isclose(b.p[2], q) and b.hist[2] == 1
    b.update(7, 2, b.pos, 0)       # reading bad: back to the prior
    assert math.isclose(b.p[2], 0.5) and b.hist[2] == 0
    b.update(1, 0, b.pos + 1, 0)   # a move changes nothing but the position
    assert b.pos == learn.start_word(cfg) + 1 and np.count_nonzero(b.hist) == 0
    assert math.isclose(learn.counter_posterior(2, 0.8), 0.64 / 0.68)


def test_car_heuristic_action_matches_oracle_policy():
    cfg = I.car50()
    b, _ = learn.car_states(cfg, 800, np.random.default_rng(3))
    o = np.asarray(oracle.Model(cfg).policy(b, None)).ravel()
    assert np.array_equal(o, learn.car_heuristic_action(cfg, b))


def test_car_belief_block_keeps_the_observed_state():
    cfg = I.car50()
    rng = np.random.default_rng(4)
    b, _ = learn.car_states(cfg, 5, rng)
    bb = learn.car_belief_block(cfg, b[:, 2], 32, rng)
    P = cfg.P
    assert np.all(bb[0] == b[0, 2]) and np.all((bb[1] & 0xFF) == (b[1, 2] & 0xFF))
    assert np.all(bb[4:4 + 2 * P] == b[4:4 + 2 * P, 2:3])
    assert len(set(bb[2].tolist())) == 32  # distinct scenario streams
    goals = bb[4 + 2 * P:]
    assert len({tuple(goals[:, k]) for k in range(32)}) > 1  # goals are drawn per scenario
