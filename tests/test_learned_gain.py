"""What the trained network gains over the method without it: the shipped
weights (imitation of the plain planner's chosen actions, `learn train`, then
approximate policy iteration from that network, `learn api --init`) against
the heuristic default policy, in rollout value (the l0 it gives) and in the
root gap u - l after planning steps of equal time; two iterations of policy
iteration from scratch already beating the heuristic from the start belief;
and the imitation labels' rules (defer where the planner chose the
heuristic's action, only actions the learned policy may take)."""
import os

import numpy as np
import pytest

from paper_1802_06215_b300 import inputs as I

pytestmark = pytest.mark.gpu
WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_1802_06215_b300", "weights", "rs15_15_pi0.npz")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build, learn
    build.build()
    return _dsp, batch, learn


def start_states(learn, cfg, n):
    return (np.full(n, learn.start_word(cfg), np.uint32), np.zeros(n, np.uint32), np.zeros((n, 32), np.int8),
            np.zeros(n, np.int32))


def test_trained_policy_raises_rollout_values(env):
    _dsp, batch, learn = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    h, meta = learn.load_weights(WEIGHTS)
    ev = learn.random_states(cfg, 4000, np.random.default_rng(77))
    st = start_states(learn, cfg, 2000)
    heur = [learn.mean_rollout_value(m, cfg, *x, np.random.default_rng(5)) for x in (st, ev)]
    _dsp.dsp_set_policy(m.h, h)
    lrn = [learn.mean_rollout_value(m, cfg, *x, np.random.default_rng(5)) for x in (st, ev)]
    _, status = m.counters()
    assert status == 0
    assert lrn[0] > 2.0 * heur[0], (lrn, heur)
    assert lrn[1] > heur[1] + 1.0, (lrn, heur)
    _dsp.dsp_mlp_destroy(h)
    m.close()


def test_trained_policy_tightens_root_gap(env):
    _dsp, batch, learn = env
    cfg = I.rs15_15()
    h, _ = learn.load_weights(WEIGHTS)
    roots = learn.eval_roots(cfg, [9100, 9101], 3, 0.05)
    out = learn.compare(cfg, h, roots, 0.3)
    assert out["learned"]["mean_root_gap"] < out["heuristic"]["mean_root_gap"], out
    assert out["learned"]["mean_root_l"] > out["heuristic"]["mean_root_l"], out
    _dsp.dsp_mlp_destroy(h)


def test_policy_iteration_from_scratch(env):
    _dsp, batch, learn = env
    cfg = I.rs15_15()
    logs = []
    h, hl = learn.policy_iteration(cfg, iterations=2, n_random=60000, n_onpolicy=4000, Kq=64, epochs=30, seed=0,
                                   log=logs.append)
    last = hl[-1]
    assert last["learned_value"]["start"] > last["heuristic_value"]["start"] + 1.0, hl
    assert last["learned_value"]["random_states"] > last["heuristic_value"]["random_states"], hl
    _dsp.dsp_mlp_destroy(h)


CAR_WEIGHTS = os.path.join(os.path.dirname(__file__), "..", "paper_1802_06215_b300", "weights", "car50_pi0.npz")


def test_trained_car_policy_raises_rollout_values(env):
    _dsp, batch, learn = env
    cfg = I.car50()
    m = batch.Model(cfg)
    b, d = learn.car_states(cfg, 2000, np.random.default_rng(21))
    heur = learn.car_mean_value(m, cfg, b, d, np.random.default_rng(2))
    h, _ = learn.load_weights(CAR_WEIGHTS)
    _dsp.dsp_set_policy(m.h, h)
    lrn = learn.car_mean_value(m, cfg, b, d, np.random.default_rng(2))
    _, status = m.counters()
    assert status == 0
    assert lrn > heur + 10.0, (lrn, heur)
    _dsp.dsp_mlp_destroy(h)
    m.close()


def test_trained_car_policy_tightens_root_gap(env):
    _dsp, batch, learn = env
    cfg = I.car50()
    h, _ = learn.load_weights(CAR_WEIGHTS)
    out = learn.compare(cfg, h, learn.car_roots(cfg, 3, 9100), 0.1)
    assert out["learned"]["mean_root_gap"] < out["heuristic"]["mean_root_gap"], out
    assert out["learned"]["mean_root_l"] > out["heuristic"]["mean_root_l"], out
    _dsp.dsp_mlp_destroy(h)


def test_imitation_labels_follow_the_planner(env):
    """Tree nodes of one planner episode: each kept label is the planner's
    action, or |A| exactly where that action is the heuristic's; a pair is
    dropped exactly when the learned policy may not take the action."""
    _dsp, batch, learn = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    ep = learn.episode(m, cfg, 1234, 6, 0.05, min_scen=16)
    assert "states" in ep and len(ep["labels"]) > 50
    st, hist, act = ep["states"], ep["hist"], ep["labels"].astype(np.int32)
    keep, y = learn.imitation_labels(m, cfg, st, hist, act)
    heur = learn.heuristic_action(m, st[0], st[3], hist)
    allowed = learn.allowed_mask(m, cfg, st[0], st[3], hist)
    na = m.num_actions
    assert np.array_equal(keep, allowed[np.arange(len(act)), act])
    assert np.array_equal(y == na, act == heur)
    assert np.all(y[act != heur] == act[act != heur])
    assert 0 < keep.sum() and np.all((y >= 0) & (y <= na))
    m.close()
