"""What the trained network gains over the method without it: the shipped
weights (approximate policy iteration, `learn api --iterations 4 --epochs 30`)
against the heuristic default policy, in rollout value (the l0 it gives) and
in the root gap u - l after planning steps of equal time; and two iterations
of policy iteration from scratch already beating the heuristic from the start
belief."""
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
