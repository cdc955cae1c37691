"""The learned-policy pipeline's host logic and the policies it labels with.

On CPU: the belief update of the planner episodes (Bayes' rule with the
sensor law 0.5 + 0.5 * 2^(-d/20) of Sec. IV-A, read from the sensor table) and
the car's belief block. On the GPU: the library's default policies
(dsp_default_policy: Rock Sample with one and two robots, the car,
navigation) and the learned policy's allowed actions, which label the
training states, equal the oracle's policy functions state for state."""
import math

import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I
from paper_1802_06215_b300 import learn


def test_belief_update_is_bayes():
    cfg = I.rs15_15()
    b = learn.Belief(cfg, learn.start_word(cfg), oracle.sensor_thresholds(2 * 14 * 14))
    c = int(cfg.rock_cells[2])
    d = math.hypot((c & 0xFF) - 0, (c >> 8) - 7)
    q = 0.5 + 0.5 * 2 ** (-d / 20)
    b.update(7, 1, b.pos, 0)       # Sense rock 2, reading good
    assert math.isclose(b.p[2], q, rel_tol=1e-9) and b.hist[2] == 1
    b.update(7, 2, b.pos, 0)       # reading bad: back to the prior
    assert math.isclose(b.p[2], 0.5) and b.hist[2] == 0
    b.update(1, 0, b.pos + 1, 0)   # a move changes nothing but the position
    assert b.pos == learn.start_word(cfg) + 1 and np.count_nonzero(b.hist) == 0
    assert math.isclose(learn.counter_posterior(2, 0.8), 0.64 / 0.68)


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


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    return _dsp, batch


@pytest.mark.gpu
@pytest.mark.parametrize("name", ["rs15_15", "mars15_15", "rs32_15"])
def test_default_policy_matches_oracle_rock_sample(gpu, name):
    _dsp, batch = gpu
    cfg = I.grid_config(32, 15, K=500, D=90, seed=5) if name == "rs32_15" else getattr(I, name)()
    rng = np.random.default_rng(0)
    n = 5000
    pos = [(0, 0), (0, 0)][: 2 if cfg.kind == I.MULTIGRID else 1]
    b = I.rs_block(cfg, n, rng, pos=pos)
    for r in range(2 if cfg.kind == I.MULTIGRID else 1):
        b[r] = (rng.integers(0, cfg.n, n) | (rng.integers(0, cfg.n, n) << 8)).astype(np.uint32)
    b[3] = rng.integers(0, 1 << cfg.m, n).astype(np.uint32)
    b[2] &= ~b[3]
    # counters around zero: ties between equally near rocks, a rock underfoot
    h = rng.integers(-2, 3, (n, 32)).astype(np.int8)
    m = batch.Model(cfg)
    want_allowed = cfg.kind == I.GRID
    got = _dsp.default_policy(m.h, b, h, want_allowed=want_allowed)
    om = oracle.Model(cfg)
    acts = got[0] if want_allowed else got
    assert np.array_equal(acts, np.asarray(om.policy(b, h)).ravel())
    if want_allowed:
        assert np.array_equal(got[1], oracle.learned_allowed(om, b, h))
        assert np.array_equal(learn.allowed_mask(m, cfg, b[0], b[3], h)[:, :5 + cfg.m],
                              ((got[1][:, None] >> np.arange(5 + cfg.m, dtype=np.uint32)) & 1).astype(bool))
    m.close()


@pytest.mark.gpu
def test_default_policy_matches_oracle_car_and_navigation(gpu):
    _dsp, batch = gpu
    cfg = I.car50()
    b, _ = learn.car_states(cfg, 2000, np.random.default_rng(3))
    m = batch.Model(cfg)
    assert np.array_equal(_dsp.default_policy(m.h, b), np.asarray(oracle.Model(cfg).policy(b, None)).ravel())
    m.close()
    cfg = I.nav13()
    rng = np.random.default_rng(2)
    b = I.nav_block(cfg, 1000, rng)
    h = np.zeros((1000, 32), np.int8)
    h[:, 0] = rng.integers(0, 256, 1000).astype(np.uint8).view(np.int8)
    m = batch.Model(cfg)
    assert np.array_equal(_dsp.default_policy(m.h, b, h), np.asarray(oracle.Model(cfg).policy(b, h)).ravel())
    m.close()
