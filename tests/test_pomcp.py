"""POMCP-style planning with the GPU as the rollout service against the CPU
oracle's planner: the same tree (node count, digest), root action values bit
for bit, visit counts, rollouts and decision, on every model."""
import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    return _dsp, batch


def roots(cfg, rng):
    if cfg.kind == I.CAR:
        base = (rng.uniform(0, 40, cfg.P), rng.uniform(0, 40, cfg.P))
        return I.car_block(cfg, cfg.K, rng, s=0.0, v=1, base=base, jitter=0.3)
    if cfg.kind == I.NAV:
        return I.nav_block(cfg, cfg.K, rng)
    pos = [(0, cfg.n // 2), (0, cfg.n // 2 - 1)][: (2 if cfg.kind == I.MULTIGRID else 1)]
    return I.rs_block(cfg, cfg.K, rng, pos=pos)


@pytest.mark.parametrize("name,cfg_fn,rounds,batch,c", [
    ("rs7_8", I.rs7_8, 12, 64, 10.0),
    ("rs15_15", I.rs15_15, 6, 256, 10.0),
    ("mars small", lambda: I.grid_config(7, 4, K=40, D=30, seed=3, robots=2), 8, 96, 10.0),
    ("car", lambda: I.car_config(P=10, K=60, D=25, seed=2), 6, 64, 100.0),
    ("nav13", lambda: I.nav_config(13, K=100, D=40, seed=2), 10, 128, 5.0),
])
def test_pomcp_matches_oracle(env, name, cfg_fn, rounds, batch, c):
    _dsp, batch_mod = env
    cfg = cfg_fn()
    b = roots(cfg, np.random.default_rng(11))
    m = batch_mod.Model(cfg)
    p = _dsp.dsp_pomcp_params(rounds=rounds, batch=batch, c=c, time_limit_s=0.0)
    g = _dsp.dsp_pomcp_plan(m.h, b, None, p, m.num_actions)
    o = oracle.Model(cfg).pomcp(b, None, rounds=rounds, batch=batch, c=c)
    m.close()
    assert g["nodes"] == o["nodes"] and g["signature"] == o["signature"], name
    assert np.array_equal(g["root_na"], o["root_na"]), name
    assert np.array_equal(g["root_q"], o["root_q"]), name
    assert g["action"] == o["action"] and g["value"] == o["value"], name
    assert g["rollouts"] == o["rollouts"] and g["simulations"] == o["simulations"], name
    assert g["scenario_steps"] == o["steps"], name


def test_pomcp_rejects_bad_parameters(env):
    _dsp, batch_mod = env
    cfg = I.rs7_8()
    m = batch_mod.Model(cfg)
    b = roots(cfg, np.random.default_rng(1))
    for kw in (dict(rounds=0, batch=8, c=1.0), dict(rounds=1, batch=0, c=1.0), dict(rounds=1, batch=8, c=-1.0)):
        with pytest.raises(_dsp.DspError):
            _dsp.dsp_pomcp_plan(m.h, b, None, _dsp.dsp_pomcp_params(time_limit_s=0.0, **kw), m.num_actions)
    m.close()
