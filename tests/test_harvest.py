"""Training-data path of the learned default policy: device features against
the oracle's feature map, the tree export of a planning step, and one short
planner episode with belief updates."""
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
    from paper_1802_06215_b300 import _dsp, batch, build, learn
    build.build()
    return torch, _dsp, batch, learn


def test_features_match_oracle(env):
    torch, _dsp, batch, learn = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    rng = np.random.default_rng(5)
    for N in (1, 255, 1000):
        b = I.rs_block(cfg, N, rng)
        b[3] = rng.integers(0, 1 << 15, N).astype(np.uint32)
        hist = rng.integers(-6, 7, (N, 32)).astype(np.int8)
        g = learn.features(m, b, hist)
        o = oracle.features_rs(oracle.Model(cfg), b, hist)
        assert np.array_equal(g.view(np.uint32), o.view(np.uint32))
    m.close()


def test_plan_nodes_export(env):
    torch, _dsp, batch, learn = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    rng = np.random.default_rng(2)
    root = I.rs_block(cfg, cfg.K, rng, pos=[(0, 7)])
    hist = np.zeros(32, np.int8)
    hist[3] = 2
    p = _dsp.dsp_search_params(threads=2, rounds=6, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0,
                               deterministic=1, use_queue=0)
    ref = _dsp.dsp_plan(m.h, root, hist, p, m.num_actions)
    res, rec, st = _dsp.dsp_plan_nodes(m.h, root, hist, p, m.num_actions, 8, 4096, m.words)
    # the export does not change the search
    assert res["signature"] == ref["signature"] and res["action"] == ref["action"]
    assert len(rec) >= 2 and st.shape == (5, len(rec))
    r0 = rec[0]
    assert r0["depth"] == 0 and r0["n"] == cfg.K and r0["action"] == res["action"]
    assert r0["U"] == res["root_u"] and r0["L"] == res["root_l"]
    assert np.array_equal(r0["hist"], hist)
    assert np.array_equal(st[:, 0], root[:, 0])
    assert np.all(rec["n"] >= 8) and np.all((rec["action"] >= 0) & (rec["action"] < m.num_actions))
    assert np.all(rec["L"] <= rec["U"] + 1e-9)
    # depth-1 nodes sit where their action leads from the root (moves are deterministic)
    nxt, _, _ = m.step(np.tile(root[:, :1], (1, m.num_actions)), np.arange(m.num_actions, dtype=np.int32), 0)
    reach = set(nxt[0].tolist())
    for k in np.nonzero(rec["depth"] == 1)[0]:
        assert int(st[0, k]) in reach
    # a cap smaller than the tree truncates
    _, rec2, _ = _dsp.dsp_plan_nodes(m.h, root, hist, p, m.num_actions, 8, 1, m.words)
    assert len(rec2) == 1
    m.close()


def test_episode_harvest(env):
    torch, _dsp, batch, learn = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    ep = learn.episode(m, cfg, 7, 3, 0.02, threads=2, min_scen=16)
    assert 1 <= ep["decisions"] <= 3
    assert len(ep["roots"]) == ep["decisions"]
    X = learn.features(m, ep["states"], ep["hist"])
    assert X.shape == (len(ep["labels"]), 64)
    o = oracle.features_rs(oracle.Model(cfg), ep["states"], ep["hist"])
    assert np.array_equal(X, o)
    # the first root is the start belief: robot at (0, n/2), all counters zero
    r0, h0 = ep["roots"][0]
    assert np.all(r0[0] == learn.start_word(cfg)) and not h0.any()
    _, st = m.counters()
    assert st == 0
    m.close()
