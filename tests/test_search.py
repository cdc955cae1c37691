"""Tree search (Sec. III-C) on the GPU expansion against the CPU oracle.

Deterministic rounds must reproduce the oracle's search bit for bit (root
bounds, decision, node count, visit counts, tree digest); free-running threads
must keep valid bounds around the exhaustive optimum."""
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


def root_states(cfg, rng, n=None):
    n = cfg.K if n is None else n
    if cfg.kind == I.CAR:
        base = (rng.uniform(0, 40, cfg.P), rng.uniform(0, 40, cfg.P))
        return I.car_block(cfg, n, rng, s=0.0, v=1, base=base, jitter=0.0)
    if cfg.kind == I.NAV:
        return I.nav_block(cfg, n, rng)
    pos = [(0, cfg.n // 2), (0, cfg.n // 2 - 1)][: (2 if cfg.kind == I.MULTIGRID else 1)]
    return I.rs_block(cfg, n, rng, pos=pos)


def plan_both(env, cfg, b, **kw):
    _dsp, batch = env
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=kw.get("threads", 1), rounds=kw.get("rounds", 20), time_limit_s=0.0,
                               c_a=kw.get("c_a", 0.0), c_o=kw.get("c_o", 0.0), xi=kw.get("xi", 0.95),
                               target_gap=kw.get("target_gap", 0.0), deterministic=1)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    o = oracle.Model(cfg).plan(b, None, threads=p.threads, rounds=p.rounds, c_a=p.c_a, c_o=p.c_o, xi=p.xi,
                               target_gap=p.target_gap)
    m.close()
    return g, o


@pytest.mark.parametrize("name,cfg_fn,kw", [
    ("rs7_8 plain DESPOT", I.rs7_8, dict(threads=1, rounds=30)),
    ("rs7_8 T=4 UCT+vloss", I.rs7_8, dict(threads=4, rounds=25, c_a=1.0, c_o=0.5)),
    ("rs15_15 T=4", I.rs15_15, dict(threads=4, rounds=10, c_a=1.0, c_o=0.5)),
    ("mars small", lambda: I.grid_config(7, 4, K=40, D=30, seed=3, robots=2), dict(threads=4, rounds=8, c_a=1.0,
                                                                                   c_o=0.5)),
    ("car small", lambda: I.car_config(P=10, K=40, D=20, seed=2), dict(threads=2, rounds=6, c_a=1.0, c_o=0.5)),
    ("navigation 13x13", lambda: I.nav_config(13, K=60, D=40, seed=2), dict(threads=4, rounds=8, c_a=1.0, c_o=0.5)),
])
def test_deterministic_rounds_match_oracle(env, name, cfg_fn, kw):
    cfg = cfg_fn()
    b = root_states(cfg, np.random.default_rng(7))
    g, o = plan_both(env, cfg, b, **kw)
    assert g["root_u"] == o["root_u"] and g["root_l"] == o["root_l"], name
    assert g["action"] == o["action"], name
    assert g["nodes"] == o["nodes"] and g["expansions"] == o["expansions"] and g["rounds"] == o["rounds"], name
    assert np.array_equal(g["root_visits"], o["root_na"]), name
    assert g["signature"] == o["signature"], name
    assert g["scenario_steps"] == o["steps"], name


def test_search_converges_to_exhaustive_optimum(env):
    """xi = 0 expands every branch with a gap: the root bounds meet at V*_D of
    the tiny scenario tree (3x3 map, 2 rocks, K = 6, D = 4)."""
    cfg = I.Config(kind=I.GRID, n=3, m=2, K=6, D=4, seed=1,
                   rock_cells=np.array([1 | (1 << 8), 2], np.int32))
    b = root_states(cfg, np.random.default_rng(1))
    vstar = oracle.Model(cfg, fp64=True).exhaustive(b, None, 0)
    g, o = plan_both(env, cfg, b, threads=2, rounds=100000, xi=0.0)
    assert abs(g["root_u"] - vstar) < 1e-5 and abs(g["root_l"] - vstar) < 1e-5


@pytest.mark.parametrize("tree_lock", [0, 1])
@pytest.mark.parametrize("threads", [1, 4, 16])
def test_free_running_threads_valid(env, threads, tree_lock):
    """Free-running threads with PO-UCT and virtual loss, on per-node atomics
    or under one tree lock: bounds stay around the exhaustive optimum and the
    budget holds."""
    _dsp, batch = env
    cfg = I.Config(kind=I.MULTIGRID, n=3, m=2, K=6, D=4, seed=4,
                   rock_cells=np.array([1 | (1 << 8), 2], np.int32))
    b = root_states(cfg, np.random.default_rng(4))
    vstar = oracle.Model(cfg, fp64=True).exhaustive(b, None, 0)
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=threads, rounds=20, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, tree_lock=tree_lock)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= vstar + 1e-5 and vstar <= g["root_u"] + 1e-5
    assert 1 <= g["expansions"] <= threads * 20
    assert g["root_visits"].sum() >= 1
    m.close()


def test_free_running_rs15_time_limit(env):
    """The 15x15 task with 4 threads under a time budget returns valid bounds."""
    _dsp, batch = env
    cfg = I.rs15_15()
    b = root_states(cfg, np.random.default_rng(2))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=4, rounds=100000, time_limit_s=0.5, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= g["root_u"] + 1e-9
    assert g["expansions"] >= 4 and g["seconds"] < 5.0
    m.close()


@pytest.mark.parametrize("mk", [lambda: I.Config(kind=I.MULTIGRID, n=3, m=2, K=6, D=4, seed=4,
                                                 rock_cells=np.array([1 | (1 << 8), 2], np.int32))])
def test_free_running_through_queue(env, mk):
    """16 threads submitting their leaves to the device job queue: valid
    bounds around the exhaustive optimum."""
    _dsp, batch = env
    cfg = mk()
    b = root_states(cfg, np.random.default_rng(4))
    vstar = oracle.Model(cfg, fp64=True).exhaustive(b, None, 0)
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=16, rounds=10, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, use_queue=1)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= vstar + 1e-5 and vstar <= g["root_u"] + 1e-5
    assert 1 <= g["expansions"] <= 160
    m.close()


def test_mars15_16_threads_queue(env):
    """The two-robot 15x15 task (400 joint actions, K = 500) planned by 16
    threads through the queue for 1 s: valid bounds, many expansions."""
    _dsp, batch = env
    cfg = I.mars15_15()
    b = root_states(cfg, np.random.default_rng(3))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=16, rounds=100000, time_limit_s=1.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, use_queue=1)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= g["root_u"] + 1e-9
    assert g["expansions"] >= 16
    m.close()


@pytest.mark.parametrize("tree_lock,launch_batch", [(0, 0), (1, 0), (0, 8), (1, 8)])
def test_free_running_one_thread_is_the_rounds_search(env, tree_lock, launch_batch):
    """One free-running thread selects, expands and backs up in the order of
    one-trial deterministic rounds (with batched launches it dispatches its
    own leaf at once), so on per-node atomics (with the final bottom-up pass)
    or under the tree lock it builds the same tree as the oracle's search:
    equal digest, bounds and visits."""
    _dsp, batch = env
    cfg = I.rs7_8()
    b = root_states(cfg, np.random.default_rng(7))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=1, rounds=30, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, tree_lock=tree_lock, batch=launch_batch)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    m.close()
    o = oracle.Model(cfg).plan(b, None, threads=1, rounds=30, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0)
    assert g["signature"] == o["signature"]
    assert g["root_u"] == o["root_u"] and g["root_l"] == o["root_l"]
    assert np.array_equal(g["root_visits"], o["root_na"])


@pytest.mark.parametrize("name,cfg_fn", [
    ("rs7_8", I.rs7_8),
    ("car small", lambda: I.car_config(P=10, K=40, D=20, seed=2)),
    ("navigation 13x13", lambda: I.nav_config(13, K=60, D=40, seed=2)),
])
def test_one_thread_through_queue_is_the_rounds_search(env, name, cfg_fn):
    """One free-running thread whose leaves go through the device job queue
    (each model's persistent kernel) builds the oracle's tree: equal digest,
    bounds and visits."""
    _dsp, batch = env
    cfg = cfg_fn()
    b = root_states(cfg, np.random.default_rng(7))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=1, rounds=12, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, use_queue=1)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    m.close()
    o = oracle.Model(cfg).plan(b, None, threads=1, rounds=12, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0)
    assert g["signature"] == o["signature"], name
    assert g["root_u"] == o["root_u"] and g["root_l"] == o["root_l"], name
    assert np.array_equal(g["root_visits"], o["root_na"]), name


@pytest.mark.parametrize("tree_lock", [0, 1])
@pytest.mark.parametrize("threads", [4, 16])
def test_free_running_batched_launches_valid(env, threads, tree_lock):
    """Threads handing their leaves to one dispatcher that expands up to 8 per
    launch: bounds around the exhaustive optimum, the budget holds."""
    _dsp, batch = env
    cfg = I.Config(kind=I.MULTIGRID, n=3, m=2, K=6, D=4, seed=4,
                   rock_cells=np.array([1 | (1 << 8), 2], np.int32))
    b = root_states(cfg, np.random.default_rng(4))
    vstar = oracle.Model(cfg, fp64=True).exhaustive(b, None, 0)
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=threads, rounds=20, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, tree_lock=tree_lock, batch=8)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= vstar + 1e-5 and vstar <= g["root_u"] + 1e-5
    assert 1 <= g["expansions"] <= threads * 20
    m.close()


def test_free_running_batched_rs15(env):
    """15x15 with 16 threads and up to 64 leaves per launch for 0.5 s: valid
    bounds, many expansions."""
    _dsp, batch = env
    cfg = I.rs15_15()
    b = root_states(cfg, np.random.default_rng(2))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=16, rounds=100000, time_limit_s=0.5, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, batch=64)
    g = _dsp.dsp_plan(m.h, b, None, p, m.num_actions)
    assert g["root_l"] <= g["root_u"] + 1e-9
    assert g["expansions"] >= 16 and g["seconds"] < 5.0
    m.close()


@pytest.mark.parametrize("launch_batch", [0, 32])
def test_lock_free_tree_bounds_consistent(env, launch_batch):
    """16 lock-free threads for 0.5 s on 15x15, then the exported tree: every
    expanded node keeps U >= L, the root's bounds are the first node's, and
    the visit counts of the root's actions add up to the root's visits."""
    _dsp, batch = env
    cfg = I.rs15_15()
    b = root_states(cfg, np.random.default_rng(5))
    m = batch.Model(cfg)
    p = _dsp.dsp_search_params(threads=16, rounds=100000, time_limit_s=0.5, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, batch=launch_batch)
    g, nodes, _ = _dsp.dsp_plan_nodes(m.h, b, None, p, m.num_actions, 1, 100000, m.words)
    m.close()
    assert len(nodes) >= 2
    assert np.all(nodes["U"] >= nodes["L"] - 1e-9)
    root = nodes[0]
    assert root["depth"] == 0 and root["U"] == g["root_u"] and root["L"] == g["root_l"]
    assert int(g["root_visits"].sum()) == int(root["visits"])


def test_deterministic_rounds_large_root(env):
    """One robot with 2000 root scenarios (leaves above 512 take phase A's
    global-memory path): the deterministic search equals the oracle's."""
    cfg = I.rs15_15_k(2000)
    b = root_states(cfg, np.random.default_rng(11))
    g, o = plan_both(env, cfg, b, threads=2, rounds=4, c_a=1.0, c_o=0.5)
    assert g["signature"] == o["signature"]
    assert g["root_u"] == o["root_u"] and g["root_l"] == o["root_l"] and g["action"] == o["action"]
    assert g["scenario_steps"] == o["steps"]
