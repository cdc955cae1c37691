"""Pins of the POMCP-style oracle planner: the virtual visits spread a fresh
node's first simulations over the actions, every simulation passes the root
once, a one-step horizon gives each action the mean reward of the scenarios
that tried it (step values pinned elsewhere), and on a tiny task the root
value rises toward the optimum of the exhaustive scenario tree (a fixed-seed
check, not a bound)."""
import numpy as np

import oracle
from paper_1802_06215_b300 import inputs as I


def tiny():
    return I.Config(kind=I.MULTIGRID, n=3, m=2, K=6, D=4, seed=4, rock_cells=np.array([1 | (1 << 8), 2], np.int32))


def test_first_round_tries_every_action_once():
    cfg = I.rs7_8()
    om = oracle.Model(cfg)
    b = I.rs_block(cfg, cfg.K, np.random.default_rng(0), pos=[(0, 3)])
    na = om.num_actions()
    r = om.pomcp(b, None, rounds=1, batch=na, c=1.0)
    assert np.array_equal(r["root_na"], np.ones(na, np.int32))
    r = om.pomcp(b, None, rounds=1, batch=3 * na, c=1.0)
    assert np.array_equal(r["root_na"], np.full(na, 3, np.int32))


def test_every_simulation_passes_the_root():
    cfg = I.nav13()
    om = oracle.Model(cfg)
    b = I.nav_block(cfg, cfg.K, np.random.default_rng(1))
    r = om.pomcp(b, None, rounds=7, batch=50, c=2.0)
    assert r["simulations"] == 350 and int(r["root_na"].sum()) == 350
    assert 0 < r["rollouts"] <= 350
    again = om.pomcp(b, None, rounds=7, batch=50, c=2.0)
    assert again["signature"] == r["signature"] and np.array_equal(again["root_q"], r["root_q"])


def test_one_step_horizon_means():
    """D = 1: simulation i takes action i mod |A| in the first round (virtual
    visits, lowest index on ties) and scenario i mod n; below depth 1 the
    value is 0, so Q(a) is the mean step reward of those pairs."""
    cfg = I.rs7_8().with_(D=1)
    om = oracle.Model(cfg)
    n = 10
    b = I.rs_block(cfg, n, np.random.default_rng(2), pos=[(2, 3)])
    na = om.num_actions()
    B = 4 * na
    r = om.pomcp(b, None, rounds=1, batch=B, c=1.0)
    sims = np.arange(B)
    acts = (sims % na).astype(np.int32)
    parts = sims % n
    _, _, rew = om.step(b[:, parts], acts, 0)
    for a in range(na):
        sel = acts == a
        q = 0.0
        for k, rr in enumerate(rew[sel]):
            q += (rr - q) / (k + 1)
        assert r["root_q"][a] == q, (a, r["root_q"][a], q)


def test_approaches_the_exhaustive_optimum_from_below():
    """On a tiny task the root value (a running mean of returns, so it lags
    the optimum) rises with the simulation count and stays below the optimum
    of the exhaustive scenario tree over the same scenarios."""
    cfg = tiny()
    om = oracle.Model(cfg, fp64=True)
    b = I.rs_block(cfg, cfg.K, np.random.default_rng(4), pos=[(0, 1), (0, 0)])
    vstar = om.exhaustive(b, None, 0)
    short = om.pomcp(b, None, rounds=100, batch=48, c=50.0)
    long = om.pomcp(b, None, rounds=2000, batch=48, c=50.0)
    assert short["value"] < long["value"] <= vstar + 1e-9, (short["value"], long["value"], vstar)
    assert long["value"] > 0.5 * vstar
