"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test ties an oracle function to a value the paper or mathematics fixes:
hand-derived transition tables (tests/golden), closed-form discounted returns,
the sensor law 0.5 + 0.5 * 2^(-d/20), an independent inverse-normal routine,
invariants of leaf expansion (Sec. III-D), the bracket l0 <= V*_D <= u0 from
exhaustive expansion, and convergence of the search to V*_D.
"""
import os

import numpy as np
import pytest
from scipy.special import ndtri

import oracle
from paper_1802_06215_b300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G32 = float(np.float32(0.95))


def rs3(robots=1, K=8, D=5, m=2):
    cfg = I.Config(kind=I.GRID if robots == 1 else I.MULTIGRID, n=3, m=m, K=K, D=D, seed=7,
                   rock_cells=np.array([1 | (1 << 8), 2 | (0 << 8)][:m], np.int32))
    return cfg


def block_rs(states, robots=1):
    """states: list of (robots list of (x, y, exited), good, sampled, scen)."""
    b = np.zeros((5, len(states)), np.uint32)
    for i, (rb, good, samp, scen) in enumerate(states):
        for r, (x, y, e) in enumerate(rb):
            b[r, i] = x | (y << 8) | (e << 16)
        b[2, i], b[3, i], b[4, i] = good, samp, scen
    return b


# ------------------------------------------------------------------ Philox --

def test_philox_round_structure():
    """One and two rounds against the published round (Salmon et al. SC'11,
    Sec. 3.3) evaluated with Python integers."""
    M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85
    rng = np.random.default_rng(3)
    for _ in range(50):
        c = [int(x) for x in rng.integers(0, 2**32, 4)]
        k0, k1 = (int(x) for x in rng.integers(0, 2**32, 2))

        def rnd(c, k0, k1):
            p0, p1 = M0 * c[0], M1 * c[2]
            return [(p1 >> 32) ^ c[1] ^ k0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ c[3] ^ k1, p0 & 0xFFFFFFFF]

        one = rnd(c, k0, k1)
        two = rnd(one, (k0 + W0) & 0xFFFFFFFF, (k1 + W1) & 0xFFFFFFFF)
        assert list(oracle.philox(c, k0, k1, 1)) == one
        assert list(oracle.philox(c, k0, k1, 2)) == two


def _avalanche(rounds, n=400):
    rng = np.random.default_rng(11)
    flips = []
    for _ in range(n):
        c = rng.integers(0, 2**32, 4).astype(np.uint32)
        bit = int(rng.integers(0, 128))
        c2 = c.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        a = oracle.philox(c, 5, 9, rounds)
        b = oracle.philox(c2, 5, 9, rounds)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)) / 128.0)
    return float(np.mean(flips)), float(np.min(flips))


def test_philox_avalanche_needs_rounds():
    """Ten rounds flip about half of the 128 output bits for any one-bit counter
    change; a single round does not. Catches dropped rounds or key schedule."""
    mean10, min10 = _avalanche(10)
    mean1, _ = _avalanche(1)
    assert 0.47 < mean10 < 0.53 and min10 > 0.3
    assert mean1 < 0.4


def test_philox_uniform_and_distinct():
    """Sequential counters give distinct, uniform words (chi-square on bytes,
    per-bit balance within 5 sigma)."""
    n = 1 << 14
    out = np.zeros((n, 4), np.uint32)
    for i in range(n):
        out[i] = oracle.scenario_random(0xDEADBEEF12345678, i, 3, 2, 0, 1)
    words = out.reshape(-1)
    assert len(np.unique(out.view(np.dtype((np.void, 16))))) == n
    by = words.view(np.uint8)
    hist = np.bincount(by, minlength=256)
    exp = len(by) / 256.0
    chi2 = float(((hist - exp) ** 2 / exp).sum())
    assert chi2 < 255 + 5 * np.sqrt(2 * 255)
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(len(words)))


def test_streams_differ_by_each_counter_field():
    base = oracle.scenario_random(1, 2, 3, 2, 1, 4)
    for args in [(2, 2, 3, 2, 1, 4), (1, 3, 3, 2, 1, 4), (1, 2, 4, 2, 1, 4), (1, 2, 3, 1, 1, 4),
                 (1, 2, 3, 2, 0, 4), (1, 2, 3, 2, 1, 5)]:
        assert not np.array_equal(oracle.scenario_random(*args), base)


# ------------------------------------------------------------------ tables --

def test_sensor_thresholds_closed_form():
    """Accuracy 0.5 + 0.5 * 2^(-d/20): exactly 1 at d = 0, 3/4 at d = 20 and
    5/8 at d = 40 (d^2 = 400, 1600)."""
    t = oracle.sensor_thresholds(1600)
    assert int(t[0]) == 2**32
    assert int(t[400]) == 3 * 2**30
    assert int(t[1600]) == 5 * 2**29
    assert np.all(np.diff(t.astype(np.float64)) <= 0)
    assert np.all(t >= 2**31)


def test_gamma_powers():
    g32, g64 = oracle.gamma_powers(0.95, 100)
    assert g32[0] == 1.0 and g64[0] == 1.0
    assert g64[1] == G32
    assert abs(g64[50] - G32 ** 50) < 1e-15
    assert np.all(np.abs(g32.astype(np.float64) - g64) <= np.abs(g64) * 2 ** -24)


def test_gauss_table_against_independent_inverse():
    """Inverse-normal quantiles (i + 0.5)/4096 against scipy's ndtri."""
    t64, t32 = oracle.gauss_table()
    ref = ndtri((np.arange(4096) + 0.5) / 4096.0)
    assert np.max(np.abs(t64 - ref)) < 1e-12
    assert np.array_equal(t32, t64.astype(np.float32))
    assert np.all(np.diff(t64) > 0)
    assert np.max(np.abs(t64 + t64[::-1])) < 1e-12


# ------------------------------------------------------------------ models --

def _load_fixture(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            lhs, rhs = line.split("|")
            rows.append(([int(x) for x in lhs.split()], [int(x) for x in rhs.split()]))
    return rows


def test_rs_transitions_golden():
    cfg = rs3()
    m = oracle.Model(cfg)
    for lhs, rhs in _load_fixture("rs3x3_transitions.txt"):
        x, y, e, good, samp, a = lhs
        b = block_rs([([(x, y, e)], good, samp, 0)])
        out, key, rew = m.step(b, [a], 0)
        x2, y2, e2, g2, s2, r, z = rhs
        exp = block_rs([([(x2, y2, e2)], g2, s2, 0)])
        assert np.array_equal(out, exp), (lhs, out[:, 0], exp[:, 0])
        assert rew[0] == r, lhs
        assert int(key[0]) & 0x3 == z, lhs
        assert bool(int(key[0]) >> 62 & 1) == bool(e2), lhs


def test_mars_transitions_golden():
    cfg = rs3(robots=2)
    m = oracle.Model(cfg)
    for lhs, rhs in _load_fixture("mars3x3_transitions.txt"):
        x0, y0, e0, x1, y1, e1, good, samp, a0, a1 = lhs
        b = block_rs([([(x0, y0, e0), (x1, y1, e1)], good, samp, 0)], robots=2)
        out, key, rew = m.step(b, [a0 * 7 + a1], 0)
        X0, Y0, E0, X1, Y1, E1, G, S, r, z0, z1, term = rhs
        exp = block_rs([([(X0, Y0, E0), (X1, Y1, E1)], G, S, 0)], robots=2)
        assert np.array_equal(out, exp), lhs
        assert rew[0] == r, lhs
        k = int(key[0])
        assert (k & ~(1 << 62)) == z0 * 3 + z1, lhs
        assert bool(k >> 62 & 1) == bool(term), lhs


@pytest.mark.parametrize("d2", [1, 25, 100, 400])
def test_sensor_frequency(d2):
    """Empirical accuracy of Sense over 10^6 scenarios within 4 sigma of
    0.5 + 0.5 * 2^(-d/20) (Sec. IV-A: accuracy decays exponentially)."""
    cfg = I.Config(kind=I.GRID, n=30, m=1, K=10**6, D=5, seed=123,
                   rock_cells=np.array([0], np.int32))
    m = oracle.Model(cfg)
    N = 10**6
    # robot placed so that squared distance to the rock at (0,0) is d2
    dx = {1: (1, 0), 25: (3, 4), 100: (6, 8), 400: (12, 16)}[d2]
    b = np.zeros((5, N), np.uint32)
    b[0] = dx[0] | (dx[1] << 8)
    b[2] = np.arange(N, dtype=np.uint32) & 1  # half the rocks good
    b[4] = np.arange(N, dtype=np.uint32)
    out, key, rew = m.step(b, np.full(N, 5, np.int32), 2)
    z = (key & np.uint64(3)).astype(np.int64)
    correct = np.where(b[2] == 1, z == 1, z == 2)
    p = 0.5 + 0.5 * 2 ** (-np.sqrt(d2) / 20)
    assert abs(correct.mean() - p) < 4 * np.sqrt(p * (1 - p) / N)


def test_rollout_closed_form_east():
    """With no rock believed good the default policy walks east: the value from
    column x at depth t0 is 10 * gamma^(n-1-x) (reward +10 on the exit step)."""
    for fp64 in (False, True):
        cfg = I.rs15_15()
        m = oracle.Model(cfg, fp64=fp64)
        rng = np.random.default_rng(0)
        for x in range(15):
            b = I.rs_block(cfg, 4, rng, pos=[(x, 3)])
            v, steps = m.rollout(b, None, 10)
            exact = 10 * G32 ** (14 - x)
            tol = 1e-12 if fp64 else 1e-6
            assert np.all(np.abs(v - exact) <= tol * exact), (x, v, exact)
            assert steps == 4 * (15 - x)


def test_rollout_closed_form_sample_then_exit():
    """A rock believed good under the robot: Sample (+10 if good, -10 if bad),
    then walk east from column x: 10 * gamma^(n-x) more."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg, fp64=True)
    cell = int(cfg.rock_cells[0])
    x, y = cell & 0xFF, cell >> 8
    b = np.zeros((5, 2), np.uint32)
    b[0] = x | (y << 8)
    b[2] = [1, 0]
    b[4] = [0, 1]
    h = np.zeros((2, 32), np.int8)
    h[:, 0] = 1
    v, _ = m.rollout(b, h, 0)
    tail = 10 * G32 ** (15 - x)
    assert abs(v[0] - (10 + tail)) < 1e-9
    assert abs(v[1] - (-10 + tail)) < 1e-9


def test_horizon_truncation_uses_tail():
    """At depth D the rollout stops and adds gamma^(D-t0) times the tail
    heuristic 10 * gamma^(n-1-x); from depth D itself the value is the tail."""
    cfg = I.rs15_15().with_(D=12)
    m = oracle.Model(cfg, fp64=True)
    rng = np.random.default_rng(2)
    b = I.rs_block(cfg, 3, rng, pos=[(0, 5)])
    v, steps = m.rollout(b, None, 12)
    assert steps == 0 and np.allclose(v, 10 * G32 ** 14, rtol=1e-12)
    v, steps = m.rollout(b, None, 10)
    # two steps east from x = 0 reach x = 2, tail 10 gamma^12 discounted by gamma^2
    assert steps == 6 and np.allclose(v, G32 ** 2 * 10 * G32 ** 12, rtol=1e-12)


def test_car_closed_form_goal():
    """Car alone (pedestrian parked far away, no action failure): from s = 55,
    v = 3 the default policy keeps 3 m/s and passes 60 m on the 6th step
    (55 + 6 * 0.99 >= 60 > 55 + 5 * 0.99), worth 1000 * gamma^5; the upper bound
    (accelerate every step) gives the same value."""
    for fp64 in (False, True):
        cfg = I.car_config(P=1, K=4, D=50).with_(fail_p=0.0, sigma=0.0)
        m = oracle.Model(cfg, fp64=fp64)
        b = np.zeros((I.words(cfg), 1), np.uint32)
        b[0] = np.float32(55.0).view(np.uint32)
        b[1] = 3
        b[4] = np.float32(40.0).view(np.uint32)  # pedestrian at its goal corner (40, 40)
        b[5] = np.float32(40.0).view(np.uint32)
        b[6] = 3
        v, steps = m.rollout(b, None, 0)
        u, _ = m.bounds(b)
        exact = 1000 * G32 ** 5
        assert steps == 6
        assert abs(v[0] - exact) < 1e-3 and abs(u[0] - exact) < 1e-3


def test_car_pedestrian_noise_moments():
    """One step of a lone pedestrian: mean displacement = 1.2 m/s * 0.33 s toward
    the goal, per-axis standard deviation sigma = 0.1 (sample of 20000)."""
    cfg = I.car_config(P=1, K=20000, D=50)
    m = oracle.Model(cfg, fp64=True)
    N = 20000
    b = np.zeros((I.words(cfg), N), np.uint32)
    b[0] = np.float32(0.0).view(np.uint32)
    b[2] = np.arange(N)
    b[4] = np.float32(10.0).view(np.uint32)
    b[5] = np.float32(10.0).view(np.uint32)
    b[6] = 0  # goal (0, 0): heading (-1, -1)/sqrt(2)
    out, key, rew = m.step(b, np.ones(N, np.int32), 1)
    px = out[4].view(np.float32).astype(np.float64)
    py = out[5].view(np.float32).astype(np.float64)
    stride = float(np.float32(1.2)) * float(np.float32(0.33)) / np.sqrt(2)
    assert abs(px.mean() - (10 - stride)) < 4 * 0.1 / np.sqrt(N)
    assert abs(py.mean() - (10 - stride)) < 4 * 0.1 / np.sqrt(N)
    assert abs(px.std() - 0.1) < 0.005 and abs(py.std() - 0.1) < 0.005


def test_car_fp32_matches_fp64():
    """The FP32 oracle against the FP64 one: rollout values within 1e-4
    relative (or 1e-3 absolute) wherever both took the same discrete path."""
    cfg = I.car_config(P=50, K=64, D=50)
    m32 = oracle.Model(cfg)
    m64 = oracle.Model(cfg, fp64=True)
    rng = np.random.default_rng(5)
    b = I.car_block(cfg, 64, rng)
    v32, s32 = m32.rollout(b, None, 3)
    v64, s64 = m64.rollout(b, None, 3)
    close = np.abs(v32 - v64) <= np.maximum(1e-4 * np.abs(v64), 1e-3)
    assert close.mean() >= 0.95
    out32, k32, r32 = m32.step(b, np.zeros(64, np.int32), 3)
    out64, k64, r64 = m64.step(b, np.zeros(64, np.int32), 3)
    p32 = out32[4:54].view(np.float32).astype(np.float64)
    p64 = out64[4:54].view(np.float32).astype(np.float64)
    assert np.max(np.abs(p32 - p64)) < 1e-4


# -------------------------------------------------------------- expansion --

def _check_partition(e, keys_fn=None):
    na, n = e["perm"].shape
    for a in range(na):
        nc = e["child_count"][a]
        off = e["child_off"][a]
        assert off[0] == 0 and off[nc] == n
        perm = e["perm"][a]
        assert sorted(perm.tolist()) == list(range(n))
        firsts = []
        for c in range(nc):
            mem = perm[off[c]:off[c + 1]]
            assert len(mem) > 0 and np.all(np.diff(mem.astype(int)) > 0)
            firsts.append(int(mem[0]))
        assert firsts == sorted(firsts)


def test_expansion_partition_and_weights():
    """Children of each action partition Phi_b (Eq. newnodes); child order is by
    first occurrence; weights n_c/K sum to |Phi_b|/K."""
    for cfg in (I.rs15_15(), I.grid_config(7, 8, K=100), I.car_config(P=10, K=40, D=20)):
        m = oracle.Model(cfg)
        for j in I.job_stream(cfg, 6, 1, max_scen=40):
            e = m.expand(j.parent, j.idx, j.last_action, j.depth, j.hist)
            _check_partition(e)
            for a in range(len(e["child_count"])):
                nc = e["child_count"][a]
                w = np.diff(e["child_off"][a][:nc + 1]) / cfg.K
                assert abs(w.sum() - len(j.idx) / cfg.K) < 1e-12


def test_children_uniform_in_observation():
    """Every member of a child has the child's observation (Eq. newnodes)."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg)
    for j in I.job_stream(cfg, 4, 2, max_scen=60):
        e = m.expand(j.parent, j.idx, j.last_action, j.depth, j.hist)
        leaf = e["leaf"]
        for a in range(len(e["child_count"])):
            _, keys, _ = m.step(leaf, np.full(leaf.shape[1], a, np.int32), j.depth)
            for c in range(e["child_count"][a]):
                o = e["child_off"][a]
                mem = e["perm"][a][o[c]:o[c + 1]]
                assert np.all(keys[mem] == e["key"][a][c])


def _q_bounds(e, K, gamma):
    na = len(e["child_count"])
    qu, ql = [], []
    for a in range(na):
        nc = e["child_count"][a]
        r = e["rew"][a][:nc].sum() / 2**32 / K
        qu.append(r + gamma * (e["u"][a][:nc] / 2**32 / K).sum())
        ql.append(r + gamma * (e["l"][a][:nc] / 2**32 / K).sum())
    return np.array(qu), np.array(ql)


def test_upper_bound_consistent():
    """U(b, a) <= u0(b) for every action: the heuristic is consistent, so one
    level of Eq. backup never raises it (checked in FP64)."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg, fp64=True)
    for j in I.job_stream(cfg, 8, 3, max_scen=50):
        e = m.expand(j.parent, j.idx, j.last_action, j.depth, j.hist)
        u, _ = m.bounds(e["leaf"])
        u0 = u.sum() / cfg.K
        qu, _ = _q_bounds(e, cfg.K, G32)
        assert np.all(qu <= u0 * (1 + 1e-9) + 1e-9)


def test_lower_bound_is_policy_value():
    """L(b, pi0(b)) = l0(b): the default policy's own first action, backed up
    over its children's rollouts, equals the rollout value from b (grid
    policy is the same for every scenario of a node)."""
    cfg = I.rs15_15()
    m = oracle.Model(cfg, fp64=True)
    for j in I.job_stream(cfg, 8, 4, max_scen=50):
        e = m.expand(j.parent, j.idx, j.last_action, j.depth, j.hist)
        leaf = e["leaf"]
        n = leaf.shape[1]
        acts = m.policy(leaf, np.tile(j.hist, (n, 1)))
        assert np.all(acts == acts[0])
        v, _ = m.rollout(leaf, np.tile(j.hist, (n, 1)), j.depth)
        _, ql = _q_bounds(e, cfg.K, G32)
        assert abs(ql[acts[0]] - v.sum() / cfg.K) < 1e-7 * max(1, abs(v.sum() / cfg.K))


# ------------------------------------------------------- exhaustive/search --

def _tiny_root(cfg, K, rng):
    b = I.rs_block(cfg, K, rng, pos=[(0, 1), (0, 0)][: (2 if cfg.kind == I.MULTIGRID else 1)])
    return b


def test_exhaustive_closed_form():
    """2x2 map, a good rock under the robot at (0,0): sample (+10), then two
    steps east (+10 on the exit): V* = 10 + 10 gamma^2."""
    cfg = I.Config(kind=I.GRID, n=2, m=1, K=2, D=4, seed=0, rock_cells=np.array([0], np.int32))
    m = oracle.Model(cfg, fp64=True)
    b = block_rs([([(0, 0, 0)], 1, 0, 0), ([(0, 0, 0)], 1, 0, 1)])
    v = m.exhaustive(b, None, 0)
    assert abs(v - (10 + 10 * G32 ** 2)) < 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bounds_bracket_optimum(seed):
    """l0 <= V*_D <= u0 at the root of tiny instances (3x3, 2 rocks, K=6,
    D=4), with V*_D from exhaustive expansion of the scenario tree."""
    cfg = rs3(K=6, D=4).with_(seed=seed)
    m = oracle.Model(cfg, fp64=True)
    rng = np.random.default_rng(seed)
    b = _tiny_root(cfg, 6, rng)
    vstar = m.exhaustive(b, None, 0)
    u, _ = m.bounds(b)
    l, _ = m.rollout(b, None, 0)
    assert l.mean() <= vstar + 1e-9 <= u.mean() + 2e-9


@pytest.mark.parametrize("seed", [0, 1])
def test_search_converges_to_optimum(seed):
    """With xi = 0 the search expands every branch with a positive gap; at the
    end the root bounds meet at V*_D (Eq. backup over the whole tree)."""
    cfg = rs3(K=6, D=4).with_(seed=seed)
    m = oracle.Model(cfg, fp64=True)
    rng = np.random.default_rng(seed)
    b = _tiny_root(cfg, 6, rng)
    vstar = m.exhaustive(b, None, 0)
    r = m.plan(b, None, threads=1, rounds=100000, xi=0.0, target_gap=0.0)
    assert abs(r["root_u"] - vstar) < 1e-6 and abs(r["root_l"] - vstar) < 1e-6
    # the FP32 oracle's search brackets the same optimum
    r32 = oracle.Model(cfg).plan(b, None, threads=1, rounds=200, xi=0.95)
    assert r32["root_l"] <= vstar + 1e-5 and vstar <= r32["root_u"] + 1e-5


def test_search_bounds_valid_multithreaded_rounds():
    """Deterministic rounds with T = 4, PO-UCT and virtual loss still bracket
    V*_D and are reproducible."""
    cfg = rs3(K=6, D=4, robots=2)
    m = oracle.Model(cfg, fp64=True)
    b = _tiny_root(cfg, 6, np.random.default_rng(9))
    vstar = m.exhaustive(b, None, 0)
    r1 = m.plan(b, None, threads=4, rounds=30, c_a=1.0, c_o=0.5)
    r2 = m.plan(b, None, threads=4, rounds=30, c_a=1.0, c_o=0.5)
    assert r1["signature"] == r2["signature"]
    assert r1["root_l"] <= vstar + 1e-9 <= r1["root_u"] + 2e-9
