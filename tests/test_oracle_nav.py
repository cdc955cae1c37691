"""Pins of the navigation oracle (Sec. IV-A, "Navigation in a Partially-Known
Map") against facts fixed outside it: rewards and moves on hand-drawn maps
with the noise switched off, readings equal to the map's true neighbours,
the noise rates by counting, closed-form corridor values, the 8-connected
upper bound, the default policy's preference order, and the partition
invariants of an expansion."""
import numpy as np

import oracle
from paper_1802_06215_b300 import inputs as I

N = 13
DIRS = [(0, 0), (0, -1), (1, -1), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1)]  # stay, N, NE, ..., NW


def cfg(fail_p=0.0, sense_p=0.0, D=90, gamma=0.95):
    return I.nav_config(N, K=64, D=D).with_(fail_p=fail_p, sense_p=sense_p, gamma=gamma)


def block_of(cells_list, pos_list, scen=None, term=None):
    """State block from boolean maps [y, x] and robot positions (x, y)."""
    count = len(cells_list)
    mw = (N * N + 31) // 32
    b = np.zeros((2 + mw, count), np.uint32)
    for i, (cells, (x, y)) in enumerate(zip(cells_list, pos_list)):
        flat = np.asarray(cells, bool).reshape(-1)
        for c in np.nonzero(flat)[0]:
            b[1 + c // 32, i] |= np.uint32(1) << np.uint32(c % 32)
        b[0, i] = x | (y << 8) | ((1 if (term and term[i]) else 0) << 16)
        b[1 + mw, i] = i if scen is None else scen[i]
    return b


def pos_of(b, i):
    return int(b[0, i] & 0xFF), int((b[0, i] >> 8) & 0xFF), bool((b[0, i] >> 16) & 1)


def true_reading(cells, x, y):
    z = 0
    for k in range(1, 9):
        nx, ny = x + DIRS[k][0], y + DIRS[k][1]
        occ = not (0 <= nx < N and 0 <= ny < N) or bool(cells[ny, nx])
        z |= int(occ) << (k - 1)
    return z


def empty_map():
    return np.zeros((N, N), bool)


def test_moves_rewards_and_readings_without_noise():
    om = oracle.Model(cfg())
    cells = empty_map()
    cells[5, 6] = True  # an obstacle right below (6, 4)
    cases = []  # (position, action, expected position, reward, terminal)
    cases.append(((6, 4), 0, (6, 4), -0.2, False))   # stay
    cases.append(((6, 4), 5, (6, 4), -1.0, False))   # S into the obstacle: crash, stays
    cases.append(((6, 4), 3, (7, 4), -0.1, False))   # E: free
    cases.append(((0, 0), 1, (0, 0), -1.0, False))   # N off the map
    cases.append(((0, 0), 8, (0, 0), -1.0, False))   # NW off the map
    cases.append(((12, 12), 4, (12, 12), -1.0, False))  # SE off the map
    cases.append(((5, 11), 4, (6, 12), 20.0, True))  # SE into the goal
    cases.append(((6, 11), 5, (6, 12), 20.0, True))  # S into the goal
    cases.append(((3, 3), 6, (2, 4), -0.1, False))   # SW
    b = block_of([cells] * len(cases), [c[0] for c in cases])
    acts = np.array([c[1] for c in cases], np.int32)
    out, keys, rew = om.step(b, acts, 3)
    for i, (p, a, q, r, term) in enumerate(cases):
        x, y, t = pos_of(out, i)
        assert (x, y) == q and t == term, (i, p, a)
        assert rew[i] == np.float32(r), (i, rew[i])
        if term:
            assert keys[i] == 1 << 62
        else:
            assert keys[i] == true_reading(cells, x, y), (i, hex(int(keys[i])))
    # the map never changes
    assert np.array_equal(out[1:-1], b[1:-1])


def test_terminal_scenarios_stay():
    om = oracle.Model(cfg())
    b = block_of([empty_map()], [(6, 12)], term=[True])
    out, keys, rew = om.step(b, np.array([5], np.int32), 0)
    assert np.array_equal(out, b) and keys[0] == 1 << 62 and rew[0] == 0.0


def test_move_failure_and_reading_noise_rates():
    """fail_p = 1: every move fails (-0.1, stays). sense_p = 1: every reading
    is the complement of the truth. sense_p = 0.25: the flip rate of 8 x 4000
    readings is 0.25 within 4 sigma."""
    cells = empty_map()
    rng = np.random.default_rng(0)
    cells[rng.random((N, N)) < 0.3] = True
    pos = [(int(x), 3) for x in rng.integers(0, N, 4000)]
    cells[3, :] = False  # the robots' row is free
    b = block_of([cells] * len(pos), pos)
    acts = np.full(len(pos), 5, np.int32)
    out, keys, rew = oracle.Model(cfg(fail_p=1.0)).step(b, acts, 7)
    assert np.all(rew == np.float32(-0.1)) and np.array_equal(out[0], b[0])
    truth = np.array([true_reading(cells, x, y) for (x, y) in pos])
    _, keys, _ = oracle.Model(cfg(sense_p=1.0)).step(b, np.zeros(len(pos), np.int32), 7)
    assert np.array_equal(keys.astype(np.int64), truth ^ 0xFF)
    _, keys, _ = oracle.Model(cfg(sense_p=0.25)).step(b, np.zeros(len(pos), np.int32), 7)
    flips = np.unpackbits((keys.astype(np.int64) ^ truth).astype(np.uint8)).sum()
    total = 8 * len(pos)
    assert abs(flips / total - 0.25) < 4 * np.sqrt(0.25 * 0.75 / total)


def test_corridor_rollout_closed_form():
    """No noise, free map, robot k rows straight above the goal below the wall:
    the default policy walks S, k moves, the last one into the goal:
    v = sum_{t<k-1} gamma^t (-0.1) + gamma^(k-1) 20 (FP32, in time order)."""
    c = cfg()
    om = oracle.Model(c)
    g32, _ = oracle.gamma_powers(c.gamma, 256)
    for k in (1, 2, 5):
        b = block_of([empty_map()], [(N // 2, N - 1 - k)])
        vals, steps = om.rollout(b, None, 0)
        v = np.float32(0)
        for t in range(k - 1):
            v = np.float32(v + np.float32(g32[t] * np.float32(-0.1)))
        v = np.float32(v + np.float32(g32[k - 1] * np.float32(20.0)))
        assert vals[0] == v and steps == k, (k, vals[0], v)


def test_horizon_truncates_with_zero_tail():
    c = cfg(D=3)
    om = oracle.Model(c)
    g32, _ = oracle.gamma_powers(c.gamma, 256)
    b = block_of([empty_map()], [(N // 2, N - 1 - 6)])
    vals, steps = om.rollout(b, None, 0)
    expect = np.float32(0)
    for t in range(3):
        expect = np.float32(expect + np.float32(g32[t] * np.float32(-0.1)))
    assert vals[0] == expect and steps == 3


def test_upper_bound_is_the_gated_chebyshev_distance():
    c = cfg()
    om = oracle.Model(c)
    g32, _ = oracle.gamma_powers(c.gamma, 256)
    wall, gates, goal = N // 2, (N // 4, N - 1 - N // 4), (N // 2, N - 1)
    rng = np.random.default_rng(1)
    maps, pos = [], []
    for _ in range(200):
        cells = empty_map()
        open_g = int(rng.integers(0, 2))
        cells[wall, :] = True
        cells[wall, gates[open_g]] = False
        x, y = int(rng.integers(0, N)), int(rng.integers(0, N - 1))
        if y == wall:
            x = gates[open_g]
        maps.append(cells)
        pos.append((x, y))
    b = block_of(maps, pos)
    u, t = om.bounds(b)
    for i, ((x, y), cells) in enumerate(zip(pos, maps)):
        gx = gates[0] if not cells[wall, gates[0]] else gates[1]
        cheb = lambda a, b: max(abs(a[0] - b[0]), abs(a[1] - b[1]))
        d = cheb((x, y), (gx, wall)) + cheb((gx, wall), goal) if y < wall else cheb((x, y), goal)
        assert u[i] == np.float32(np.float32(20.0) * g32[d - 1]), (i, x, y, d)
        assert t[i] == 0.0
    # admissible on the no-noise corridor: u >= the rollout's value
    cb = block_of([empty_map()], [(N // 2, N - 4)])
    uu, _ = om.bounds(cb)
    vv, _ = om.rollout(cb, None, 0)
    assert uu[0] >= vv[0]


def test_default_policy_preference_order():
    """The first of S, SE, SW, E, W, NE, NW, N whose last reading was free;
    stay when all eight read occupied."""
    om = oracle.Model(cfg())
    order = [5, 4, 6, 3, 7, 2, 8, 1]
    lasts = list(range(256))
    b = block_of([empty_map()] * 256, [(6, 6)] * 256)
    h = np.zeros((256, 32), np.int8)
    h[:, 0] = np.array(lasts, np.uint8).view(np.int8)
    acts = om.policy(b, h)
    for z, a in zip(lasts, acts):
        want = next((d for d in order if not (z >> (d - 1)) & 1), 0)
        assert a == want, (z, a, want)


def test_expansion_partitions_scenarios():
    c = I.nav13()
    om = oracle.Model(c)
    jobs = I.job_stream(c, 4, 5, max_scen=60)
    for j in jobs:
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=len(j.idx))
        n = len(j.idx)
        for a in range(9):
            nc = int(o["child_count"][a])
            off = o["child_off"][a][: nc + 1]
            assert off[0] == 0 and off[-1] == n and np.all(np.diff(off) > 0)
            assert sorted(o["perm"][a].tolist()) == list(range(n))
            keys = o["key"][a][:nc]
            assert len(set(keys.tolist())) == nc
