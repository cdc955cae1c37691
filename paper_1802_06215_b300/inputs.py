"""Seeded synthetic inputs shaped like the paper's tasks (Sec. IV-A).

This module only draws random numbers with numpy and lays them out in the state
block format; it holds none of the method's arithmetic (no step function, no
policy, no bounds). Tests feed the same arrays to the CUDA library and to the
CPU oracle; the benchmark uses it for its job streams.

State block format (the boundary's, see include/dsp.h): a uint32 array of shape
(words, capacity), field-major, scenario i of field f at [f, i].
  Rock Sample (5 words): f0/f1 robot r as x | y<<8 | exited<<16, f2 good-rock
  mask, f3 sampled-rock mask, f4 scenario id.
  Car (4 + 2P + ceil(P/4) words): f0 s (float bits), f1 v | terminal<<8,
  f2 scenario id, f3 zero, P words pedestrian x, P words y (float bits),
  goals four to a word.
  Navigation (2 + ceil(n*n/32) words): f0 x | y<<8 | terminal<<16, then the
  occupancy map (bit c of cell c = y*n + x), then the scenario id.
"""
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

GRID, MULTIGRID, CAR, NAV = 0, 1, 2, 3


@dataclass
class Config:
    kind: int
    n: int = 7
    m: int = 8
    P: int = 0
    gamma: float = 0.95
    K: int = 100
    D: int = 90
    seed: int = 0
    plan_step: int = 0
    rock_cells: Optional[np.ndarray] = None
    path_len: float = 60.0
    dt: float = 0.33
    ped_speed: float = 1.2
    sigma: float = 0.1
    fail_p: float = 0.01
    sense_p: float = 0.03

    def with_(self, **kw):
        return replace(self, **kw)


def rock_cells(n, m, seed):
    """m distinct cells of the n x n map (x | y << 8), drawn uniformly."""
    rng = np.random.default_rng([seed, 0x524F434B])
    cells = rng.choice(n * n, size=m, replace=False)
    xs, ys = cells % n, cells // n
    return (xs | (ys << 8)).astype(np.int32)


def grid_config(n=7, m=8, K=100, D=90, seed=0, robots=1):
    return Config(kind=GRID if robots == 1 else MULTIGRID, n=n, m=m, K=K, D=D, seed=seed,
                  rock_cells=rock_cells(n, m, seed))


def car_config(P=50, K=500, D=50, seed=0):
    return Config(kind=CAR, n=0, m=0, P=P, K=K, D=D, seed=seed, rock_cells=np.zeros(1, np.int32))


# The five workloads of the benchmark suite, by what they are.
def rs7_8():
    """7x7 map, 8 rocks, K=100, D=90 (one robot, 13 actions)."""
    return grid_config(7, 8, K=100, D=90, seed=0)


def rs15_15():
    """15x15 map, 15 rocks, K=500, D=90 (one robot, 20 actions)."""
    return grid_config(15, 15, K=500, D=90, seed=0)


def mars15_15():
    """Two robots on a 15x15 map with 15 rocks, 400 joint actions, K=500, D=90."""
    return grid_config(15, 15, K=500, D=90, seed=0, robots=2)


def car50():
    """Car among 50 pedestrians, K=500, D=50."""
    return car_config(P=50, K=500, D=50, seed=0)


# Variants of the same kernels (Sec. IV: crowd sizes, map sizes, numbers of
# scenarios).
def car_p(P):
    """Car among P pedestrians, K=500, D=50."""
    return car_config(P=P, K=500, D=50, seed=0)


def mars11_11():
    """Two robots on an 11x11 map with 11 rocks, 256 joint actions, K=500, D=90."""
    return grid_config(11, 11, K=500, D=90, seed=0, robots=2)


def mars20_20():
    """Two robots on a 20x20 map with 20 rocks, 625 joint actions, K=500, D=90."""
    return grid_config(20, 20, K=500, D=90, seed=0, robots=2)


def rs15_15_k(K):
    """rs15_15 with K scenarios (up to 8192 for one robot)."""
    return grid_config(15, 15, K=K, D=90, seed=0)


def nav_config(n=13, K=500, D=90, seed=0):
    """Navigation in a partially known n x n map: 9 actions, moves fail with
    p = 0.03, each of the 8 adjacent-cell readings is wrong with p = 0.03."""
    return Config(kind=NAV, n=n, m=0, P=0, K=K, D=D, seed=seed, rock_cells=np.zeros(1, np.int32), fail_p=0.03,
                  sense_p=0.03)


def nav13():
    """The paper's 13x13 navigation map, K=500, D=90."""
    return nav_config(13, K=500, D=90, seed=0)


def words(cfg):
    if cfg.kind in (GRID, MULTIGRID):
        return 5
    if cfg.kind == NAV:
        return 2 + (cfg.n * cfg.n + 31) // 32
    return 4 + 2 * cfg.P + (cfg.P + 3) // 4


def nav_layout(cfg):
    """The map's known cells: (free, occupied) boolean arrays of shape (n, n)
    indexed [y, x]. Start row y = 0 and the goal (n/2, n-1) are known free;
    the wall row y = n/2 is known occupied except its two gates (x = n/4 and
    n-1-n/4); 20 landmark cells (drawn once per world seed, off the start
    row, the wall row and the goal) are known occupied. Every other cell,
    the gates included, is unknown to the robot (124 of 169 on 13 x 13)."""
    n = cfg.n
    free = np.zeros((n, n), bool)
    occ = np.zeros((n, n), bool)
    free[0, :] = True
    free[n - 1, n // 2] = True
    wall = n // 2
    gates = (n // 4, n - 1 - n // 4)
    occ[wall, :] = True
    for g in gates:
        occ[wall, g] = False
    rng = np.random.default_rng([cfg.seed, 0x4E41564C])
    cand = [(y, x) for y in range(1, n) for x in range(n) if y != wall and not (y == n - 1 and x == n // 2)]
    for k in rng.choice(len(cand), size=min(20, len(cand)), replace=False):
        occ[cand[k]] = True
    return free, occ


def nav_maps(cfg, count, rng, p_occ=0.1):
    """Occupancy maps of `count` scenarios, uint32 words (ceil(n*n/32), count):
    known cells as the layout says, one gate open (uniform), the other unknown
    cells occupied with probability p_occ."""
    n = cfg.n
    free, occ = nav_layout(cfg)
    known = free | occ
    wall = n // 2
    gates = (n // 4, n - 1 - n // 4)
    cells = rng.random((count, n, n)) < p_occ
    cells = np.where(known[None], occ[None], cells)
    open_g = rng.integers(0, 2, count)
    cells[:, wall, gates[0]] = open_g != 0
    cells[:, wall, gates[1]] = open_g == 0
    flat = cells.reshape(count, n * n)
    mw = (n * n + 31) // 32
    out = np.zeros((mw, count), np.uint32)
    for c in range(n * n):
        out[c // 32] |= flat[:, c].astype(np.uint32) << np.uint32(c % 32)
    return out, cells


def nav_block(cfg, count, rng, pos=None, spread=0, scen=None, p_occ=0.1, maps=None):
    """Random navigation scenarios: a map per scenario (nav_maps), and the
    robot at `pos` (x, y), within `spread` cells of it (localisation
    uncertainty), or uniform on the start row; never on an occupied cell."""
    n = cfg.n
    words_map, cells = nav_maps(cfg, count, rng, p_occ) if maps is None else maps
    b = np.zeros((words(cfg), count), np.uint32)
    mw = (n * n + 31) // 32
    b[1:1 + mw] = words_map
    xs = np.zeros(count, np.int64)
    ys = np.zeros(count, np.int64)
    for i in range(count):
        for _ in range(64):
            if pos is None:
                x, y = int(rng.integers(0, n)), 0
            else:
                x = int(np.clip(pos[0] + rng.integers(-spread, spread + 1), 0, n - 1))
                y = int(np.clip(pos[1] + rng.integers(-spread, spread + 1), 0, n - 1))
            if not cells[i, y, x] and not (x == n // 2 and y == n - 1):
                break
        else:  # no free cell found near pos: the start row is free
            x, y = int(rng.integers(0, n)), 0
        xs[i], ys[i] = x, y
    b[0] = (xs.astype(np.uint32) | (ys.astype(np.uint32) << 8))
    b[1 + mw] = (np.arange(count) if scen is None else scen).astype(np.uint32)
    return b


def _f32_bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def rs_block(cfg, count, rng, pos=None, sampled=None, scen=None, p_good=0.5, exited=None):
    """Random Rock Sample scenarios. Positions, sampled masks and exit flags may
    be shared (scalars) or per scenario; good masks are independent draws."""
    robots = 2 if cfg.kind == MULTIGRID else 1
    b = np.zeros((5, count), np.uint32)
    for r in range(robots):
        if pos is None:
            x = rng.integers(0, cfg.n, count)
            y = rng.integers(0, cfg.n, count)
        else:
            x = np.full(count, pos[r][0])
            y = np.full(count, pos[r][1])
        ex = np.zeros(count, np.uint32) if exited is None else np.full(count, exited[r], np.uint32)
        b[r] = (x.astype(np.uint32) | (y.astype(np.uint32) << 8) | (ex << 16))
    good = np.zeros(count, np.uint32)
    for i in range(cfg.m):
        good |= (rng.random(count) < p_good).astype(np.uint32) << np.uint32(i)
    samp = np.zeros(count, np.uint32) if sampled is None else np.full(count, sampled, np.uint32)
    b[2] = good & ~samp
    b[3] = samp
    b[4] = (np.arange(count) if scen is None else scen).astype(np.uint32)
    return b


def car_block(cfg, count, rng, s=None, v=None, base=None, jitter=0.0, scen=None):
    """Random car scenarios: pedestrians uniform on [0,40]^2 (or a shared base
    layout plus Gaussian jitter), hidden goals uniform over the four corners."""
    P = cfg.P
    b = np.zeros((words(cfg), count), np.uint32)
    ss = rng.uniform(0.0, 20.0, count) if s is None else np.full(count, s)
    vv = rng.integers(0, 4, count) if v is None else np.full(count, v)
    b[0] = _f32_bits(ss)
    b[1] = vv.astype(np.uint32)
    b[2] = (np.arange(count) if scen is None else scen).astype(np.uint32)
    if base is None:
        px = rng.uniform(0.0, 40.0, (P, count))
        py = rng.uniform(0.0, 40.0, (P, count))
    else:
        px = base[0][:, None] + jitter * rng.standard_normal((P, count))
        py = base[1][:, None] + jitter * rng.standard_normal((P, count))
    b[4:4 + P] = _f32_bits(px)
    b[4 + P:4 + 2 * P] = _f32_bits(py)
    goals = rng.integers(0, 4, (P, count)).astype(np.uint32)
    for w in range((P + 3) // 4):
        acc = np.zeros(count, np.uint32)
        for k in range(4):
            j = 4 * w + k
            if j < P:
                acc |= goals[j] << np.uint32(8 * k)
        b[4 + 2 * P + w] = acc
    return b


def random_hist(cfg, rng, senses):
    """Per-rock belief counters of a random history with `senses` readings."""
    h = np.zeros(32, np.int8)
    for _ in range(senses):
        i = rng.integers(0, max(cfg.m, 1))
        h[i] = np.clip(int(h[i]) + (1 if rng.random() < 0.6 else -1), -127, 127)
    return h


@dataclass
class Job:
    parent: np.ndarray        # (words, parent_count) state block of the parent
    idx: np.ndarray           # uint16 positions of the leaf's scenarios in the parent
    last_action: int          # -1 when the parent block already is the leaf (a root)
    depth: int                # depth of the leaf
    hist: np.ndarray          # int8[32] belief counters of the leaf's history
    first_action: int = 0
    n_actions: int = 0


def _num_actions(cfg):
    if cfg.kind == CAR:
        return 3
    if cfg.kind == NAV:
        return 9
    a = 5 + cfg.m
    return a if cfg.kind == GRID else a * a


def job_stream(cfg, n_jobs, seed, max_scen=None, depth_max=10, min_scen=1):
    """Leaf-expansion jobs with depth ~ U{0..depth_max} and |Phi_b| ~ U{min..max}.

    Rock Sample: every scenario of a job shares the robot positions, the
    sampled mask and the history (as in a real tree node); good masks differ.
    Car: pedestrians share a base layout with per-scenario jitter, goals differ.
    The last action never leaves the map, so leaves are live."""
    rng = np.random.default_rng([seed, 0x4A4F4253])
    K = cfg.K
    max_scen = K if max_scen is None else max_scen
    na = _num_actions(cfg)
    jobs = []
    for _ in range(n_jobs):
        n = int(rng.integers(min_scen, max_scen + 1))
        depth = int(rng.integers(0, depth_max + 1))
        extra = int(rng.integers(0, n + 1)) if depth > 0 else 0
        pc = min(n + extra, K)
        scen = np.sort(rng.choice(K, size=pc, replace=False)).astype(np.uint32)
        if cfg.kind in (GRID, MULTIGRID):
            robots = 2 if cfg.kind == MULTIGRID else 1
            pos = [(int(rng.integers(0, cfg.n - 1)), int(rng.integers(0, cfg.n))) for _ in range(robots)]
            nsamp = int(rng.integers(0, min(cfg.m, depth // 3 + 1) + 1))
            sampled = 0
            for i in rng.choice(cfg.m, size=nsamp, replace=False):
                sampled |= 1 << int(i)
            parent = rs_block(cfg, pc, rng, pos=pos, sampled=sampled, scen=scen)
            hist = random_hist(cfg, rng, depth)
            if depth > 0:
                per = 5 + cfg.m
                while True:
                    a = int(rng.integers(0, na))
                    if robots == 1:
                        ok = not (a == 1 and pos[0][0] == cfg.n - 1)
                    else:
                        ok = not ((a // per == 1 and pos[0][0] == cfg.n - 1) or (a % per == 1 and pos[1][0] == cfg.n - 1))
                    if ok:
                        break
                last = a
            else:
                last = -1
        elif cfg.kind == NAV:
            # a tree node's scenarios: one map each, the robot within a cell of
            # a common position (localisation uncertainty grows with depth)
            y0 = int(rng.integers(0, min(cfg.n - 1, depth + 1)))
            x0 = int(rng.integers(0, cfg.n))
            parent = nav_block(cfg, pc, rng, pos=(x0, y0), spread=1 if depth > 0 else 0, scen=scen)
            hist = np.zeros(32, np.int8)
            if depth > 0:
                hist[0] = np.array([rng.integers(0, 256)], np.uint8).view(np.int8)[0]
            last = int(rng.integers(0, 9)) if depth > 0 else -1
        else:
            s0 = float(rng.uniform(0.0, 20.0))
            v0 = int(rng.integers(0, 4))
            base = (rng.uniform(0.0, 40.0, cfg.P), rng.uniform(0.0, 40.0, cfg.P))
            parent = car_block(cfg, pc, rng, s=s0, v=v0, base=base, jitter=0.1 * np.sqrt(depth + 1), scen=scen)
            hist = np.zeros(32, np.int8)
            last = int(rng.integers(0, 3)) if depth > 0 else -1
        idx = np.sort(rng.choice(pc, size=n, replace=False)).astype(np.uint16)
        if depth == 0:
            idx = np.arange(n, dtype=np.uint16)
        jobs.append(Job(parent=parent, idx=idx, last_action=last, depth=depth, hist=hist, first_action=0,
                        n_actions=na))
    return jobs
