"""GPU vs CPU oracle, Rock Sample models: bit-exact (integer states, keys,
grouping, fixed-point sums of FP32 values computed in the same order)."""
import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import batch, build
    build.build()
    return batch


def rs32_32():
    """The largest map: 32x32 with 32 rocks, whose 64 KB policy-key table
    needs the rollout kernels' opt-in shared memory."""
    return I.grid_config(32, 32, K=100, D=120, seed=3)


def mars11_11():
    """Two robots, 11x11 and 11 rocks: 256 joint actions (K = 200 keeps the
    oracle quick)."""
    return I.grid_config(11, 11, K=200, D=90, seed=0, robots=2)


def mars20_20():
    """Two robots, 20x20 and 20 rocks: 625 joint actions."""
    return I.grid_config(20, 20, K=200, D=90, seed=0, robots=2)


CONFIGS = {"rs7_8": I.rs7_8, "rs15_15": I.rs15_15, "mars15_15": I.mars15_15, "rs32_32": rs32_32,
           "mars11_11": mars11_11, "mars20_20": mars20_20}


def _cmp_expand(g, o, n, tag=""):
    na = len(o["child_count"])
    assert np.array_equal(g["leaf"], o["leaf"]), tag + " leaf states"
    assert np.array_equal(g["child_count"], o["child_count"]), tag + " child counts"
    for a in range(na):
        nc = int(o["child_count"][a])
        assert np.array_equal(g["child_off"][a][: nc + 1], o["child_off"][a][: nc + 1]), (tag, a, "off")
        assert np.array_equal(g["key"][a][:nc], o["key"][a][:nc]), (tag, a, "key")
        assert np.array_equal(g["rew"][a][:nc], o["rew"][a][:nc]), (tag, a, "rew")
        assert np.array_equal(g["u"][a][:nc], o["u"][a][:nc]), (tag, a, "u")
        assert np.array_equal(g["l"][a][:nc], o["l"][a][:nc]), (tag, a, "l")
    assert np.array_equal(g["perm"], o["perm"]), tag + " perm"


def test_tables_match_oracle(dsp):
    for name, mk in CONFIGS.items():
        cfg = mk()
        m = dsp.Model(cfg)
        t = m.table(0)
        assert np.array_equal(t, oracle.sensor_thresholds(len(t) - 1)), name
        g32, _ = oracle.gamma_powers(cfg.gamma, 256)
        assert np.array_equal(m.table(1), g32), name
        m.close()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_step_parity(dsp, name):
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(1)
    N = 4000
    b = I.rs_block(cfg, N, rng)
    b[2] &= ~b[3]
    # a few robots already out of the map
    b[0, :50] |= 1 << 16
    acts = rng.integers(0, m.num_actions, N).astype(np.int32)
    for depth in (0, 7, 89):
        go, gk, gr = m.step(b, acts, depth)
        oo, ok, orr = om.step(b, acts, depth)
        assert np.array_equal(go, oo)
        assert np.array_equal(gk, ok)
        assert np.array_equal(gr.astype(np.float64), orr)
    m.close()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_rollout_parity(dsp, name):
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(2)
    N = 3000
    b = I.rs_block(cfg, N, rng)
    b[2] &= ~b[3]
    hist = rng.integers(-2, 3, (N, 32)).astype(np.int8)
    for d0 in (0, 45, 88, cfg.D):
        gv = m.rollout(b, hist, d0)
        ov, _ = om.rollout(b, hist, d0)
        assert np.array_equal(gv.astype(np.float64), ov), d0
    m.close()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_expand_parity_ragged(dsp, name):
    """Ragged |Phi_b| (1..K, several units per job and several jobs per unit
    size), random depths, roots and updated leaves."""
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    njobs = 24 if cfg.kind == I.GRID else 6
    jobs = I.job_stream(cfg, njobs, 11)
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"{name} job {k}")
        total += o["steps"]
    assert steps == total
    m.close()


def test_expand_edge_cases(dsp):
    """|Phi_b| = 1 and the maximum 512; a leaf at depth D-1 (children take the
    tail heuristic); every child terminal (robot exits); action subsets."""
    cfg = I.rs15_15().with_(K=512, D=20)
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(4)
    jobs = []
    for n, depth, pos, last in [(1, 0, (3, 3), -1), (512, 0, (0, 7), -1), (300, 19, (5, 5), 2),
                                (77, 5, (14, 2), 0), (512, 10, (13, 13), 1)]:
        pb = I.rs_block(cfg, n, rng, pos=[pos])
        idx = np.arange(n, dtype=np.uint16) if depth == 0 else np.sort(rng.permutation(n)).astype(np.uint16)
        h = I.random_hist(cfg, rng, 6)
        jobs.append(I.Job(parent=pb, idx=idx, last_action=last, depth=depth, hist=h, first_action=0,
                          n_actions=m.num_actions))
    # an action subset
    j = jobs[3]
    jobs.append(I.Job(parent=j.parent, idx=j.idx, last_action=j.last_action, depth=j.depth, hist=j.hist,
                      first_action=4, n_actions=9))
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    res = jb.all_results()
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, a0=j.first_action, na=j.n_actions,
                      cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"edge {k}")
    # exit from the last column: the E children are terminal with zero bounds
    r = res[3]
    assert r["child_count"][1] == 1 and (int(r["key"][1][0]) >> 62) & 1
    assert r["u"][1][0] == 0 and r["l"][1][0] == 0
    m.close()


def test_expand_empty_batch(dsp):
    m = dsp.Model(I.rs7_8())
    from paper_1802_06215_b300 import _dsp
    _dsp.dsp_expand_leaves(m.h, None, 0, 0)
    m.close()


def test_expand_full_size_sampled(dsp):
    """The benchmark's workload (4096 jobs, 15x15 map, 15 rocks, K=500, D=90)
    in the benchmark's launch configuration; a sample of jobs checked against
    the oracle, the partition invariant on all of them."""
    cfg = I.rs15_15()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 4096, 0)
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    _, status = m.counters()
    assert status == 0
    res = jb.all_results()
    for k in range(0, 4096, 211):
        j = jobs[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"full job {k}")
    for k in range(4096):
        r = res[k]
        n = len(jobs[k].idx)
        for a in range(m.num_actions):
            nc = r["child_count"][a]
            assert r["child_off"][a][nc] == n
        assert np.all(np.sort(r["perm"], axis=1) == np.arange(n))
    m.close()


@pytest.mark.parametrize("block", [128, 512])
def test_expand_parity_block_sizes(dsp, block):
    """Every rollout-phase CTA size the autotuner may pick gives the oracle's
    result."""
    from paper_1802_06215_b300 import _dsp
    cfg = I.rs15_15()
    m = dsp.Model(cfg)
    _dsp.dsp_set_tuning(m.h, block, 0)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 10, 5)
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    _, status = m.counters()
    assert status == 0
    res = jb.all_results()
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"block {block} job {k}")
    m.close()


def test_expand_parity_large_jobs(dsp):
    """One robot with K = 5000: jobs above 512 scenarios take phase A's
    global-memory path (leaf states in the job's leaf-state block); children,
    grouped positions, leaf states and the fixed-point sums bit for bit, next
    to small jobs of the same launch."""
    cfg = I.rs15_15_k(5000)
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    import dataclasses
    jobs = I.job_stream(cfg, 6, 21)
    jobs += [dataclasses.replace(jobs[0], idx=jobs[0].idx[:300].copy()),
             dataclasses.replace(jobs[2], idx=jobs[2].idx[:513].copy())]
    assert max(len(j.idx) for j in jobs) > 512 and min(len(j.idx) for j in jobs) <= 512
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        g = res[k]
        assert np.array_equal(g["leaf"], o["leaf"]), k
        assert np.array_equal(g["child_count"], o["child_count"]), k
        for a in range(m.num_actions):
            nc = int(o["child_count"][a])
            for f in ("key", "rew", "u", "l"):
                assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (k, a, f)
            assert np.array_equal(g["child_off"][a][: nc + 1], o["child_off"][a][: nc + 1]), (k, a)
        assert np.array_equal(g["perm"], o["perm"]), k
        total += o["steps"]
    assert steps == total
    m.close()


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("name", ["rs7_8", "rs15_15", "rs32_32", "rs15_15_k5000"])
def test_expand_parity_rollout_forms(dsp, name, form):
    """Both forms of the one-robot rollout phase give the oracle's result:
    blocks (the rollout phase rebuilds each (action, scenario)'s child state
    and mask from the leaf states, grouped positions and the children's
    offsets and keys) and items (a stored rollout item per pair). Ragged jobs
    with roots and updated leaves, an action subset, |Phi_b| = 1 and 33 (a
    ragged last block), and, at K = 5000, jobs above 512 scenarios next to
    small ones."""
    import dataclasses
    from paper_1802_06215_b300 import _dsp
    cfg = I.rs15_15_k(5000) if name == "rs15_15_k5000" else (rs32_32() if name == "rs32_32" else getattr(I, name)())
    m = dsp.Model(cfg)
    _dsp.dsp_set_launch_shape(m.h, rs_form=form)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 8, 31)
    jobs += [dataclasses.replace(jobs[0], idx=jobs[0].idx[:1].copy()),
             dataclasses.replace(jobs[1], idx=jobs[1].idx[:33].copy(), first_action=3,
                                 n_actions=m.num_actions - 5)]
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, a0=j.first_action, na=j.n_actions,
                      cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"{name} form {form} job {k}")
        total += o["steps"]
    assert steps == total
    m.close()


@pytest.mark.parametrize("form", [1, 2])
def test_expand_parity_mixed_leaves(dsp, form):
    """Leaves whose scenarios differ in the robot's position and sampled mask
    (not a tree node's, but a valid input) take the grouping phase's general
    path, next to jobs whose scenarios share them (the fast path): all match
    the oracle, with roots and updated leaves, in both rollout forms."""
    from paper_1802_06215_b300 import _dsp
    cfg = I.rs15_15()
    m = dsp.Model(cfg)
    _dsp.dsp_set_launch_shape(m.h, rs_form=form)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(17)
    jobs = []
    for n, depth, last in [(200, 0, -1), (77, 4, 0), (300, 6, 4), (33, 2, 7)]:
        pb = I.rs_block(cfg, n, rng)  # per-scenario positions
        samp = rng.integers(0, 1 << cfg.m, n).astype(np.uint32) & rng.integers(0, 1 << cfg.m, n).astype(np.uint32)
        pb[3] = samp
        pb[2] &= ~samp
        idx = np.arange(n, dtype=np.uint16) if depth == 0 else np.sort(rng.permutation(n)[: n - n // 3]).astype(np.uint16)
        jobs.append(I.Job(parent=pb, idx=idx, last_action=last, depth=depth, hist=I.random_hist(cfg, rng, depth),
                          first_action=0, n_actions=m.num_actions))
    jobs += I.job_stream(cfg, 4, 23)
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"mixed job {k} form {form}")
        total += o["steps"]
    assert steps == total
    m.close()


def test_expand_parity_two_robots_shared_cells(dsp):
    """Two robots, leaves that share both positions (as a tree node's do)
    placed on the joint step's corner cases: both robots on one rock (a
    joint Sample of the same rock, a Sense after the other robot's Sample),
    one robot or both already exited, robots on the east and north borders;
    next to leaves with per-scenario positions and a job split over several
    action ranges. All match the oracle."""
    cfg = I.mars11_11()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(29)
    rock = [(int(c) & 0xFF, int(c) >> 8) for c in cfg.rock_cells]
    n1 = cfg.n - 1
    cases = [
        # (positions, exited, sampled, n, depth)
        ([rock[0], rock[0]], (0, 0), 0, 150, 0),
        ([rock[1], rock[1]], (0, 0), 1 << 2, 64, 3),
        ([rock[2], rock[3]], (1, 0), 0, 90, 5),
        ([rock[4], (n1, 0)], (0, 1), 1 << 4, 33, 2),
        ([(n1, n1), (n1, 5)], (0, 0), 0, 120, 7),
        ([(0, 0), (3, 3)], (1, 1), 0, 40, 4),
        ([rock[5], (n1, n1)], (0, 0), 1 << 5, 1, 1),
    ]
    jobs = []
    for pos, ex, samp, n, depth in cases:
        pb = I.rs_block(cfg, n, rng, pos=pos, sampled=samp, exited=ex)
        jobs.append(I.Job(parent=pb, idx=np.arange(n, dtype=np.uint16), last_action=-1, depth=depth,
                          hist=I.random_hist(cfg, rng, depth), first_action=0, n_actions=m.num_actions))
    for n, depth in [(80, 2), (17, 6)]:
        pb = I.rs_block(cfg, n, rng)  # per-scenario positions
        samp = rng.integers(0, 1 << cfg.m, n).astype(np.uint32) & rng.integers(0, 1 << cfg.m, n).astype(np.uint32)
        pb[3] = samp
        pb[2] &= ~samp
        jobs.append(I.Job(parent=pb, idx=np.arange(n, dtype=np.uint16), last_action=-1, depth=depth,
                          hist=I.random_hist(cfg, rng, depth), first_action=0, n_actions=m.num_actions))
    # one node's actions in three ranges
    pb = I.rs_block(cfg, 70, rng, pos=[rock[6], rock[6]])
    third = m.num_actions // 3
    for lo, hi in [(0, third), (third, 2 * third), (2 * third, m.num_actions)]:
        jobs.append(I.Job(parent=pb, idx=np.arange(70, dtype=np.uint16), last_action=-1, depth=3,
                          hist=np.zeros(32, np.int8), first_action=lo, n_actions=hi - lo))
    jobs += I.job_stream(cfg, 4, 31)
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, a0=j.first_action, na=j.n_actions,
                      cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"two-robot job {k}")
        total += o["steps"]
    assert steps == total
    m.close()


@pytest.mark.parametrize("name", ["rs15_15", "mars15_15"])
def test_expand_parity_slice_boundaries(dsp, name):
    """Children of 1, 127, 128, 129, 256, 257 and 500 items: the rollout
    phase takes each child's items in slices of up to 128 (a move gives every
    scenario of a shared-position job one child of n items), so these sizes
    put a child's last slice at one item, a full slice and one past it; with
    a leaf of mixed positions beside them (items that take the per-item
    path). All match the oracle."""
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(41)
    robots = 2 if name.startswith("mars") else 1
    jobs = []
    for k, n in enumerate([1, 127, 128, 129, 256, 257, 500]):
        pos = [(int(rng.integers(0, cfg.n - 1)), int(rng.integers(0, cfg.n))) for _ in range(robots)]
        pb = I.rs_block(cfg, n, rng, pos=pos, sampled=int(1 << (k % cfg.m)))
        depth = k % 4
        jobs.append(I.Job(parent=pb, idx=np.arange(n, dtype=np.uint16), last_action=-1, depth=depth,
                          hist=I.random_hist(cfg, rng, depth), first_action=0, n_actions=m.num_actions))
    pb = I.rs_block(cfg, 300, rng)  # per-scenario positions
    jobs.append(I.Job(parent=pb, idx=np.arange(300, dtype=np.uint16), last_action=-1, depth=1,
                      hist=I.random_hist(cfg, rng, 1), first_action=0, n_actions=m.num_actions))
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, a0=j.first_action, na=j.n_actions,
                      cap=m.max_children(len(j.idx)))
        _cmp_expand(res[k], o, len(j.idx), f"{name} job {k}")
        total += o["steps"]
    assert steps == total
    m.close()
