"""Rollouts with the learned policy on the GPU against the CPU oracle.

The network runs as BF16 tensor-core tiles on the GPU and as a BF16/FP32
restatement in the oracle, so logits agree only to rounding. The GPU logs
every step's action and the tile's logits; the oracle replays the logged
actions (values then agree bit for bit, g being stepped identically) and
computes its own logits at every step. The bar:
  * every logit within 1e-2 relative of the oracle's, |g - o| <= 1e-2 (1 + |o|)
    (the floor of 1e-2 serves logits near zero);
  * argmax agreement wherever the oracle's top-2 margin over the allowed
    columns exceeds 1e-2: no logged action's oracle logit trails the oracle's
    best by more than 1e-2."""
import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I

pytestmark = pytest.mark.gpu
G32 = float(np.float32(0.95))


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    return torch, _dsp, batch


def bf16_exact(a):
    a = np.asarray(a, np.float32).copy()
    u = a.view(np.uint32)
    u += 0x7FFF + ((u >> 16) & 1)
    u &= 0xFFFF0000
    return a


def weights(seed, zero=False):
    rng = np.random.default_rng(seed)
    w = {"W1": rng.normal(0, np.sqrt(2 / 64), (64, 256)), "b1": rng.normal(0, 0.1, 256),
         "W2": rng.normal(0, np.sqrt(2 / 256), (256, 256)), "b2": rng.normal(0, 0.1, 256),
         "W3": rng.normal(0, 3 * np.sqrt(2 / 256), (256, 32)), "b3": rng.normal(0, 0.5, 32)}
    if zero:
        for k in w:
            w[k][:] = 0
    return {k: bf16_exact(v).astype(np.float64) for k, v in w.items()}


def install(_dsp, m, w):
    h = _dsp.dsp_mlp_create(64, 0)
    _dsp.dsp_mlp_set_weights(h, _dsp.pack_params(w))
    _dsp.dsp_set_policy(m.h, h)
    return h


TOL = 1e-2


def logged_rollout(torch, _dsp, m, cfg, b, hist, d0, want_logits=False):
    n = b.shape[1]
    bd = torch.tensor(b.view(np.int32), device="cuda")
    hd = torch.tensor(hist, device="cuda")
    val = torch.zeros(n, dtype=torch.float32, device="cuda")
    act = torch.full((n, cfg.D), -1, dtype=torch.int32, device="cuda")
    lg = torch.full((n, cfg.D, 32), float("nan"), dtype=torch.float32, device="cuda") if want_logits else None
    _dsp.dsp_rollout_logged(m.h, bd.data_ptr(), n, n, hd.data_ptr(), d0, val.data_ptr(), act.data_ptr(),
                            logits_ptr=lg.data_ptr() if want_logits else 0)
    torch.cuda.synchronize()
    if want_logits:
        return val.cpu().numpy(), act.cpu().numpy(), lg.cpu().numpy()
    return val.cpu().numpy(), act.cpu().numpy()


def check_replay(om, b, hist, d0, w, val, act, glog):
    """The oracle replays the logged actions: values bit for bit, logits of
    every step element-wise, argmax wherever the margin exceeds TOL."""
    ov, bad, steps, olog = oracle.rollout_learned(om, b, hist, d0, w, logged=act, tol=TOL, want_logits=True)
    assert np.array_equal(val.astype(np.float64), ov)
    assert bad.sum() == 0, (int(bad.sum()), steps)
    live = act >= 0
    assert int(live.sum()) == steps
    assert np.array_equal(np.isfinite(olog[..., 0]), live) and np.array_equal(np.isfinite(glog[..., 0]), live)
    g, o = glog[live].astype(np.float64), olog[live]
    err = np.abs(g - o)
    assert np.all(err <= TOL * (1.0 + np.abs(o))), float((err / (1.0 + np.abs(o))).max())
    return steps, float(err.max())


@pytest.mark.parametrize("seed,side", [(1, 15), (2, 15), (3, 15), (4, 32), (5, 7)])
def test_learned_rollout_replays_in_oracle(env, seed, side):
    """Random networks on 300 states; the 32x32 map takes the kernel's
    feature path without the pair table (it does not fit in shared memory)."""
    torch, _dsp, batch = env
    cfg = I.rs15_15().with_(D=40) if side == 15 else I.grid_config(side, min(15, side), K=500, D=40, seed=side)
    m = batch.Model(cfg)
    w = weights(seed)
    hm = install(_dsp, m, w)
    rng = np.random.default_rng(seed)
    N = 300
    b = I.rs_block(cfg, N, rng)
    b[2] &= ~b[3]
    hist = rng.integers(-3, 4, (N, 32)).astype(np.int8)
    val, act, glog = logged_rollout(torch, _dsp, m, cfg, b, hist, 5, want_logits=True)
    om = oracle.Model(cfg)
    check_replay(om, b, hist, 5, w, val, act, glog)
    # the policy does sense and sample, not only walk
    used = set(act[act >= 0].tolist())
    assert len(used) >= 4
    _, st = m.counters()
    assert st == 0
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def test_constant_east_network_closed_form(env):
    """Logits equal to a bias favouring E: the learned rollout walks east, worth
    10 * gamma^(n-1-x)."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    w = weights(0, zero=True)
    w["b3"][1] = 4.0
    hm = install(_dsp, m, w)
    rng = np.random.default_rng(0)
    for x in (0, 9, 14):
        b = I.rs_block(cfg, 70, rng, pos=[(x, 5)])
        val, act = logged_rollout(torch, _dsp, m, cfg, b, np.zeros((70, 32), np.int8), 2)
        assert np.allclose(val, 10 * G32 ** (14 - x), rtol=1e-6)
        assert np.all(act[:, : 15 - x] == 1)
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def test_learned_expansion(env):
    """With a learned policy the expansion keeps the oracle's children, rewards
    and u0 (they do not depend on the policy), and each child's l0 sum equals
    the sum of the logged single rollouts of its scenarios, which the oracle
    replays bit for bit."""
    torch, _dsp, batch = env
    cfg = I.rs15_15().with_(D=30)
    m = batch.Model(cfg)
    w = weights(9)
    hm = install(_dsp, m, w)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 6, 4, max_scen=80)
    jb = batch.JobBatch(m, jobs)
    jb.run()
    _, st = m.counters()
    assert st == 0
    res = jb.all_results()
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        g = res[k]
        assert np.array_equal(g["perm"], o["perm"]) and np.array_equal(g["child_count"], o["child_count"])
        leaf = o["leaf"]
        n = leaf.shape[1]
        for a in range(m.num_actions):
            nc = int(o["child_count"][a])
            assert np.array_equal(g["rew"][a][:nc], o["rew"][a][:nc])
            assert np.array_equal(g["u"][a][:nc], o["u"][a][:nc])
            nxt, keys, _ = om.step(leaf, np.full(n, a, np.int32), j.depth)
            hist = np.tile(j.hist, (n, 1))
            if a >= 5:
                z = (keys & np.uint64(3)).astype(np.int64)
                hist[:, a - 5] = np.clip(hist[:, a - 5].astype(int) + np.where(z == 1, 1, np.where(z == 2, -1, 0)),
                                         -127, 127)
            val, act, glog = logged_rollout(torch, _dsp, m, cfg, nxt, hist, j.depth + 1, want_logits=True)
            check_replay(om, nxt, hist, j.depth + 1, w, val, act, glog)
            fixed = np.round(val.astype(np.float64) * 2 ** 32).astype(np.int64)
            for c in range(nc):
                mem = g["perm"][a][g["child_off"][a][c]:g["child_off"][a][c + 1]]
                assert g["l"][a][c] == fixed[mem].sum(), (k, a, c)
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def test_defer_network_is_the_heuristic(env):
    """A network that always defers reproduces the heuristic rollout kernel
    bit for bit (values and step counts)."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    rng = np.random.default_rng(11)
    N = 4000
    b = I.rs_block(cfg, N, rng)
    b[3] = rng.integers(0, 1 << 15, N).astype(np.uint32)
    b[2] &= ~b[3]
    hist = rng.integers(-2, 4, (N, 32)).astype(np.int8)
    m.reset_counters()
    vh = m.rollout(b, hist, 3)
    sh, _ = m.counters()
    w = weights(0, zero=True)
    w["b3"][20] = 3.0
    w["b3"][4] = 1.0
    hm = install(_dsp, m, w)
    m.reset_counters()
    vl = m.rollout(b, hist, 3)
    sl, st = m.counters()
    assert st == 0 and sl == sh
    assert np.array_equal(np.asarray(vh).view(np.uint32), np.asarray(vl).view(np.uint32))
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def _child_hist(j, a, keys, n):
    hist = np.tile(j.hist, (n, 1))
    if a >= 5:
        z = (keys & np.uint64(3)).astype(np.int64)
        hist[:, a - 5] = np.clip(hist[:, a - 5].astype(int) + np.where(z == 1, 1, np.where(z == 2, -1, 0)),
                                 -127, 127)
    return hist


def test_learned_expansion_full_size_sampled(env):
    """The benchmark's learned-policy expansion as timed: the shipped weights,
    15x15 with 15 rocks, K = 500, D = 90, the first 256 jobs of the 4096-job
    stream (|Phi_b| ~ U{1..500}) in one launch. Children, rewards and u0 of
    every job equal the oracle's. For sampled (job, action) pairs (the
    smallest, median and largest job; a move and a Sense), each child's l0 sum
    equals the sum of that action's logged single rollouts, and the oracle
    replays 24 of those rollouts: values bit for bit, logits element-wise,
    argmax."""
    torch, _dsp, batch = env
    import os
    from paper_1802_06215_b300 import learn
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h, _ = learn.load_weights(os.path.join(root, "paper_1802_06215_b300", "weights", "rs15_15_pi0.npz"))
    w = {k: v.astype(np.float64) for k, v in _dsp.unpack_params(_dsp.dsp_mlp_get_weights(h)).items()}
    _dsp.dsp_set_policy(m.h, h)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 4096, 1000)[:256]
    jb = batch.JobBatch(m, jobs)
    jb.run()
    torch.cuda.synchronize()
    _, st = m.counters()
    assert st == 0
    res = jb.all_results()
    # policy-independent parts of every job (the oracle's heuristic expansion)
    for k in range(0, 256, 16):
        j = jobs[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        g = res[k]
        assert np.array_equal(g["perm"], o["perm"]) and np.array_equal(g["child_count"], o["child_count"]), k
        for a in range(m.num_actions):
            nc = int(o["child_count"][a])
            assert np.array_equal(g["rew"][a][:nc], o["rew"][a][:nc]), (k, a)
            assert np.array_equal(g["u"][a][:nc], o["u"][a][:nc]), (k, a)
    sizes = np.array([len(j.idx) for j in jobs])
    order = np.argsort(sizes, kind="stable")
    picks = [int(order[0]), int(order[len(order) // 2]), int(order[-1])]
    rng = np.random.default_rng(5)
    worst = 0.0
    for k in picks:
        j = jobs[k]
        g = res[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        leaf = o["leaf"]
        n = leaf.shape[1]
        for a in (1, 5 + int(rng.integers(0, cfg.m))):
            nxt, keys, _ = om.step(leaf, np.full(n, a, np.int32), j.depth)
            hist = _child_hist(j, a, keys, n)
            val, act, glog = logged_rollout(torch, _dsp, m, cfg, nxt, hist, j.depth + 1, want_logits=True)
            fixed = np.round(val.astype(np.float64) * 2 ** 32).astype(np.int64)
            nc = int(o["child_count"][a])
            for c in range(nc):
                mem = g["perm"][a][g["child_off"][a][c]:g["child_off"][a][c + 1]]
                assert g["l"][a][c] == fixed[mem].sum(), (k, a, c)
            sel = np.sort(rng.choice(n, size=min(n, 24), replace=False))
            _, e = check_replay(om, nxt[:, sel], hist[sel], j.depth + 1, w, val[sel], act[sel], glog[sel])
            worst = max(worst, e)
    print("largest logit difference", worst)
    _dsp.dsp_set_policy(m.h, None)
    _dsp.dsp_mlp_destroy(h)
    m.close()
