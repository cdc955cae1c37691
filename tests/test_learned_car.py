"""The learned default policy of the car on the GPU (tcgen05 tiles, two lanes
per scenario) against the CPU oracle: features bit for bit, logged rollouts
replayed by the oracle (values bit for bit in FP32, every action the oracle's
argmax within a logit margin), the defer network equal to the heuristic, and
the learned expansion's l0 sums equal to the replayed single rollouts."""
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


def logged(torch, _dsp, m, cfg, b, d0):
    """Values, actions and the tensor-core tile's logits of every step."""
    n = b.shape[1]
    bd = torch.tensor(np.ascontiguousarray(b).view(np.int32), device="cuda")
    val = torch.zeros(n, dtype=torch.float32, device="cuda")
    act = torch.full((n, cfg.D), -1, dtype=torch.int32, device="cuda")
    lg = torch.full((n, cfg.D, 32), float("nan"), dtype=torch.float32, device="cuda")
    _dsp.dsp_rollout_logged(m.h, bd.data_ptr(), n, n, 0, d0, val.data_ptr(), act.data_ptr(),
                            logits_ptr=lg.data_ptr())
    torch.cuda.synchronize()
    return val.cpu().numpy(), act.cpu().numpy(), lg.cpu().numpy()


def check_replay(om, b, d0, w, val, act, glog):
    """Oracle replay of the logged actions: values bit for bit, no logged
    action trailing the oracle's best logit by more than 1e-2 (argmax agreement
    wherever the top-2 margin exceeds 1e-2), and every logit of every step
    within |g - o| <= 1e-2 (1 + |o|)."""
    ov, bad, steps, olog = oracle.rollout_learned(om, b, None, d0, w, logged=act, tol=TOL, want_logits=True)
    assert np.array_equal(val.astype(np.float64), ov)
    assert bad.sum() == 0
    live = act >= 0
    assert int(live.sum()) == steps
    assert np.array_equal(np.isfinite(glog[..., 0]), live) and np.array_equal(np.isfinite(olog[..., 0]), live)
    g, o = glog[live].astype(np.float64), olog[live]
    assert np.all(np.abs(g - o) <= TOL * (1.0 + np.abs(o))), float((np.abs(g - o) / (1 + np.abs(o))).max())


@pytest.mark.parametrize("P", [50, 7])
def test_car_features_match_oracle(env, P):
    torch, _dsp, batch = env
    cfg = I.car_config(P=P)
    m = batch.Model(cfg)
    rng = np.random.default_rng(P)
    for n in (1, 129, 700):
        b = I.car_block(cfg, n, rng)
        bd = torch.tensor(b.view(np.int32), device="cuda")
        f = torch.empty((n, 64), dtype=torch.float32, device="cuda")
        _dsp.dsp_features(m.h, bd.data_ptr(), n, n, 0, f.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        o = oracle.features_car(oracle.Model(cfg), b)
        assert np.array_equal(f.cpu().numpy().view(np.uint32), o.view(np.uint32))
    m.close()


@pytest.mark.parametrize("seed", [1, 2])
def test_car_learned_rollout_replays_in_oracle(env, seed):
    torch, _dsp, batch = env
    cfg = I.car50()
    m = batch.Model(cfg)
    w = weights(seed)
    hm = install(_dsp, m, w)
    rng = np.random.default_rng(seed)
    b = I.car_block(cfg, 300, rng)
    for d0 in (0, 30):
        val, act, glog = logged(torch, _dsp, m, cfg, b, d0)
        check_replay(oracle.Model(cfg), b, d0, w, val, act, glog)
        assert len(set(act[act >= 0].tolist())) >= 2
    _, st = m.counters()
    assert st == 0
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def test_car_defer_network_is_the_heuristic(env):
    torch, _dsp, batch = env
    cfg = I.car50()
    m = batch.Model(cfg)
    rng = np.random.default_rng(5)
    b = I.car_block(cfg, 1000, rng)
    m.reset_counters()
    vh = m.rollout(b, None, 4)
    sh, _ = m.counters()
    w = weights(0, zero=True)
    w["b3"][3] = 3.0
    w["b3"][0] = 1.0
    hm = install(_dsp, m, w)
    m.reset_counters()
    vl = m.rollout(b, None, 4)
    sl, st = m.counters()
    assert st == 0 and sl == sh
    assert np.array_equal(np.asarray(vh).view(np.uint32), np.asarray(vl).view(np.uint32))
    _dsp.dsp_mlp_destroy(hm)
    m.close()


def test_car_learned_expansion(env):
    """With a learned policy the car expansion keeps the oracle's children,
    rewards and u0, and each child's l0 sum equals the sum of the logged
    single rollouts of its scenarios from their stepped states."""
    torch, _dsp, batch = env
    cfg = I.car50()
    m = batch.Model(cfg)
    w = weights(11)
    hm = install(_dsp, m, w)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 5, 6, max_scen=60)
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
            nxt, _, _ = om.step(leaf, np.full(n, a, np.int32), j.depth)
            val, act, glog = logged(torch, _dsp, m, cfg, nxt, j.depth + 1)
            check_replay(om, nxt, j.depth + 1, w, val, act, glog)
            fixed = np.round(val.astype(np.float64) * 2 ** 32).astype(np.int64)
            for c in range(nc):
                mem = g["perm"][a][g["child_off"][a][c]:g["child_off"][a][c + 1]]
                assert g["l"][a][c] == fixed[mem].sum(), (k, a, c)
    _dsp.dsp_mlp_destroy(hm)
    m.close()
