"""GPU vs CPU oracle, navigation in a partially known map (Sec. IV-A): g,
the default-policy rollout and the whole leaf expansion, bit for bit (integer
states, 8-bit readings, FP32 rewards and values in the same order, exact
fixed-point sums)."""
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


CONFIGS = {"nav13": I.nav13, "nav13 noisy": lambda: I.nav13().with_(fail_p=0.2, sense_p=0.2),
           "nav9": lambda: I.nav_config(9, K=200, D=60, seed=5), "nav16": lambda: I.nav_config(16, K=200, D=60, seed=6),
           # the smallest map with every move failing and every reading flipped
           # (thresholds of 2^32), and an odd map without noise
           "nav5 p=1": lambda: I.nav_config(5, K=100, D=60, seed=7).with_(fail_p=1.0, sense_p=1.0),
           "nav15 p=0": lambda: I.nav_config(15, K=200, D=60, seed=8).with_(fail_p=0.0, sense_p=0.0)}


@pytest.mark.parametrize("name", list(CONFIGS))
def test_step_parity(dsp, name):
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(4)
    N = 3000
    b = I.nav_block(cfg, N, rng, pos=(cfg.n // 2, cfg.n // 2 + 1), spread=cfg.n)
    b[0, :40] |= 1 << 16  # some terminal scenarios
    acts = rng.integers(0, 9, N).astype(np.int32)
    for depth in (0, 17, 59):
        go, gk, gr = m.step(b, acts, depth)
        oo, ok, orr = om.step(b, acts, depth)
        assert np.array_equal(go, oo), (name, depth)
        assert np.array_equal(gk, ok), (name, depth)
        assert np.array_equal(gr.astype(np.float64), orr), (name, depth)
    m.close()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_rollout_parity(dsp, name):
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(9)
    N = 1500
    b = I.nav_block(cfg, N, rng, pos=(cfg.n // 2, 2), spread=cfg.n)
    h = np.zeros((N, 32), np.int8)
    h[:, 0] = rng.integers(0, 256, N).astype(np.uint8).view(np.int8)
    for d0 in (0, 30, cfg.D - 1, cfg.D):
        gv = m.rollout(b, h, d0)
        ov, _ = om.rollout(b, h, d0)
        assert np.array_equal(gv.astype(np.float64), ov), (name, d0)
    m.close()


@pytest.mark.parametrize("name", list(CONFIGS))
def test_expand_parity_ragged(dsp, name):
    """Ragged |Phi_b|, random depths, roots and updated leaves; children by
    the 8-bit reading, in the oracle's order, with bit-exact sums."""
    cfg = CONFIGS[name]()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 10, 13)
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
        assert np.array_equal(g["leaf"], o["leaf"]), (name, k)
        assert np.array_equal(g["child_count"], o["child_count"]), (name, k)
        for a in range(9):
            nc = int(o["child_count"][a])
            for f in ("key", "rew", "u", "l"):
                assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (name, k, a, f)
            assert np.array_equal(g["child_off"][a][: nc + 1], o["child_off"][a][: nc + 1]), (name, k, a)
        assert np.array_equal(g["perm"], o["perm"]), (name, k)
        total += o["steps"]
    assert steps == total
    m.close()


def test_expand_full_size_sampled(dsp):
    """The benchmark's launch (512 jobs of up to 500 scenarios): sampled jobs
    against the oracle, and the step count against the oracle's on those."""
    cfg = I.nav13()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 512, 1000)
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    _, status = m.counters()
    assert status == 0
    res = jb.all_results()
    for k in (0, 77, 255, 511):
        j = jobs[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        g = res[k]
        assert np.array_equal(g["child_count"], o["child_count"]), k
        for a in range(9):
            nc = int(o["child_count"][a])
            for f in ("key", "rew", "u", "l"):
                assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (k, a, f)
        assert np.array_equal(g["perm"], o["perm"]), k
    m.close()
