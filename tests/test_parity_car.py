"""GPU vs CPU oracle, car among pedestrians: the FP32 kernels follow the FP32
oracle's operation order with --fmad=false, so states, keys, rewards and
fixed-point sums are expected bit-exact; the stated tolerance (1e-5 relative
on values) is checked as well."""
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


def test_gauss_table_matches_oracle(dsp):
    m = dsp.Model(I.car50())
    _, o32 = oracle.gauss_table()
    assert np.array_equal(m.table(2), o32)
    g32, _ = oracle.gamma_powers(0.95, 256)
    assert np.array_equal(m.table(1), g32)
    m.close()


@pytest.mark.parametrize("P", [50, 7, 1])
def test_step_parity(dsp, P):
    cfg = I.car_config(P=P, K=500, D=50)
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(P)
    N = 1500
    b = I.car_block(cfg, N, rng)
    b[1, :20] |= 1 << 8  # some terminal scenarios
    acts = rng.integers(0, 3, N).astype(np.int32)
    for depth in (0, 13, 49):
        go, gk, gr = m.step(b, acts, depth)
        oo, ok, orr = om.step(b, acts, depth)
        assert np.array_equal(go, oo), depth
        assert np.array_equal(gk, ok), depth
        assert np.array_equal(gr.astype(np.float64), orr), depth
    m.close()


def test_rollout_parity(dsp):
    cfg = I.car50()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(3)
    b = I.car_block(cfg, 400, rng)
    for d0 in (0, 30, 49, 50):
        gv = m.rollout(b, None, d0)
        ov, _ = om.rollout(b, None, d0)
        assert np.array_equal(gv.astype(np.float64), ov), d0
    m.close()


def _cmp(g, o, tag):
    assert np.array_equal(g["leaf"], o["leaf"]), tag
    assert np.array_equal(g["child_count"], o["child_count"]), tag
    for a in range(len(o["child_count"])):
        nc = int(o["child_count"][a])
        assert np.array_equal(g["child_off"][a][: nc + 1], o["child_off"][a][: nc + 1]), (tag, a)
        assert np.array_equal(g["key"][a][:nc], o["key"][a][:nc]), (tag, a)
        for f in ("rew", "u", "l"):
            gv, ov = g[f][a][:nc] / 2**32, o[f][a][:nc] / 2**32
            assert np.all(np.abs(gv - ov) <= 1e-5 * np.maximum(np.abs(ov), 1.0)), (tag, a, f)
            assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (tag, a, f, "bit-exact")
    assert np.array_equal(g["perm"], o["perm"]), tag


@pytest.mark.parametrize("tps", [16, 8, 32, 4])
def test_expand_parity(dsp, tps):
    """Ragged |Phi_b|, random depths; every within-step split (threads per
    scenario) gives the oracle's result."""
    from paper_1802_06215_b300 import _dsp
    cfg = I.car50()
    m = dsp.Model(cfg)
    _dsp.dsp_set_tuning(m.h, 0, tps)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 6, 21, max_scen=70)
    jb = dsp.JobBatch(m, jobs)
    m.reset_counters()
    jb.run()
    steps, status = m.counters()
    assert status == 0
    res = jb.all_results()
    total = 0
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp(res[k], o, f"tps{tps} job {k}")
        total += o["steps"]
    assert steps == total
    m.close()


@pytest.mark.parametrize("P", [6, 7, 12, 20])
def test_expand_parity_crowd_sizes(dsp, P):
    """The crowd sizes of the pedestrian-count study, at the default lanes per
    scenario and at 4 and 8: each lane owns one to three pedestrian pairs (the
    kernel sized to the crowd), some lanes fewer or none."""
    from paper_1802_06215_b300 import _dsp
    cfg = I.car_p(P)
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 6, 23 + P, max_scen=70)
    expect = [om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
              for j in jobs]
    for tps in (0, 4, 8):
        _dsp.dsp_set_tuning(m.h, 0, tps)
        jb = dsp.JobBatch(m, jobs)
        m.reset_counters()
        jb.run()
        steps, status = m.counters()
        assert status == 0
        res = jb.all_results()
        for k, o in enumerate(expect):
            _cmp(res[k], o, f"P{P} tps{tps} job {k}")
        assert steps == sum(o["steps"] for o in expect)
        del jb
    m.close()


def test_expand_shared_observations(dsp):
    """Scenarios with identical pedestrians and goals (no noise, no action
    failure) share observations, so children hold several scenarios."""
    cfg = I.car_config(P=12, K=64, D=30).with_(sigma=0.0, fail_p=0.0)
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    rng = np.random.default_rng(8)
    base = (rng.uniform(0, 40, 12), rng.uniform(0, 40, 12))
    pb = I.car_block(cfg, 64, rng, s=5.0, v=1, base=base, jitter=0.0)
    # half the scenarios take scenario 0's goals, the rest scenario 1's
    gw = 4 + 2 * 12
    pb[gw:, 0::2] = pb[gw:, 0:1]
    pb[gw:, 1::2] = pb[gw:, 1:2]
    jobs = [I.Job(parent=pb, idx=np.arange(64, dtype=np.uint16), last_action=-1, depth=0,
                  hist=np.zeros(32, np.int8), first_action=0, n_actions=3)]
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    _, status = m.counters()
    assert status == 0
    o = om.expand(pb, jobs[0].idx, -1, 0, None, cap=m.max_children(64))
    _cmp(jb.all_results()[0], o, "shared")
    assert o["child_count"].max() <= 2
    m.close()


def test_expand_full_size_sampled(dsp):
    """The benchmark's car workload (1024 jobs, 50 pedestrians, K=500, D=50) in
    its launch configuration; a sample checked against the oracle."""
    cfg = I.car50()
    m = dsp.Model(cfg)
    om = oracle.Model(cfg)
    jobs = I.job_stream(cfg, 1024, 0)
    jb = dsp.JobBatch(m, jobs)
    jb.run()
    _, status = m.counters()
    assert status == 0
    res = jb.all_results()
    for k in (0, 500, 1023):
        j = jobs[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        _cmp(res[k], o, f"full job {k}")
    m.close()
