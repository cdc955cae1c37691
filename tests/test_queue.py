"""Device job queue: many host threads submit leaves of uneven |Phi_b| to one
persistent kernel; every job's results must equal the CPU oracle's leaf
expansion (Eq. expand, newnodes, ub, lb) bit for bit, and dsp_expand_leaves's."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I

pytestmark = pytest.mark.gpu

FIELDS = ("leaf", "child_count", "child_off", "key", "rew", "u", "l", "perm")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    return torch, _dsp, batch


def _run_threads(_dsp, q, jb, n_threads):
    errors = []
    idx = list(range(len(jb.jobs)))

    def worker(tid):
        try:
            for k in idx[tid::n_threads]:
                t = _dsp.dsp_queue_submit(q, jb.descs[k], 10_000_000_000)
                _dsp.dsp_queue_wait(q, t, 30_000_000_000)
        except Exception as e:  # reported below
            errors.append(e)

    th = [threading.Thread(target=worker, args=(i,)) for i in range(n_threads)]
    for x in th:
        x.start()
    for x in th:
        x.join()
    assert not errors, errors


def _rs32_32():
    return I.grid_config(32, 32, K=100, D=120, seed=3)


def _cmp_oracle(cfg, m, jobs, results, plan_steps=None):
    """Each job's queue results against the oracle's expansion of the same leaf."""
    oms = {}
    for k, (j, g) in enumerate(zip(jobs, results)):
        ps = cfg.plan_step if plan_steps is None else plan_steps[k]
        om = oms.setdefault(ps, oracle.Model(cfg, plan_step=ps))
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        assert np.array_equal(g["leaf"], o["leaf"]), (k, "leaf")
        assert np.array_equal(g["child_count"], o["child_count"]), (k, "child_count")
        assert np.array_equal(g["perm"], o["perm"]), (k, "perm")
        for a in range(len(o["child_count"])):
            nc = int(o["child_count"][a])
            assert np.array_equal(g["child_off"][a][: nc + 1], o["child_off"][a][: nc + 1]), (k, a, "off")
            for f in ("key", "rew", "u", "l"):
                assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (k, a, f)


@pytest.mark.parametrize("mk,njobs,threads", [(I.mars15_15, 48, 16), (I.rs15_15, 96, 16), (I.rs7_8, 40, 4),
                                              (_rs32_32, 24, 4)])
def test_queue_matches_batch(env, mk, njobs, threads):
    torch, _dsp, batch = env
    cfg = mk()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, njobs, 17)
    ref = batch.JobBatch(m, jobs)
    ref.run()
    torch.cuda.synchronize()
    out = batch.JobBatch(m, jobs)
    q = _dsp.dsp_queue_create(m.h, 64)
    _run_threads(_dsp, q, out, threads)
    launches, submitted = _dsp.dsp_queue_stats(q)
    _dsp.dsp_queue_destroy(q)
    assert submitted == njobs and launches >= 1
    _, status = m.counters()
    assert status == 0
    got = out.all_results()
    for k, (a, b) in enumerate(zip(ref.all_results(), got)):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (k, f)
    _cmp_oracle(cfg, m, jobs, got)
    m.close()


def test_queue_two_robots_sixteen_producers_oracle(env):
    """Two robots on 15x15 with 15 rocks (400 joint actions), K = 500, D = 90:
    16 host threads submit 64 leaves with |Phi_b| ~ U{1..500} and depth ~
    U{0..10} into one persistent kernel; every job equals the oracle."""
    torch, _dsp, batch = env
    cfg = I.mars15_15()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 64, 41)
    sizes = [len(j.idx) for j in jobs]
    assert min(sizes) < 100 and max(sizes) > 400
    out = batch.JobBatch(m, jobs)
    q = _dsp.dsp_queue_create(m.h, 32)
    _run_threads(_dsp, q, out, 16)
    launches, submitted = _dsp.dsp_queue_stats(q)
    _dsp.dsp_queue_destroy(q)
    assert submitted == len(jobs)
    _, status = m.counters()
    assert status == 0
    _cmp_oracle(cfg, m, jobs, out.all_results())
    m.close()


@pytest.mark.parametrize("mk,njobs,threads", [(I.car50, 24, 8), (lambda: I.car_p(6), 16, 4), (I.nav13, 32, 16)])
def test_queue_car_and_navigation_oracle(env, mk, njobs, threads):
    """The car among 50 and 6 pedestrians and navigation in a partially known
    map through their own persistent queue kernels: host threads submit
    leaves of uneven |Phi_b| (1..500); every job equals the oracle's expansion
    (the car bit for bit in FP32, as the batch call) and the batch call's."""
    torch, _dsp, batch = env
    cfg = mk()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, njobs, 19)
    ref = batch.JobBatch(m, jobs)
    ref.run()
    torch.cuda.synchronize()
    out = batch.JobBatch(m, jobs)
    q = _dsp.dsp_queue_create(m.h, 16)
    _run_threads(_dsp, q, out, threads)
    launches, submitted = _dsp.dsp_queue_stats(q)
    _dsp.dsp_queue_destroy(q)
    assert submitted == njobs and launches >= 1
    _, status = m.counters()
    assert status == 0
    got = out.all_results()
    for k, (a, b) in enumerate(zip(ref.all_results(), got)):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (k, f)
    _cmp_oracle(cfg, m, jobs, got)
    m.close()


def test_queue_car_refuses_learned_policy(env):
    torch, _dsp, batch = env
    from paper_1802_06215_b300 import learn
    import os
    cfg = I.car50()
    m = batch.Model(cfg)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h, _ = learn.load_weights(os.path.join(root, "paper_1802_06215_b300", "weights", "car50_pi0.npz"))
    _dsp.dsp_set_policy(m.h, h)
    jb = batch.JobBatch(m, I.job_stream(cfg, 1, 3, max_scen=20))
    q = _dsp.dsp_queue_create(m.h, 4)
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_queue_submit(q, jb.descs[0], 1000)
    assert e.value.status == _dsp.DSP_E_UNSUPPORTED
    _dsp.dsp_queue_destroy(q)
    _dsp.dsp_mlp_destroy(h)
    m.close()


def test_queue_relaunch_after_idle(env):
    """With a 50 us idle limit the kernel's bounded wait runs out between
    bursts; the monitor relaunches it and every job still completes."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 12, 23, max_scen=100)
    ref = batch.JobBatch(m, jobs)
    ref.run()
    out = batch.JobBatch(m, jobs)
    q = _dsp.dsp_queue_create(m.h, 4, 50_000)
    for burst in (range(0, 6), range(6, 12)):
        tickets = [_dsp.dsp_queue_submit(q, out.descs[k], 10_000_000_000) for k in burst]
        for t in tickets:
            _dsp.dsp_queue_wait(q, t, 30_000_000_000)
        time.sleep(0.05)
    launches, submitted = _dsp.dsp_queue_stats(q)
    _dsp.dsp_queue_destroy(q)
    assert submitted == 12 and launches >= 2
    got = out.all_results()
    for k, (a, b) in enumerate(zip(ref.all_results(), got)):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (k, f)
    _cmp_oracle(cfg, m, jobs, got)
    m.close()


def test_queue_rejects_bad_input(env):
    torch, _dsp, batch = env
    m = batch.Model(I.rs7_8())
    q = _dsp.dsp_queue_create(m.h, 8)
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_queue_wait(q, 5, 1000)  # never issued
    assert e.value.status == _dsp.DSP_E_INVALID
    bad = _dsp.dsp_leaf_job()  # null pointers, zero scenarios
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_queue_submit(q, bad, 1000)
    assert e.value.status in (_dsp.DSP_E_INVALID, _dsp.DSP_E_UNSUPPORTED)
    _dsp.dsp_queue_destroy(q)
    m.close()


def test_queue_jobs_keep_their_plan_step(env):
    """Each job draws its random streams under the plan step the model had
    when it was submitted (Sense readings differ between plan steps): jobs
    submitted under alternating plan steps, while one persistent kernel runs,
    equal batch expansions taken under the same plan steps."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 10, 31, max_scen=200)
    steps = [5 if k % 2 == 0 else 9 for k in range(len(jobs))]
    refs = {}
    for ps in (5, 9):
        m.set_plan_step(ps)
        r = batch.JobBatch(m, jobs)
        r.run()
        torch.cuda.synchronize()
        refs[ps] = r.all_results()
    assert any(not np.array_equal(refs[5][k]["key"], refs[9][k]["key"]) for k in range(len(jobs)))
    out = batch.JobBatch(m, jobs)
    q = _dsp.dsp_queue_create(m.h, 16)
    tickets = []
    for k in range(len(jobs)):
        m.set_plan_step(steps[k])
        tickets.append(_dsp.dsp_queue_submit(q, out.descs[k], 10_000_000_000))
    for t in tickets:
        _dsp.dsp_queue_wait(q, t, 30_000_000_000)
    _dsp.dsp_queue_destroy(q)
    got = out.all_results()
    for k in range(len(jobs)):
        for f in FIELDS:
            assert np.array_equal(refs[steps[k]][k][f], got[k][f]), (k, f)
    _cmp_oracle(cfg, m, jobs, got, plan_steps=steps)
    _, status = m.counters()
    assert status == 0
    m.close()


def test_search_keeps_its_queue_across_planning_steps(env):
    """Two free-running planning steps through the device queue on one model:
    the model keeps the queue (and its persistent kernel's graph) and both
    steps finish with consistent root bounds."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    root = I.rs_block(cfg, cfg.K, np.random.default_rng(1), pos=[(0, 7)])
    p = _dsp.dsp_search_params(threads=4, rounds=40, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0,
                               deterministic=0, use_queue=1)
    for k in range(2):
        m.set_plan_step(100 + k)
        r = _dsp.dsp_plan(m.h, root, None, p, m.num_actions)
        assert r["expansions"] >= 1 and r["root_l"] <= r["root_u"] + 1e-9
        assert 0 <= r["action"] < m.num_actions
    _, status = m.counters()
    assert status == 0
    m.close()
