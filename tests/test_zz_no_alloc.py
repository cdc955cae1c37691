"""The allocation-free expansion entry point against the ordinary one.

dsp_expand_leaves_noalloc serves callers that cannot allocate device memory
while planning (a fixed memory pool owns the GPU, or a replanning loop cannot
afford an allocation that may wait on the device). It must give exactly the
results of dsp_expand_leaves, call after call, although every call reuses the
same fixed scratch array; it must leave the device's free memory unchanged,
and it must not wait for work queued earlier on its stream. This file is
collected last on purpose.
"""
import os
import time

import numpy as np
import pytest

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


FIELDS = ("leaf", "child_count", "child_off", "key", "rew", "u", "l", "perm")


def _results(jb):
    return jb.all_results()


@pytest.mark.parametrize("mk", [I.rs15_15, I.mars15_15])
def test_noalloc_matches_expand_leaves_twice(env, mk):
    """Two calls in a row on different job sets, each compared with
    dsp_expand_leaves on the same jobs (bit-exact, as every Rock Sample
    comparison here)."""
    torch, _dsp, batch = env
    cfg = mk()
    m = batch.Model(cfg)
    for call, seed in enumerate((31, 32)):
        jobs = I.job_stream(cfg, 24 if cfg.kind == I.GRID else 4, seed)
        ref = batch.JobBatch(m, jobs)
        ref.run()
        out = batch.JobBatch(m, jobs)
        stream = torch.cuda.current_stream()
        _dsp.dsp_expand_leaves_noalloc(m.h, out.descs, len(jobs), stream.cuda_stream)
        torch.cuda.synchronize()
        _, status = m.counters()
        assert status == 0
        for k, (a, b) in enumerate(zip(_results(ref), _results(out))):
            for f in FIELDS:
                assert np.array_equal(a[f], b[f]), (call, k, f)
    m.close()


def test_noalloc_rejects_oversize(env):
    """A call needing more than 2^20 (action, scenario) items is refused with a
    message naming the limit, and nothing runs."""
    torch, _dsp, batch = env
    cfg = I.mars15_15()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 8, 5, min_scen=500, max_scen=500)  # 8 * 500 * 400 = 1.6e6 items
    jb = batch.JobBatch(m, jobs[:1])
    descs = (type(jb.descs[0]) * len(jobs))(*([jb.descs[0]] * len(jobs)))
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_expand_leaves_noalloc(m.h, descs, len(jobs), 0)
    assert e.value.status == _dsp.DSP_E_UNSUPPORTED
    assert "at most" in str(e.value)
    m.close()


def _weights(_dsp):
    from paper_1802_06215_b300 import learn
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    h, _ = learn.load_weights(os.path.join(root, "paper_1802_06215_b300", "weights", "rs15_15_pi0.npz"))
    return h


def test_noalloc_learned_policy_twice_without_allocating(env):
    """With the learned default policy installed (tensor-core rollouts on the
    shared scratch), two calls in a row equal dsp_expand_leaves bit for bit,
    and after the first call's set-up the device's free memory does not move."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    h = _weights(_dsp)
    _dsp.dsp_set_policy(m.h, h)
    stream = torch.cuda.current_stream()
    warm = batch.JobBatch(m, I.job_stream(cfg, 4, 40))
    _dsp.dsp_expand_leaves_noalloc(m.h, warm.descs, len(warm.jobs), stream.cuda_stream)
    torch.cuda.synchronize()
    for call, seed in enumerate((41, 42)):
        jobs = I.job_stream(cfg, 16, seed)
        ref = batch.JobBatch(m, jobs)
        ref.run()
        out = batch.JobBatch(m, jobs)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        _dsp.dsp_expand_leaves_noalloc(m.h, out.descs, len(jobs), stream.cuda_stream)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call
        _, status = m.counters()
        assert status == 0
        for k, (a, b) in enumerate(zip(_results(ref), _results(out))):
            for f in FIELDS:
                assert np.array_equal(a[f], b[f]), (call, k, f)
    _dsp.dsp_mlp_destroy(h)
    m.close()


def test_noalloc_does_not_wait_for_earlier_work(env):
    """Behind a ~0.2 s kernel already queued on the stream, the call returns
    at once (its copy source is page-locked), and its results are still right."""
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 8, 43)
    ref = batch.JobBatch(m, jobs)
    ref.run()
    out = batch.JobBatch(m, jobs)
    stream = torch.cuda.current_stream()
    _dsp.dsp_expand_leaves_noalloc(m.h, out.descs, len(jobs), stream.cuda_stream)
    torch.cuda.synchronize()
    out = batch.JobBatch(m, jobs)
    torch.cuda.synchronize()
    ev = torch.cuda.Event()
    torch.cuda._sleep(int(0.2 * 2.0e9))
    ev.record(stream)
    t0 = time.perf_counter()
    _dsp.dsp_expand_leaves_noalloc(m.h, out.descs, len(jobs), stream.cuda_stream)
    dt = time.perf_counter() - t0
    busy = not ev.query()
    torch.cuda.synchronize()
    assert busy and dt < 0.05, (busy, dt)
    for k, (a, b) in enumerate(zip(_results(ref), _results(out))):
        for f in FIELDS:
            assert np.array_equal(a[f], b[f]), (k, f)
    m.close()


def test_noalloc_refuses_while_timing(env):
    torch, _dsp, batch = env
    cfg = I.rs15_15()
    m = batch.Model(cfg)
    jb = batch.JobBatch(m, I.job_stream(cfg, 2, 44))
    _dsp.dsp_kernel_timing(m.h, 1)
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_expand_leaves_noalloc(m.h, jb.descs, 2, 0)
    assert e.value.status == _dsp.DSP_E_UNSUPPORTED
    _dsp.dsp_kernel_timing(m.h, 0)
    m.close()
