"""Autotuner: the cache round trip (host logic, no GPU) and, on the GPU, that
the chosen launch shape keeps the oracle's results."""
import json

import numpy as np
import pytest

import oracle
from paper_1802_06215_b300 import inputs as I


def test_cache_key_and_roundtrip(tmp_path, monkeypatch):
    from paper_1802_06215_b300 import _dsp, autotune
    calls = []

    class FakeModel:
        cfg = I.rs15_15()
        num_actions = 20
        h = None

    monkeypatch.setattr(_dsp, "dsp_set_launch_shape", lambda h, **kw: calls.append(kw))

    def measure(model, batch, reps):
        return {"block_b": 512, "ctas_b": 4, "warps_a": 10, "tps": 0, "ctas_car": 0, "rs_form": 2, "ms": 1.5,
                "default_ms": 1.7}

    path = str(tmp_path / "tune.json")
    r1 = autotune.autotune(FakeModel(), None, "NVIDIA B300", path, measure=measure)
    assert r1["cached"] is False and r1["block_b"] == 512
    data = json.load(open(path))
    key = autotune.cache_key(FakeModel.cfg, 20, "NVIDIA B300")
    assert data[key]["block_b"] == 512 and data[key]["warps_a"] == 10 and "B300" in key and "K500" in key
    r2 = autotune.autotune(FakeModel(), None, "NVIDIA B300", path, measure=None)
    assert r2["cached"] is True and calls[-1] == {"block_b": 512, "ctas_b": 4, "warps_a": 10, "tps": 0,
                                                  "ctas_car": 0, "rs_form": 2}
    # another GPU name is another entry
    r3 = autotune.autotune(FakeModel(), None, "other GPU", path, measure=measure)
    assert r3["cached"] is False and len(json.load(open(path))) == 2


@pytest.mark.gpu
@pytest.mark.parametrize("mk", [I.rs15_15, I.car50])
def test_autotune_keeps_results(mk, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, autotune, batch, build
    build.build()
    cfg = mk()
    m = batch.Model(cfg)
    jobs = I.job_stream(cfg, 64 if cfg.kind != I.CAR else 16, 3)
    jb = batch.JobBatch(m, jobs)
    best = autotune.autotune(m, jb, torch.cuda.get_device_name(), str(tmp_path / "t.json"), reps=2)
    assert best["ms"] > 0 and best["ms"] <= best["default_ms"] and best["tried"] > 1
    got = _dsp.dsp_get_launch_shape(m.h)
    assert got == {k: best[k] for k in _dsp.SHAPE_FIELDS}
    jb.run()
    _, status = m.counters()
    assert status == 0
    om = oracle.Model(cfg)
    res = jb.all_results()
    for k in (0, len(jobs) - 1):
        j = jobs[k]
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        assert np.array_equal(res[k]["perm"], o["perm"])
        for a in range(len(o["child_count"])):
            nc = int(o["child_count"][a])
            assert np.array_equal(res[k]["l"][a][:nc], o["l"][a][:nc])
    m.close()


SHAPES = [
    ("rs15_15", dict(block_b=128, ctas_b=4, warps_a=10)),
    ("rs15_15", dict(block_b=512, ctas_b=6, warps_a=5)),
    ("rs15_15", dict(block_b=256, ctas_b=1, warps_a=1)),
    ("mars15_15", dict(block_b=128, warps_a=8)),
    ("mars15_15", dict(block_b=512, ctas_b=2, warps_a=16)),
    ("car50", dict(tps=8, ctas_car=2)),
    ("car50", dict(tps=16, ctas_car=1)),
    ("nav13", dict(ctas_b=2)),
]


@pytest.mark.gpu
@pytest.mark.parametrize("name,shape", SHAPES)
def test_launch_shapes_keep_oracle_results(name, shape):
    """Every launch shape the autotuner may pick gives the oracle's expansion
    bit for bit (children, perms, keys, and the exact sums)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    cfg = getattr(I, name)()
    m = batch.Model(cfg)
    _dsp.dsp_set_launch_shape(m.h, **shape)
    assert {k: v for k, v in _dsp.dsp_get_launch_shape(m.h).items() if v} == shape
    jobs = I.job_stream(cfg, 24 if cfg.kind in (I.GRID, I.NAV) else 6, 8, max_scen=200)
    jb = batch.JobBatch(m, jobs)
    jb.run()
    torch.cuda.synchronize()
    _, status = m.counters()
    assert status == 0
    om = oracle.Model(cfg)
    res = jb.all_results()
    for k, j in enumerate(jobs):
        o = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist, cap=m.max_children(len(j.idx)))
        g = res[k]
        assert np.array_equal(g["child_count"], o["child_count"]) and np.array_equal(g["perm"], o["perm"]), k
        for a in range(len(o["child_count"])):
            nc = int(o["child_count"][a])
            for f in ("key", "rew", "u", "l"):
                assert np.array_equal(g[f][a][:nc], o[f][a][:nc]), (k, a, f)
    with pytest.raises(_dsp.DspError):
        _dsp.dsp_set_launch_shape(m.h, block_b=100)
    m.close()
