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

    monkeypatch.setattr(_dsp, "dsp_set_tuning", lambda h, b, t: calls.append((b, t)))

    def measure(model, batch, reps):
        return {"block": 512, "tps": 16, "ms": 1.5}

    path = str(tmp_path / "tune.json")
    r1 = autotune.autotune(FakeModel(), None, "NVIDIA B300", path, measure=measure)
    assert r1["cached"] is False and r1["block"] == 512
    data = json.load(open(path))
    key = autotune.cache_key(FakeModel.cfg, 20, "NVIDIA B300")
    assert data[key]["block"] == 512 and "B300" in key and "K500" in key
    r2 = autotune.autotune(FakeModel(), None, "NVIDIA B300", path, measure=None)
    assert r2["cached"] is True and calls[-1] == (512, 16)
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
    assert best["ms"] > 0
    assert _dsp.dsp_get_tuning(m.h) == (best["block"], best["tps"])
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
