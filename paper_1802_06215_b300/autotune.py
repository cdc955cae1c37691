"""Autotuner cache: the launch shape dsp_autotune_shape measured, kept per
(model, K, |A|, horizon, GPU) in a JSON file so later runs reuse it.

The measuring itself runs in the CUDA library (dsp_autotune_shape: the
rollout phase's CTA size and CTAs per SM, the grouping phase's warps per CTA,
the car's lanes per scenario and CTAs per SM, one-robot Rock Sample's
rollout-phase form); this module only builds the
cache key and reads and writes the file.
"""
import ctypes as C
import json
import os

from . import _dsp


def cache_key(cfg, num_actions, gpu_name):
    return (f"kind{cfg.kind}-n{cfg.n}-m{cfg.m}-P{cfg.P}-K{cfg.K}-D{cfg.D}-A{num_actions}-"
            f"{gpu_name.replace(' ', '_')}")


def _load(path):
    if path and os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def _store(path, cache):
    if not path:
        return
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def dsp_autotune(h, jobs_array, n_jobs, reps=5, stream=0):
    """The library's narrower tuner (rollout CTA size, car lanes per scenario)."""
    L = _dsp.lib()
    L.dsp_autotune.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_float)]
    b, t, ms = C.c_int32(0), C.c_int32(0), C.c_float(0)
    _dsp.check(L.dsp_autotune(h, C.cast(jobs_array, C.c_void_p), n_jobs, reps, C.c_void_p(stream), C.byref(b),
                              C.byref(t), C.byref(ms)))
    return {"block": b.value, "tps": t.value, "ms": ms.value}


def autotune(model, batch, gpu_name, cache_path=None, reps=3, measure=None):
    """Sets the model's launch shape from the cache, or measures it on `batch`
    (a JobBatch) and stores it. `measure(model, batch, reps)` replaces the
    library call (for tests of the cache); it returns the shape fields and
    "ms". Returns the shape with "cached"."""
    key = cache_key(model.cfg, model.num_actions, gpu_name)
    cache = _load(cache_path)
    if key in cache:
        best = cache[key]
        _dsp.dsp_set_launch_shape(model.h, **{k: best.get(k, 0) for k in _dsp.SHAPE_FIELDS})
        return dict(best, cached=True)
    if measure is None:
        best = _dsp.dsp_autotune_shape(model.h, batch.descs, len(batch.jobs), reps)
    else:
        best = measure(model, batch, reps)
        _dsp.dsp_set_launch_shape(model.h, **{k: best.get(k, 0) for k in _dsp.SHAPE_FIELDS})
    cache[key] = {k: best.get(k, 0) for k in _dsp.SHAPE_FIELDS + ("ms", "default_ms")}
    _store(cache_path, cache)
    return dict(best, cached=False)
