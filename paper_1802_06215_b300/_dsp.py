"""ctypes binding of libdsp.so (include/dsp.h): same names, argument marshalling only.

Every computation runs in the CUDA library; this module only converts Python
values and torch tensor addresses into the C arguments. It fails loudly when
the library has not been built: there is no CPU fallback.
"""
import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdsp.so")

DSP_OK, DSP_E_INVALID, DSP_E_OOM, DSP_E_CUDA, DSP_E_TIMEOUT, DSP_E_QUEUE_FULL, DSP_E_UNSUPPORTED, DSP_E_DEVICE = range(8)
STATUS_NAMES = ["DSP_OK", "DSP_E_INVALID", "DSP_E_OOM", "DSP_E_CUDA", "DSP_E_TIMEOUT", "DSP_E_QUEUE_FULL",
                "DSP_E_UNSUPPORTED", "DSP_E_DEVICE"]


class DspError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


class dsp_model_desc(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("P", C.c_int32), ("gamma", C.c_float),
        ("K", C.c_int32), ("D", C.c_int32), ("seed", C.c_uint64), ("plan_step", C.c_uint32),
        ("rock_cells", C.POINTER(C.c_int32)), ("path_len", C.c_float), ("dt", C.c_float),
        ("ped_speed", C.c_float), ("sigma", C.c_float), ("fail_p", C.c_double), ("sense_p", C.c_double),
    ]


class dsp_leaf_job(C.Structure):
    _fields_ = [
        ("parent", C.c_void_p), ("parent_cap", C.c_int32), ("n_scen", C.c_int32), ("idx", C.c_void_p),
        ("last_action", C.c_int32), ("depth", C.c_int32), ("hist", C.c_int8 * 32),
        ("first_action", C.c_int32), ("n_actions", C.c_int32), ("child_cap", C.c_int32),
        ("leaf_states", C.c_void_p), ("child_count", C.c_void_p), ("child_off", C.c_void_p),
        ("child_key", C.c_void_p), ("rew_sum", C.c_void_p), ("u_sum", C.c_void_p), ("l_sum", C.c_void_p),
        ("perm", C.c_void_p),
    ]


_lib = None


def lib():
    """The loaded library; raises if libdsp.so is missing (build it with
    paper_1802_06215_b300.build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -m paper_1802_06215_b300.build)")
        L = C.CDLL(LIB_PATH)
        L.dsp_last_error.restype = C.c_char_p
        L.dsp_create_model.argtypes = [C.POINTER(dsp_model_desc), C.POINTER(C.c_void_p)]
        L.dsp_destroy_model.argtypes = [C.c_void_p]
        L.dsp_destroy_model.restype = None
        for f in ("dsp_state_words", "dsp_num_actions"):
            getattr(L, f).argtypes = [C.c_void_p]
            getattr(L, f).restype = C.c_int32
        L.dsp_max_children.argtypes = [C.c_void_p, C.c_int32]
        L.dsp_max_children.restype = C.c_int32
        L.dsp_set_plan_step.argtypes = [C.c_void_p, C.c_uint32]
        L.dsp_get_table.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32)]
        L.dsp_step.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                               C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
        L.dsp_rollout.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                  C.c_void_p]
        L.dsp_expand_leaves.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.dsp_read_counters.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
        L.dsp_reset_counters.argtypes = [C.c_void_p, C.c_void_p]
        L.dsp_alu_probe.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.c_void_p]
        L.dsp_expand_leaves_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
        L.dsp_set_tuning.argtypes = [C.c_void_p, C.c_int32, C.c_int32]
        L.dsp_get_tuning.argtypes = [C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
        _lib = L
    return _lib


def check(status):
    if status != DSP_OK:
        raise DspError(status, lib().dsp_last_error().decode())


def dsp_last_error():
    return lib().dsp_last_error().decode()


def desc_from_config(cfg):
    import numpy as np
    rocks = np.ascontiguousarray(cfg.rock_cells if cfg.rock_cells is not None else np.zeros(1), dtype=np.int32)
    d = dsp_model_desc(kind=cfg.kind, n=cfg.n, m=cfg.m, P=cfg.P, gamma=cfg.gamma, K=cfg.K, D=cfg.D, seed=cfg.seed,
                       plan_step=cfg.plan_step, rock_cells=rocks.ctypes.data_as(C.POINTER(C.c_int32)),
                       path_len=cfg.path_len, dt=cfg.dt, ped_speed=cfg.ped_speed, sigma=cfg.sigma,
                       fail_p=cfg.fail_p, sense_p=getattr(cfg, "sense_p", 0.03))
    d._keep = rocks
    return d


def dsp_create_model(desc):
    h = C.c_void_p()
    check(lib().dsp_create_model(C.byref(desc), C.byref(h)))
    return h


def dsp_destroy_model(h):
    lib().dsp_destroy_model(h)


def dsp_state_words(h):
    return lib().dsp_state_words(h)


def dsp_num_actions(h):
    return lib().dsp_num_actions(h)


def dsp_max_children(h, n_scen):
    return lib().dsp_max_children(h, n_scen)


def dsp_set_plan_step(h, plan_step):
    check(lib().dsp_set_plan_step(h, plan_step))


def dsp_get_table(h, which, out_ptr):
    cnt = C.c_int32(0)
    check(lib().dsp_get_table(h, which, C.c_void_p(out_ptr), C.byref(cnt)))
    return cnt.value


def dsp_step(h, in_block, in_cap, count, actions, depth, out_block, out_cap, obs_key, reward, stream=0):
    check(lib().dsp_step(h, C.c_void_p(in_block), in_cap, count, C.c_void_p(actions), depth, C.c_void_p(out_block),
                         out_cap, C.c_void_p(obs_key), C.c_void_p(reward), C.c_void_p(stream)))


def dsp_rollout(h, block, cap, count, hist, start_depth, value, stream=0):
    check(lib().dsp_rollout(h, C.c_void_p(block), cap, count, C.c_void_p(hist), start_depth, C.c_void_p(value),
                            C.c_void_p(stream)))


def dsp_expand_leaves(h, jobs_array, n_jobs, stream=0):
    check(lib().dsp_expand_leaves(h, C.cast(jobs_array, C.c_void_p), n_jobs, C.c_void_p(stream)))


def dsp_expand_leaves_noalloc(h, jobs_array, n_jobs, stream=0):
    """dsp_expand_leaves without device allocation (fixed library scratch;
    limits and sharing rules in include/dsp.h)."""
    check(lib().dsp_expand_leaves_noalloc(h, C.cast(jobs_array, C.c_void_p), n_jobs, C.c_void_p(stream)))


def dsp_read_counters(h):
    s = C.c_uint64(0)
    st = C.c_uint32(0)
    check(lib().dsp_read_counters(h, C.byref(s), C.byref(st)))
    return s.value, st.value


def dsp_reset_counters(h, stream=0):
    check(lib().dsp_reset_counters(h, C.c_void_p(stream)))


def dsp_set_tuning(h, block, tps):
    check(lib().dsp_set_tuning(h, block, tps))


class dsp_launch_shape(C.Structure):
    _fields_ = [("block_b", C.c_int32), ("ctas_b", C.c_int32), ("warps_a", C.c_int32), ("tps", C.c_int32),
                ("ctas_car", C.c_int32), ("rs_form", C.c_int32)]


SHAPE_FIELDS = tuple(f for f, _ in dsp_launch_shape._fields_)


def dsp_set_launch_shape(h, **shape):
    """Fields of dsp_launch_shape (missing ones 0 = default)."""
    s = dsp_launch_shape(**{k: int(shape.get(k, 0)) for k in SHAPE_FIELDS})
    L = lib()
    L.dsp_set_launch_shape.argtypes = [C.c_void_p, C.POINTER(dsp_launch_shape)]
    check(L.dsp_set_launch_shape(h, C.byref(s)))


def dsp_get_launch_shape(h):
    s = dsp_launch_shape()
    L = lib()
    L.dsp_get_launch_shape.argtypes = [C.c_void_p, C.POINTER(dsp_launch_shape)]
    check(L.dsp_get_launch_shape(h, C.byref(s)))
    return {k: getattr(s, k) for k in SHAPE_FIELDS}


def dsp_autotune_shape(h, jobs_array, n_jobs, reps=3, stream=0):
    """Times the default and every candidate launch shape on the jobs, keeps
    the fastest in the model; returns {shape fields..., ms, default_ms, tried}."""
    best = dsp_launch_shape()
    bms, dms, tried = C.c_float(0), C.c_float(0), C.c_int32(0)
    L = lib()
    L.dsp_autotune_shape.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                     C.POINTER(dsp_launch_shape), C.POINTER(C.c_float), C.POINTER(C.c_float),
                                     C.POINTER(C.c_int32)]
    check(L.dsp_autotune_shape(h, C.cast(jobs_array, C.c_void_p), n_jobs, reps, C.c_void_p(stream), C.byref(best),
                               C.byref(bms), C.byref(dms), C.byref(tried)))
    out = {k: getattr(best, k) for k in SHAPE_FIELDS}
    out.update(ms=bms.value, default_ms=dms.value, tried=tried.value)
    return out


def dsp_get_tuning(h):
    b, t = C.c_int32(0), C.c_int32(0)
    check(lib().dsp_get_tuning(h, C.byref(b), C.byref(t)))
    return b.value, t.value


def dsp_alu_probe(sink, iters, stream=0):
    ops = C.c_double(0)
    check(lib().dsp_alu_probe(C.c_void_p(sink), iters, C.byref(ops), C.c_void_p(stream)))
    return ops.value


class dsp_search_params(C.Structure):
    _fields_ = [("threads", C.c_int32), ("rounds", C.c_int32), ("time_limit_s", C.c_double), ("c_a", C.c_double),
                ("c_o", C.c_double), ("xi", C.c_double), ("target_gap", C.c_double), ("deterministic", C.c_int32),
                ("use_queue", C.c_int32), ("tree_lock", C.c_int32), ("batch", C.c_int32)]


class dsp_search_result(C.Structure):
    _fields_ = [("root_u", C.c_double), ("root_l", C.c_double), ("action", C.c_int32), ("nodes", C.c_int32),
                ("expansions", C.c_int32), ("rounds", C.c_int32), ("scenario_steps", C.c_uint64),
                ("signature", C.c_uint64), ("seconds", C.c_double)]


def dsp_plan(h, root_states, hist, params, num_actions):
    """root_states: numpy uint32 (words, n); hist: numpy int8[32] or None."""
    import numpy as np
    rs = np.ascontiguousarray(root_states, dtype=np.uint32)
    n = rs.shape[1]
    hs = None if hist is None else np.ascontiguousarray(hist, dtype=np.int8)
    res = dsp_search_result()
    visits = np.zeros(num_actions, np.int32)
    L = lib()
    L.dsp_plan.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(dsp_search_params),
                           C.POINTER(dsp_search_result), C.c_void_p]
    check(L.dsp_plan(h, rs.ctypes.data, n, None if hs is None else hs.ctypes.data, C.byref(params), C.byref(res),
                     visits.ctypes.data))
    out = {f: getattr(res, f) for f, _ in dsp_search_result._fields_}
    out["root_visits"] = visits
    return out


def dsp_plan_multi(hs, root_states, hist, params, num_actions):
    """dsp_plan with leaf expansions routed over several models (one per GPU);
    hs: list of model handles."""
    import numpy as np
    rs = np.ascontiguousarray(root_states, dtype=np.uint32)
    n = rs.shape[1]
    hv = None if hist is None else np.ascontiguousarray(hist, dtype=np.int8)
    arr = (C.c_void_p * len(hs))(*hs)
    res = dsp_search_result()
    visits = np.zeros(num_actions, np.int32)
    L = lib()
    L.dsp_plan_multi.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p,
                                 C.POINTER(dsp_search_params), C.POINTER(dsp_search_result), C.c_void_p]
    check(L.dsp_plan_multi(C.cast(arr, C.c_void_p), len(hs), rs.ctypes.data, n,
                           None if hv is None else hv.ctypes.data, C.byref(params), C.byref(res),
                           visits.ctypes.data))
    out = {f: getattr(res, f) for f, _ in dsp_search_result._fields_}
    out["root_visits"] = visits
    return out


def dsp_route_leaves(n_models, first_expansion, parent_model):
    """(target model, copy flag) per leaf: the host-only routing rule of
    dsp_plan_multi."""
    import numpy as np
    pm = np.ascontiguousarray(parent_model, dtype=np.int32)
    k = len(pm)
    tgt = np.zeros(k, np.int32)
    cp = np.zeros(k, np.int32)
    L = lib()
    L.dsp_route_leaves.argtypes = [C.c_int32, C.c_int64, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    check(L.dsp_route_leaves(k, first_expansion, n_models, pm.ctypes.data, tgt.ctypes.data, cp.ctypes.data))
    return tgt, cp


class dsp_pomcp_params(C.Structure):
    _fields_ = [("rounds", C.c_int32), ("batch", C.c_int32), ("c", C.c_double), ("time_limit_s", C.c_double)]


class dsp_pomcp_result(C.Structure):
    _fields_ = [("action", C.c_int32), ("value", C.c_double), ("nodes", C.c_int32), ("simulations", C.c_int32),
                ("rollouts", C.c_int32), ("rounds", C.c_int32), ("scenario_steps", C.c_uint64),
                ("signature", C.c_uint64), ("seconds", C.c_double)]


def dsp_pomcp_plan(h, root_states, hist, params, num_actions):
    """POMCP-style planning; root_states: numpy uint32 (words, n); hist: numpy int8[32] or None."""
    import numpy as np
    rs = np.ascontiguousarray(root_states, dtype=np.uint32)
    n = rs.shape[1]
    hs = None if hist is None else np.ascontiguousarray(hist, dtype=np.int8)
    res = dsp_pomcp_result()
    q = np.zeros(num_actions, np.float64)
    na = np.zeros(num_actions, np.int32)
    L = lib()
    L.dsp_pomcp_plan.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(dsp_pomcp_params),
                                 C.POINTER(dsp_pomcp_result), C.c_void_p, C.c_void_p]
    check(L.dsp_pomcp_plan(h, rs.ctypes.data, n, None if hs is None else hs.ctypes.data, C.byref(params),
                           C.byref(res), q.ctypes.data, na.ctypes.data))
    out = {f: getattr(res, f) for f, _ in dsp_pomcp_result._fields_}
    out["root_q"] = q
    out["root_na"] = na
    return out


def dsp_queue_create(h, capacity, idle_ns=0):
    L = lib()
    L.dsp_queue_create.argtypes = [C.c_void_p, C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]
    q = C.c_void_p()
    check(L.dsp_queue_create(h, capacity, idle_ns, C.byref(q)))
    return q


def dsp_queue_submit(q, job, timeout_ns=0):
    """job: a dsp_leaf_job (device pointers); returns the ticket."""
    L = lib()
    L.dsp_queue_submit.argtypes = [C.c_void_p, C.POINTER(dsp_leaf_job), C.c_uint64, C.POINTER(C.c_uint64)]
    t = C.c_uint64(0)
    check(L.dsp_queue_submit(q, C.byref(job), timeout_ns, C.byref(t)))
    return t.value


def dsp_queue_wait(q, ticket, timeout_ns=0):
    L = lib()
    L.dsp_queue_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_uint64]
    check(L.dsp_queue_wait(q, ticket, timeout_ns))


def dsp_queue_stats(q):
    L = lib()
    L.dsp_queue_stats.argtypes = [C.c_void_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
    a, b = C.c_uint64(0), C.c_uint64(0)
    check(L.dsp_queue_stats(q, C.byref(a), C.byref(b)))
    return a.value, b.value


def dsp_queue_destroy(q):
    L = lib()
    L.dsp_queue_destroy.argtypes = [C.c_void_p]
    L.dsp_queue_destroy.restype = None
    L.dsp_queue_destroy(q)


def dsp_kernel_timing(h, enable):
    """(summed ms of the expansion kernels recorded so far, calls); then
    recording is switched on or off."""
    L = lib()
    L.dsp_kernel_timing.argtypes = [C.c_void_p, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int32)]
    ms, n = C.c_double(0), C.c_int32(0)
    check(L.dsp_kernel_timing(h, 1 if enable else 0, C.byref(ms), C.byref(n)))
    return ms.value, n.value


MLP_PARAMS = 64 * 256 + 256 + 256 * 256 + 256 + 256 * 32 + 32
MLP_SHAPES = (("W1", (64, 256)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 32)),
              ("b3", (32,)))


def pack_params(w):
    import numpy as np
    return np.concatenate([np.asarray(w[k], np.float32).reshape(-1) for k, _ in MLP_SHAPES])


def unpack_params(flat):
    out, o = {}, 0
    for k, shp in MLP_SHAPES:
        n = 1
        for s in shp:
            n *= s
        out[k] = flat[o:o + n].reshape(shp)
        o += n
    return out


def dsp_mlp_create(max_batch, seed):
    L = lib()
    L.dsp_mlp_create.argtypes = [C.c_int32, C.c_uint64, C.POINTER(C.c_void_p)]
    h = C.c_void_p()
    check(L.dsp_mlp_create(max_batch, seed, C.byref(h)))
    return h


def dsp_mlp_destroy(h):
    L = lib()
    L.dsp_mlp_destroy.argtypes = [C.c_void_p]
    L.dsp_mlp_destroy.restype = None
    L.dsp_mlp_destroy(h)


def dsp_mlp_set_weights(h, flat):
    import numpy as np
    a = np.ascontiguousarray(flat, np.float32)
    L = lib()
    L.dsp_mlp_set_weights.argtypes = [C.c_void_p, C.c_void_p]
    check(L.dsp_mlp_set_weights(h, a.ctypes.data))


def dsp_mlp_get_weights(h):
    import numpy as np
    a = np.zeros(MLP_PARAMS, np.float32)
    L = lib()
    L.dsp_mlp_get_weights.argtypes = [C.c_void_p, C.c_void_p]
    check(L.dsp_mlp_get_weights(h, a.ctypes.data))
    return a


def dsp_mlp_forward(h, X_ptr, B, logits_ptr, stream=0):
    L = lib()
    L.dsp_mlp_forward.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
    check(L.dsp_mlp_forward(h, C.c_void_p(X_ptr), B, C.c_void_p(logits_ptr), C.c_void_p(stream)))


def dsp_mlp_grad(h, X_ptr, y_ptr, B, n_actions, stream=0):
    import numpy as np
    g = np.zeros(MLP_PARAMS, np.float32)
    loss = C.c_float(0)
    L = lib()
    L.dsp_mlp_grad.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.POINTER(C.c_float),
                               C.c_void_p, C.c_void_p]
    check(L.dsp_mlp_grad(h, C.c_void_p(X_ptr), C.c_void_p(y_ptr), B, n_actions, C.byref(loss), g.ctypes.data,
                         C.c_void_p(stream)))
    return loss.value, g


def dsp_mlp_train_step(h, X_ptr, y_ptr, B, n_actions, lr, stream=0):
    loss = C.c_float(0)
    L = lib()
    L.dsp_mlp_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_float,
                                     C.POINTER(C.c_float), C.c_void_p]
    check(L.dsp_mlp_train_step(h, C.c_void_p(X_ptr), C.c_void_p(y_ptr), B, n_actions, lr, C.byref(loss),
                               C.c_void_p(stream)))
    return loss.value


def dsp_set_policy(model_h, mlp_h):
    """Makes the MLP's current weights the model's rollout policy (copied; a
    null mlp_h returns the model to the heuristic policy)."""
    L = lib()
    L.dsp_set_policy.argtypes = [C.c_void_p, C.c_void_p]
    check(L.dsp_set_policy(model_h, mlp_h))


def default_policy(model_h, block, hist=None, want_allowed=False):
    """dsp_default_policy on host arrays: block (words, count) uint32, hist
    (count, 32) int8 or None. Returns actions (count,) int32 and, with
    want_allowed, the allowed-action bits (count,) uint32."""
    import numpy as np
    import torch
    b = np.ascontiguousarray(block, dtype=np.uint32)
    count = b.shape[1]
    bd = torch.tensor(b.view(np.int32), device="cuda")
    hd = None if hist is None else torch.tensor(np.ascontiguousarray(hist, dtype=np.int8).reshape(count, 32),
                                                 device="cuda")
    act = torch.zeros(count, dtype=torch.int32, device="cuda")
    al = torch.zeros(count, dtype=torch.int32, device="cuda") if want_allowed else None
    L = lib()
    L.dsp_default_policy.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_void_p]
    st = torch.cuda.current_stream().cuda_stream
    check(L.dsp_default_policy(model_h, C.c_void_p(bd.data_ptr()), count, count,
                               C.c_void_p(hd.data_ptr() if hd is not None else None), C.c_void_p(act.data_ptr()),
                               C.c_void_p(al.data_ptr() if al is not None else None), C.c_void_p(st)))
    torch.cuda.synchronize()
    if want_allowed:
        return act.cpu().numpy(), al.cpu().numpy().view(np.uint32)
    return act.cpu().numpy()


def dsp_rollout_logged(model_h, block_ptr, cap, count, hist_ptr, start_depth, value_ptr, actions_ptr=0, stream=0,
                       logits_ptr=0):
    """dsp_rollout with the learned policy; actions (device count x D int32)
    receives the action of every step, logits (device count x D x 32 FP32)
    the tensor-core tile's logits of every step; entries after a rollout
    ends are left untouched."""
    L = lib()
    L.dsp_rollout_logged.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32,
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    check(L.dsp_rollout_logged(model_h, C.c_void_p(block_ptr), cap, count, C.c_void_p(hist_ptr), start_depth,
                               C.c_void_p(value_ptr), C.c_void_p(actions_ptr or None), C.c_void_p(logits_ptr or None),
                               C.c_void_p(stream)))


class dsp_plan_node(C.Structure):
    _fields_ = [("depth", C.c_int32), ("n", C.c_int32), ("action", C.c_int32), ("visits", C.c_int32),
                ("U", C.c_double), ("L", C.c_double), ("hist", C.c_int8 * 32)]


def dsp_plan_nodes(h, root_states, hist, params, num_actions, min_scen, cap, words):
    """dsp_plan plus the export of the tree's expanded nodes: returns the plan
    result dict, a list-free numpy view of the nodes (depth, n, action,
    visits, U, L, hist) and the (words, count) block of their first states."""
    import numpy as np
    rs = np.ascontiguousarray(root_states, dtype=np.uint32)
    n = rs.shape[1]
    hs = None if hist is None else np.ascontiguousarray(hist, dtype=np.int8)
    res = dsp_search_result()
    visits = np.zeros(num_actions, np.int32)
    nodes = (dsp_plan_node * cap)()
    states = np.zeros((words, cap), np.uint32)
    count = C.c_int32(0)
    L = lib()
    L.dsp_plan_nodes.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(dsp_search_params),
                                 C.POINTER(dsp_search_result), C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                 C.c_void_p, C.POINTER(C.c_int32)]
    check(L.dsp_plan_nodes(h, rs.ctypes.data, n, None if hs is None else hs.ctypes.data, C.byref(params),
                           C.byref(res), visits.ctypes.data, min_scen, cap, nodes, states.ctypes.data,
                           C.byref(count)))
    k = count.value
    rec = np.frombuffer(nodes, dtype=np.dtype([("depth", "<i4"), ("n", "<i4"), ("action", "<i4"),
                                               ("visits", "<i4"), ("U", "<f8"), ("L", "<f8"),
                                               ("hist", "i1", 32)]), count=k).copy()
    out = {f: getattr(res, f) for f, _ in dsp_search_result._fields_}
    out["root_visits"] = visits
    return out, rec, np.ascontiguousarray(states[:, :k])


def dsp_features(h, block_ptr, cap, count, hist_ptr, out_ptr, stream=0):
    L = lib()
    L.dsp_features.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    check(L.dsp_features(h, C.c_void_p(block_ptr), cap, count, C.c_void_p(hist_ptr), C.c_void_p(out_ptr),
                         C.c_void_p(stream)))
