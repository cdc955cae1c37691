"""CPU oracle of GPU leaf expansion — TEST INFRASTRUCTURE ONLY.

A plain, single-threaded restatement of the paper's method (DESPOT leaf
initialisation, Sec. III-A and III-D; the HyP-DESPOT tree search, Sec. III-C)
in C++ (`*.hpp`, `capi.cpp`, `mlp.cpp`), reached from Python through ctypes.
Only `tests/`, the package's smoke check and the benchmark's CPU-baseline leg
may import this package; the product library never calls it and shares no
code with it.

Parity status: every function here is pinned by tests under `tests/` marked
"not gpu" (closed forms, invariants, exhaustive enumeration, hand-worked
goldens); Philox4x32-10 by the generator's published known-answer vectors.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None


class _Model(C.Structure):
    _fields_ = [
        ("kind", C.c_int32), ("n", C.c_int32), ("m", C.c_int32), ("P", C.c_int32),
        ("gamma", C.c_float), ("K", C.c_int32), ("D", C.c_int32), ("seed", C.c_uint64),
        ("plan_step", C.c_uint32), ("rock_cells", C.POINTER(C.c_int32)),
        ("path_len", C.c_float), ("dt", C.c_float), ("ped_speed", C.c_float), ("sigma", C.c_float),
        ("fail_p", C.c_double), ("fp64", C.c_int32), ("sense_p", C.c_double),
    ]


class _SearchParams(C.Structure):
    _fields_ = [("threads", C.c_int32), ("rounds", C.c_int32), ("c_a", C.c_double), ("c_o", C.c_double),
                ("xi", C.c_double), ("target_gap", C.c_double)]


class _SearchResult(C.Structure):
    _fields_ = [("root_u", C.c_double), ("root_l", C.c_double), ("action", C.c_int32), ("nodes", C.c_int32),
                ("expansions", C.c_int32), ("rounds", C.c_int32), ("steps", C.c_uint64),
                ("signature", C.c_uint64)]


class _PomcpResult(C.Structure):
    _fields_ = [("action", C.c_int32), ("value", C.c_double), ("nodes", C.c_int32), ("simulations", C.c_int32),
                ("rollouts", C.c_int32), ("steps", C.c_uint64), ("signature", C.c_uint64)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


_U32, _U64, _I32, _I64, _U16, _I8, _F32, _F64 = (C.c_uint32, C.c_uint64, C.c_int32, C.c_int64, C.c_uint16,
                                                 C.c_int8, C.c_float, C.c_double)


def philox(ctr, k0, k1, rounds=10):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(_p(c, _U32), C.c_uint32(k0), C.c_uint32(k1), C.c_int32(rounds), _p(out, _U32))
    return out


def scenario_random(seed, scen, depth, purpose, element, plan_step):
    out = np.zeros(4, np.uint32)
    lib().orc_scenario_random(C.c_uint64(seed), C.c_uint32(scen), C.c_uint32(depth), C.c_uint32(purpose),
                              C.c_uint32(element), C.c_uint32(plan_step), _p(out, _U32))
    return out


def sensor_thresholds(max_d2):
    out = np.zeros(max_d2 + 1, np.uint64)
    lib().orc_sensor_thresholds(C.c_int32(max_d2), _p(out, _U64))
    return out


def gauss_table():
    o64 = np.zeros(4096, np.float64)
    o32 = np.zeros(4096, np.float32)
    lib().orc_gauss_table(_p(o64, _F64), _p(o32, _F32))
    return o64, o32


def gamma_powers(gamma, n):
    o32 = np.zeros(n, np.float32)
    o64 = np.zeros(n, np.float64)
    lib().orc_gamma_powers(C.c_float(gamma), C.c_int32(n), _p(o32, _F32), _p(o64, _F64))
    return o32, o64


class Model:
    """Oracle view of a model configuration (any object with the config fields)."""

    def __init__(self, cfg, fp64=False, plan_step=None):
        self.cfg = cfg
        self._rocks = np.ascontiguousarray(cfg.rock_cells if cfg.rock_cells is not None else np.zeros(1),
                                           dtype=np.int32)
        self.c = _Model(kind=cfg.kind, n=cfg.n, m=cfg.m, P=cfg.P, gamma=cfg.gamma, K=cfg.K, D=cfg.D,
                        seed=cfg.seed, plan_step=cfg.plan_step if plan_step is None else plan_step,
                        rock_cells=_p(self._rocks, _I32), path_len=cfg.path_len, dt=cfg.dt,
                        ped_speed=cfg.ped_speed, sigma=cfg.sigma, fail_p=cfg.fail_p, fp64=1 if fp64 else 0,
                        sense_p=getattr(cfg, "sense_p", 0.03))

    @property
    def words(self):
        return lib().orc_state_words(C.byref(self.c))

    def num_actions(self):
        if self.cfg.kind == 2:
            return 3
        if self.cfg.kind == 3:
            return 9
        a = 5 + self.cfg.m
        return a if self.cfg.kind == 0 else a * a

    def step(self, block, actions, depth):
        block = np.ascontiguousarray(block, np.uint32)
        w, cap = block.shape
        count = len(actions)
        out = np.zeros((w, count), np.uint32)
        keys = np.zeros(count, np.uint64)
        rew = np.zeros(count, np.float64)
        acts = np.ascontiguousarray(actions, np.int32)
        rc = lib().orc_step(C.byref(self.c), _p(block, _U32), C.c_int32(cap), C.c_int32(count), _p(acts, _I32),
                            C.c_int32(depth), _p(out, _U32), C.c_int32(count), _p(keys, _U64), _p(rew, _F64))
        assert rc == 0
        return out, keys, rew

    def rollout(self, block, hist, start_depth):
        block = np.ascontiguousarray(block, np.uint32)
        w, cap = block.shape
        vals = np.zeros(cap, np.float64)
        steps = C.c_uint64(0)
        h = None if hist is None else np.ascontiguousarray(hist, np.int8).reshape(cap, 32)
        rc = lib().orc_rollout(C.byref(self.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap),
                               None if h is None else _p(h, _I8), C.c_int32(start_depth), _p(vals, _F64),
                               C.byref(steps))
        assert rc == 0
        return vals, steps.value

    def bounds(self, block):
        block = np.ascontiguousarray(block, np.uint32)
        w, cap = block.shape
        u = np.zeros(cap, np.float64)
        t = np.zeros(cap, np.float64)
        assert lib().orc_bounds(C.byref(self.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap), _p(u, _F64),
                                _p(t, _F64)) == 0
        return u, t

    def policy(self, block, hist):
        block = np.ascontiguousarray(block, np.uint32)
        w, cap = block.shape
        acts = np.zeros(cap, np.int32)
        h = None if hist is None else np.ascontiguousarray(hist, np.int8).reshape(cap, 32)
        assert lib().orc_policy(C.byref(self.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap),
                                None if h is None else _p(h, _I8), _p(acts, _I32)) == 0
        return acts

    def expand(self, parent_block, idx, last_action, depth, hist, a0=0, na=None, cap=None):
        parent_block = np.ascontiguousarray(parent_block, np.uint32)
        w, pcap = parent_block.shape
        idx = np.ascontiguousarray(idx, np.uint16)
        n = len(idx)
        na = self.num_actions() if na is None else na
        cap = n if cap is None else cap
        h = np.zeros(32, np.int8) if hist is None else np.ascontiguousarray(hist, np.int8)
        leaf = np.zeros((w, n), np.uint32)
        cc = np.zeros(na, np.int32)
        co = np.zeros(na * (cap + 1), np.int32)
        key = np.zeros(na * cap, np.uint64)
        rew = np.zeros(na * cap, np.int64)
        u = np.zeros(na * cap, np.int64)
        l = np.zeros(na * cap, np.int64)
        perm = np.zeros(na * n, np.uint16)
        steps = C.c_uint64(0)
        rc = lib().orc_expand(C.byref(self.c), _p(parent_block, _U32), C.c_int32(pcap), C.c_int32(pcap),
                              _p(idx, _U16), C.c_int32(n), C.c_int32(last_action), C.c_int32(depth), _p(h, _I8),
                              C.c_int32(a0), C.c_int32(na), C.c_int32(cap), _p(leaf, _U32), _p(cc, _I32),
                              _p(co, _I32), _p(key, _U64), _p(rew, _I64), _p(u, _I64), _p(l, _I64),
                              _p(perm, _U16), C.byref(steps))
        assert rc == 0
        return dict(leaf=leaf, child_count=cc, child_off=co.reshape(na, cap + 1), key=key.reshape(na, cap),
                    rew=rew.reshape(na, cap), u=u.reshape(na, cap), l=l.reshape(na, cap),
                    perm=perm.reshape(na, n), steps=steps.value)

    def plan(self, root_block, hist, threads=1, rounds=100, c_a=0.0, c_o=0.0, xi=0.95, target_gap=0.0):
        root_block = np.ascontiguousarray(root_block, np.uint32)
        w, n = root_block.shape
        h = np.zeros(32, np.int8) if hist is None else np.ascontiguousarray(hist, np.int8)
        prm = _SearchParams(threads=threads, rounds=rounds, c_a=c_a, c_o=c_o, xi=xi, target_gap=target_gap)
        res = _SearchResult()
        na = np.zeros(self.num_actions(), np.int32)
        assert lib().orc_plan(C.byref(self.c), _p(root_block, _U32), C.c_int32(n), _p(h, _I8), C.byref(prm),
                              C.byref(res), _p(na, _I32)) == 0
        return dict(root_u=res.root_u, root_l=res.root_l, action=res.action, nodes=res.nodes,
                    expansions=res.expansions, rounds=res.rounds, steps=res.steps, signature=res.signature,
                    root_na=na)

    def pomcp(self, root_block, hist, rounds=10, batch=64, c=1.0):
        """POMCP-style planning from the root scenarios (oracle/pomcp.hpp)."""
        root_block = np.ascontiguousarray(root_block, np.uint32)
        w, n = root_block.shape
        h = np.zeros(32, np.int8) if hist is None else np.ascontiguousarray(hist, np.int8)
        na = self.num_actions()
        q = np.zeros(na, np.float64)
        nav = np.zeros(na, np.int32)
        out = _PomcpResult()
        rc = lib().orc_pomcp(C.byref(self.c), _p(root_block, _U32), C.c_int32(n), _p(h, _I8), C.c_int32(rounds),
                             C.c_int32(batch), C.c_double(c), C.byref(out), _p(q, _F64), _p(nav, _I32))
        assert rc == 0
        return dict(action=out.action, value=out.value, nodes=out.nodes, simulations=out.simulations,
                    rollouts=out.rollouts, steps=out.steps, signature=out.signature, root_q=q, root_na=nav)

    def exhaustive(self, block, hist, depth):
        block = np.ascontiguousarray(block, np.uint32)
        w, n = block.shape
        h = np.zeros(32, np.int8) if hist is None else np.ascontiguousarray(hist, np.int8)
        f = lib().orc_exhaustive
        f.restype = C.c_double
        return f(C.byref(self.c), _p(block, _U32), C.c_int32(n), _p(h, _I8), C.c_int32(depth))


def ops_reset():
    """Clears the op counter (op-counting mode: primitive operations of the
    model definitions, counted in the oracle's calls on this thread)."""
    lib().orc_ops_reset()


def ops_read():
    f = lib().orc_ops_read
    f.restype = C.c_uint64
    return int(f())


MLP_IN, MLP_HID, MLP_OUT = 64, 256, 32


def _w(weights):
    names = ("W1", "b1", "W2", "b2", "W3", "b3")
    arrs = [np.ascontiguousarray(weights[k], np.float64) for k in names]
    return arrs, [_p(a, _F64) for a in arrs]


def mlp_forward(weights, X, bf16=False):
    """Logits (B, 32) of the policy network; bf16=True: BF16 weights, features
    and activations with FP32 sums (the tensor-core arithmetic)."""
    keep, ptrs = _w(weights)
    X = np.ascontiguousarray(X, np.float64)
    out = np.zeros((X.shape[0], MLP_OUT), np.float64)
    lib().orc_mlp_forward(*ptrs, _p(X, _F64), C.c_int32(X.shape[0]), C.c_int32(1 if bf16 else 0), _p(out, _F64))
    return out


def mlp_loss_grad(weights, X, y, n_actions, bf16_forward=False):
    """Mean softmax cross-entropy and its FP64 gradient (dict like weights);
    bf16_forward=True evaluates it at the BF16/FP32 forward's activations."""
    keep, ptrs = _w(weights)
    X = np.ascontiguousarray(X, np.float64)
    y = np.ascontiguousarray(y, np.int32)
    g = {k: np.zeros_like(np.asarray(weights[k], np.float64)) for k in ("W1", "b1", "W2", "b2", "W3", "b3")}
    loss = C.c_double(0)
    lib().orc_mlp_loss_grad(*ptrs, _p(X, _F64), _p(y, _I32), C.c_int32(X.shape[0]), C.c_int32(n_actions),
                            C.byref(loss), *[_p(g[k], _F64) for k in ("W1", "b1", "W2", "b2", "W3", "b3")],
                            C.c_int32(1 if bf16_forward else 0))
    return loss.value, g


def features_rs(model, block, hist):
    block = np.ascontiguousarray(block, np.uint32)
    w, cap = block.shape
    h = None if hist is None else np.ascontiguousarray(hist, np.int8).reshape(cap, 32)
    out = np.zeros((cap, MLP_IN), np.float32)
    lib().orc_features_rs(C.byref(model.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap),
                          None if h is None else _p(h, _I8), _p(out, _F32))
    return out


def features_car(model, block):
    """Learned-policy features of car states (64 per state)."""
    block = np.ascontiguousarray(block, np.uint32)
    w, cap = block.shape
    out = np.zeros((cap, MLP_IN), np.float32)
    rc = lib().orc_features_car(C.byref(model.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap), _p(out, _F32))
    assert rc == 0
    return out


def learned_allowed(model, block, hist):
    """Bits of the actions the learned policy may take per one-robot Rock
    Sample state (bit |A|, defer, always set)."""
    block = np.ascontiguousarray(block, np.uint32)
    w, cap = block.shape
    h = None if hist is None else np.ascontiguousarray(hist, np.int8).reshape(cap, 32)
    out = np.zeros(cap, np.uint32)
    rc = lib().orc_learned_allowed(C.byref(model.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap),
                                   None if h is None else _p(h, _I8), _p(out, _U32))
    assert rc == 0
    return out


def rollout_learned(model, block, hist, start_depth, weights, logged=None, tol=1e-2, want_logits=False):
    """Learned-policy rollout values (one-robot Rock Sample or the car); with `logged` actions
    (count x D) it replays them and returns, per scenario, the steps whose
    logged action loses to the network's argmax by more than `tol`. With
    want_logits it also returns the logits of every step (count x D x 32,
    NaN after the rollout ends)."""
    block = np.ascontiguousarray(block, np.uint32)
    w, cap = block.shape
    h = None if hist is None else np.ascontiguousarray(hist, np.int8).reshape(cap, 32)
    keep, ptrs = _w(weights)
    vals = np.zeros(cap, np.float64)
    bad = np.zeros(cap, np.int32)
    lg = None if logged is None else np.ascontiguousarray(logged, np.int32)
    steps = C.c_uint64(0)
    lo = np.full((cap, model.cfg.D, MLP_OUT), np.nan) if want_logits else None
    rc = lib().orc_rollout_learned(C.byref(model.c), _p(block, _U32), C.c_int32(cap), C.c_int32(cap),
                                   None if h is None else _p(h, _I8), C.c_int32(start_depth), *ptrs,
                                   None if lg is None else _p(lg, _I32), C.c_double(tol), _p(vals, _F64),
                                   _p(bad, _I32), C.byref(steps), None if lo is None else _p(lo, _F64))
    assert rc == 0
    if want_logits:
        return vals, bad, steps.value, lo
    return vals, bad, steps.value
