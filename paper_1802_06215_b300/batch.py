"""Device-resident batches of leaf-expansion jobs for the C ABI.

Packs many jobs (parent state blocks, scenario indexes, result arrays) into one
device arena so that a single dsp_expand_leaves call expands them all; torch
provides the memory and the stream. Marshalling only: no step of the method
runs here.
"""
import ctypes as C

import numpy as np
import torch

from . import _dsp


def _align(x, a=256):
    return (x + a - 1) // a * a


class Model:
    """A dsp_model handle plus the sizes the binding needs."""

    def __init__(self, cfg):
        self.cfg = cfg
        self.desc = _dsp.desc_from_config(cfg)
        self.h = _dsp.dsp_create_model(self.desc)
        self.words = _dsp.dsp_state_words(self.h)
        self.num_actions = _dsp.dsp_num_actions(self.h)

    def close(self):
        if self.h:
            _dsp.dsp_destroy_model(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def max_children(self, n):
        return _dsp.dsp_max_children(self.h, n)

    def set_plan_step(self, k):
        _dsp.dsp_set_plan_step(self.h, k)

    def table(self, which):
        buf = np.zeros(8192, np.uint64)
        n = _dsp.dsp_get_table(self.h, which, buf.ctypes.data)
        if which == 0:
            return buf[:n].copy()
        return buf.view(np.float32)[:n].copy()

    def step(self, block, actions, depth, stream=None):
        """block: (words, cap) int32/uint32 tensor or array; returns numpy."""
        dev = torch.device("cuda")
        b = torch.as_tensor(np.ascontiguousarray(block).view(np.int32), device=dev)
        count = len(actions)
        a = torch.as_tensor(np.ascontiguousarray(actions, np.int32), device=dev)
        out = torch.zeros((self.words, count), dtype=torch.int32, device=dev)
        keys = torch.zeros(count, dtype=torch.int64, device=dev)
        rew = torch.zeros(count, dtype=torch.float32, device=dev)
        s = torch.cuda.current_stream() if stream is None else stream
        _dsp.dsp_step(self.h, b.data_ptr(), b.shape[1], count, a.data_ptr(), depth, out.data_ptr(), count,
                      keys.data_ptr(), rew.data_ptr(), s.cuda_stream)
        torch.cuda.synchronize()
        return (out.cpu().numpy().view(np.uint32), keys.cpu().numpy().view(np.uint64),
                rew.cpu().numpy())

    def rollout(self, block, hist, start_depth, stream=None):
        dev = torch.device("cuda")
        b = torch.as_tensor(np.ascontiguousarray(block).view(np.int32), device=dev)
        count = b.shape[1]
        h = None if hist is None else torch.as_tensor(np.ascontiguousarray(hist, np.int8).reshape(count, 32),
                                                      device=dev)
        v = torch.zeros(count, dtype=torch.float32, device=dev)
        s = torch.cuda.current_stream() if stream is None else stream
        _dsp.dsp_rollout(self.h, b.data_ptr(), count, count, 0 if h is None else h.data_ptr(), start_depth,
                         v.data_ptr(), s.cuda_stream)
        torch.cuda.synchronize()
        return v.cpu().numpy()

    def counters(self):
        return _dsp.dsp_read_counters(self.h)

    def reset_counters(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        _dsp.dsp_reset_counters(self.h, s.cuda_stream)


class JobBatch:
    """Jobs packed in one device arena: inputs first (parents, indexes), then
    the results that stay on the device (each leaf's states and grouped
    positions: the parent block and index lists of the children's later
    expansions), then the per-child results a host tree search reads (counts,
    offsets, keys, reward, u and l sums). `host_inputs` is a pinned copy of
    the input part for end-to-end runs that copy inputs in and the host-read
    results out every step, as dsp_plan does."""

    def __init__(self, model, jobs, device="cuda", child_cap=None):
        self.model = model
        self.jobs = jobs
        W = model.words
        na_all = [j.n_actions or model.num_actions for j in jobs]
        layout = []
        off = 0
        for j, na in zip(jobs, na_all):
            n = len(j.idx)
            pc = j.parent.shape[1]
            cap = model.max_children(n) if child_cap is None else child_cap
            e = {}
            e["parent"] = off; off = _align(off + 4 * W * pc)
            e["idx"] = off; off = _align(off + 2 * n)
            layout.append(e)
        self.input_bytes = off
        for j, na, e in zip(jobs, na_all, layout):
            n = len(j.idx)
            cap = model.max_children(n) if child_cap is None else child_cap
            e["n"], e["na"], e["cap"] = n, na, cap
            e["leaf"] = off; off = _align(off + 4 * W * n)
            e["perm"] = off; off = _align(off + 2 * na * n)
        self.host_out_start = off
        for j, na, e in zip(jobs, na_all, layout):
            cap = e["cap"]
            e["cc"] = off; off = _align(off + 4 * na)
            e["co"] = off; off = _align(off + 4 * na * (cap + 1))
            e["key"] = off; off = _align(off + 8 * na * cap)
            e["rew"] = off; off = _align(off + 8 * na * cap)
            e["u"] = off; off = _align(off + 8 * na * cap)
            e["l"] = off; off = _align(off + 8 * na * cap)
        self.total_bytes = off
        self.device_out_bytes = self.host_out_start - self.input_bytes  # leaf states, grouped positions
        self.output_bytes = off - self.host_out_start  # what download_outputs copies
        self.layout = layout
        host = torch.zeros(self.input_bytes, dtype=torch.uint8, pin_memory=True)
        hn = host.numpy()
        for j, e in zip(jobs, layout):
            pb = np.ascontiguousarray(j.parent, np.uint32).view(np.uint8).reshape(-1)
            hn[e["parent"]:e["parent"] + pb.size] = pb
            ib = np.ascontiguousarray(j.idx, np.uint16).view(np.uint8)
            hn[e["idx"]:e["idx"] + ib.size] = ib
        self.host_inputs = host
        self.arena = torch.zeros(self.total_bytes, dtype=torch.uint8, device=device)
        self.arena[: self.input_bytes].copy_(host)
        base = self.arena.data_ptr()
        self.descs = (_dsp.dsp_leaf_job * len(jobs))()
        for k, (j, e) in enumerate(zip(jobs, layout)):
            d = self.descs[k]
            d.parent = base + e["parent"]
            d.parent_cap = j.parent.shape[1]
            d.n_scen = e["n"]
            d.idx = base + e["idx"]
            d.last_action = j.last_action
            d.depth = j.depth
            for i in range(32):
                d.hist[i] = int(j.hist[i])
            d.first_action = j.first_action
            d.n_actions = e["na"]
            d.child_cap = e["cap"]
            d.leaf_states = base + e["leaf"]
            d.child_count = base + e["cc"]
            d.child_off = base + e["co"]
            d.child_key = base + e["key"]
            d.rew_sum = base + e["rew"]
            d.u_sum = base + e["u"]
            d.l_sum = base + e["l"]
            d.perm = base + e["perm"]
        self.host_outputs = None

    def run(self, stream=None):
        s = torch.cuda.current_stream() if stream is None else stream
        _dsp.dsp_expand_leaves(self.model.h, self.descs, len(self.jobs), s.cuda_stream)

    def upload_inputs(self, stream=None):
        """Host -> device copy of every job's parent block and indexes."""
        self.arena[: self.input_bytes].copy_(self.host_inputs, non_blocking=True)

    def download_outputs(self):
        """Device -> host copy (pinned) of the per-child results a host tree
        search reads; leaf states and grouped positions stay on the device."""
        if self.host_outputs is None:
            self.host_outputs = torch.zeros(self.output_bytes, dtype=torch.uint8, pin_memory=True)
        self.host_outputs.copy_(self.arena[self.host_out_start:], non_blocking=True)
        return self.host_outputs

    def results(self, k):
        """Numpy results of job k (same keys as the oracle's expand())."""
        a = self.arena.cpu().numpy()
        e = self.layout[k]
        n, na, cap, W = e["n"], e["na"], e["cap"], self.model.words

        def view(name, dt, count):
            return a[e[name]:e[name] + np.dtype(dt).itemsize * count].view(dt)

        return dict(leaf=view("leaf", np.uint32, W * n).reshape(W, n), child_count=view("cc", np.int32, na),
                    child_off=view("co", np.int32, na * (cap + 1)).reshape(na, cap + 1),
                    key=view("key", np.uint64, na * cap).reshape(na, cap),
                    rew=view("rew", np.int64, na * cap).reshape(na, cap),
                    u=view("u", np.int64, na * cap).reshape(na, cap), l=view("l", np.int64, na * cap).reshape(na, cap),
                    perm=view("perm", np.uint16, na * n).reshape(na, n))

    def all_results(self):
        a = self.arena.cpu().numpy()
        out = []
        for k in range(len(self.jobs)):
            out.append(self.results_from(a, k))
        return out

    def results_from(self, a, k):
        e = self.layout[k]
        n, na, cap, W = e["n"], e["na"], e["cap"], self.model.words

        def view(name, dt, count):
            return a[e[name]:e[name] + np.dtype(dt).itemsize * count].view(dt)

        return dict(leaf=view("leaf", np.uint32, W * n).reshape(W, n), child_count=view("cc", np.int32, na),
                    child_off=view("co", np.int32, na * (cap + 1)).reshape(na, cap + 1),
                    key=view("key", np.uint64, na * cap).reshape(na, cap),
                    rew=view("rew", np.int64, na * cap).reshape(na, cap),
                    u=view("u", np.int64, na * cap).reshape(na, cap), l=view("l", np.int64, na * cap).reshape(na, cap),
                    perm=view("perm", np.uint16, na * n).reshape(na, n))
