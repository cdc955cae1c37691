#!/usr/bin/env python
"""Benchmark of GPU leaf expansion (HyP-DESPOT, Sec. III-D) on B300.

One step = one dsp_expand_leaves call over a batch of synthetic leaf jobs
shaped like the paper's tasks: every (leaf, action, scenario) is stepped,
grouped by observation, and bounded by u0 and default-policy rollouts to depth
D. Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rs15_15]
  python bench.py --impl reference ...   # the CPU oracle on the host cores

value = scenario-steps/s (g calls on live scenarios, counted in-kernel) with
inputs resident in HBM; e2e = the same through pinned host buffers with the
inputs copied in and every result copied out inside the timed region (two job
arenas on two streams take alternate steps, so transfers overlap kernels). A
planning step (multi-threaded tree search, Sec. III-C) afterwards gives the
root bound gap.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1802_06215_b300 import inputs  # noqa: E402

WORKLOADS = {
    # name: (config factory, jobs per step, description, planning (threads, seconds, use_queue))
    "rs15_15": (inputs.rs15_15, 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=500, D=90; 4096 leaf jobs, "
                                      "|Phi_b|~U{1..500}, depth~U{0..10}", (4, 0.5, 0)),
    "rs7_8": (inputs.rs7_8, 4096, "Rock Sample 7x7, 8 rocks, |A|=13, K=100, D=90; 4096 leaf jobs, "
                                  "|Phi_b|~U{1..100}, depth~U{0..10}", (4, 0.5, 0)),
    "mars15_15": (inputs.mars15_15, 512, "two-robot Rock Sample 15x15, 15 rocks, |A|=400, K=500, D=90; 512 leaf "
                                         "jobs, |Phi_b|~U{1..500}, depth~U{0..10}", (16, 0.5, 1)),
    "car50": (inputs.car50, 1024, "car among 50 pedestrians, |A|=3, K=500, D=50; 1024 leaf jobs, "
                                  "|Phi_b|~U{1..500}, depth~U{0..10}", (4, 0.1, 0)),
    # variants of the same kernels (--sweep)
    "car6": (lambda: inputs.car_p(6), 1024, "car among 6 pedestrians, |A|=3, K=500, D=50; 1024 leaf jobs",
             (4, 0.1, 0)),
    "car12": (lambda: inputs.car_p(12), 1024, "car among 12 pedestrians, |A|=3, K=500, D=50; 1024 leaf jobs",
              (4, 0.1, 0)),
    "car20": (lambda: inputs.car_p(20), 1024, "car among 20 pedestrians, |A|=3, K=500, D=50; 1024 leaf jobs",
              (4, 0.1, 0)),
    "mars11_11": (inputs.mars11_11, 512, "two-robot Rock Sample 11x11, 11 rocks, |A|=256, K=500, D=90; 512 leaf "
                                         "jobs", (16, 0.5, 1)),
    "mars20_20": (inputs.mars20_20, 512, "two-robot Rock Sample 20x20, 20 rocks, |A|=625, K=500, D=90; 512 leaf "
                                         "jobs", (16, 0.5, 1)),
    "nav13": (inputs.nav13, 512, "navigation in a partially known 13x13 map, |A|=9, 8-bit readings, K=500, D=90; "
                                 "512 leaf jobs, |Phi_b|~U{1..500}, depth~U{0..10}", (4, 0.5, 0)),
    "rs15_15_k100": (lambda: inputs.rs15_15_k(100), 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=100, D=90; "
                                                         "4096 leaf jobs, |Phi_b|~U{1..100}", (4, 0.5, 0)),
    "rs15_15_k250": (lambda: inputs.rs15_15_k(250), 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=250, D=90; "
                                                         "4096 leaf jobs, |Phi_b|~U{1..250}", (4, 0.5, 0)),
    "rs15_15_k1000": (lambda: inputs.rs15_15_k(1000), 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=1000, D=90; "
                                                           "4096 leaf jobs, |Phi_b|~U{1..1000}", (4, 0.5, 0)),
    "rs15_15_k5000": (lambda: inputs.rs15_15_k(5000), 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=5000, D=90; "
                                                           "4096 leaf jobs, |Phi_b|~U{1..5000}", (4, 0.5, 0)),
}
SWEEP = ["car6", "car12", "car20", "car50", "rs15_15_k100", "rs15_15_k250", "rs15_15", "rs15_15_k1000",
         "rs15_15_k5000", "mars11_11", "mars15_15", "mars20_20", "nav13"]
SMS, LANES_PER_SM, MAX_SM_MHZ = 148, 128, 2032.0
try:
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as _f:
        MEASURED = json.load(_f)
except (OSError, ValueError):
    MEASURED = {}
METRIC = "scenario-steps/sec and leaf expansions/sec at K=500, D=90 (fraction of roofline); root gap"
E2E_LANES = 3  # job arenas (and streams) of the end-to-end measurement

KERNEL_SOURCES = {
    "rs": ["expand_rs.cu", "rs_model.cuh", "rs_common.cuh", "common.cuh"],
    "car": ["expand_car.cu", "car_model.cuh", "group.cuh", "common.cuh"],
    "nav": ["expand_nav.cu", "nav_model.cuh", "group.cuh", "common.cuh"],
}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="rs15_15", choices=list(WORKLOADS))
    p.add_argument("--jobs", type=int, default=0, help="override jobs per step")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU baseline sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-plan", action="store_true")
    p.add_argument("--no-learned", action="store_true", help="skip the learned-policy comparison")
    p.add_argument("--no-autotune", action="store_true", help="run the default launch shape, untuned")
    p.add_argument("--shape", default="",
                   help="run this launch shape, untuned: comma-separated field=value of dsp_launch_shape "
                        "(e.g. rs_form=2,block_b=256)")
    p.add_argument("--plan-worlds", type=int, default=16,
                   help="rs15_15: planner episodes on this many seeded worlds (100 steps, 4 threads, 200 trials each)")
    p.add_argument("--e2e-lanes", type=int, default=E2E_LANES,
                   help="job arenas (and streams) taking the end-to-end steps in turn")
    p.add_argument("--no-companions", action="store_true",
                   help="measure only --workload (a default rs15_15 run also measures car50 and mars15_15, "
                        "each under its own key)")
    p.add_argument("--episodes", type=int, default=0,
                   help="run planner episodes on this many held-out Rock Sample 15x15 worlds (heuristic and learned "
                        "default policy) and exit")
    p.add_argument("--episode-steps", type=int, default=100)
    p.add_argument("--plan-seconds", type=float, default=0.1)
    p.add_argument("--learned-rollouts", type=int, default=0,
                   help="time only the learned-policy rollout kernel on this many start states and exit")
    p.add_argument("--plan-scaling", default="", choices=["", "rs15_15", "mars15_15"],
                   help="planning throughput against search threads (per-leaf launches, batched launches, "
                        "the device queue)")
    p.add_argument("--plan-locks", action="store_true", help="--plan-scaling: also under one tree lock")
    p.add_argument("--pomcp", default="", choices=[""] + list(WORKLOADS),
                   help="POMCP-style planner with GPU rollouts against the oracle's (one line per batch size)")
    p.add_argument("--sweep", default="", help="'all' or comma-separated workloads: one line per variant")
    p.add_argument("--ref-step-seconds", type=float, default=60.0,
                   help="cap on the oracle's time per step in the reference arm")
    return p.parse_args()


class ClockSampler:
    """SM clocks and throttle reasons sampled every 2 ms through NVML while the
    timed region runs (nvidia-smi every 100 ms if NVML is unavailable)."""

    REASONS = {0x8: "hw_slowdown", 0x40: "hw_thermal_slowdown", 0x20: "sw_thermal_slowdown",
               0x4: "sw_power_cap"}

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.method = "nvml"
        self.error = None
        self.stop = threading.Event()

    def __enter__(self):
        self.t = threading.Thread(target=self._run, daemon=True)
        self.t.start()
        return self

    def _run(self):
        try:
            import pynvml
            pynvml.nvmlInit()
            h = pynvml.nvmlDeviceGetHandleByIndex(self.index)
            mx = pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM)
            reasons = getattr(pynvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                pynvml.nvmlDeviceGetCurrentClocksThrottleReasons
            while not self.stop.is_set():
                sm = pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)
                self.samples.append((sm, mx, reasons(h)))
                time.sleep(0.002)
            return
        except Exception as e:
            self.error = repr(e)[:120]
            self.method = "nvidia-smi"
        proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index),
                                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.active",
                                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=subprocess.PIPE,
                                stderr=subprocess.DEVNULL, text=True)
        while not self.stop.is_set():
            line = proc.stdout.readline()
            try:
                a, b, r = (x.strip() for x in line.split(","))
                self.samples.append((float(a), float(b), int(r, 16)))
            except ValueError:
                pass
        proc.terminate()

    def __exit__(self, *a):
        self.stop.set()
        self.t.join(timeout=5)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        reasons = set()
        for _, _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        out = {"sm_mhz": statistics.median(s[0] for s in self.samples),
               "sm_max_mhz": max(s[1] for s in self.samples), "reasons": sorted(reasons),
               "samples": len(self.samples), "method": self.method}
        if self.error:
            out["nvml_error"] = self.error
        return out


def cpu_oracle_run(cfg, jobs, seconds, threads):
    """The oracle, as it stands, over jobs in order until `seconds` elapse
    (threads > 1: a thread pool over jobs; ctypes releases the GIL)."""
    import concurrent.futures as cf

    import oracle
    om = oracle.Model(cfg)
    t0 = time.perf_counter()
    done, steps = 0, 0
    if threads == 1:
        oracle.ops_reset()
        for j in jobs:
            e = om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist)
            steps += e["steps"]
            done += 1
            if time.perf_counter() - t0 > seconds:
                break
        ops = oracle.ops_read()
    else:
        ops = 0
        with cf.ThreadPoolExecutor(threads) as ex:
            k = 0
            while k < len(jobs) and time.perf_counter() - t0 <= seconds:
                chunk = jobs[k:k + 4 * threads]
                for e in ex.map(lambda j: om.expand(j.parent, j.idx, j.last_action, j.depth, j.hist), chunk):
                    steps += e["steps"]
                done += len(chunk)
                k += len(chunk)
    dt = time.perf_counter() - t0
    return dict(steps=steps, jobs=done, seconds=dt, ops=ops)


def _dtype(cfg):
    return "f32" if cfg.kind in (inputs.CAR, inputs.NAV) else "int32"


def run_reference(args, rank, world):
    if rank != 0:
        return
    mk, njobs, desc, _ = WORKLOADS[args.workload]
    cfg = mk()
    njobs = args.jobs or njobs
    jobs = inputs.job_stream(cfg, njobs, 1000)
    cores = os.cpu_count() or 1
    per_step = min(args.ref_step_seconds, max(1.0, 60.0 / max(1, args.steps + args.warmup)))
    for _ in range(args.warmup):
        cpu_oracle_run(cfg, jobs, min(per_step, 2.0), cores)
    tot_steps, tot_jobs, tot_t = 0, 0, 0.0
    for _ in range(args.steps):
        r = cpu_oracle_run(cfg, jobs, per_step, cores)
        tot_steps += r["steps"]
        tot_jobs += r["jobs"]
        tot_t += r["seconds"]
    value = tot_steps / tot_t
    sample = f"each step: leading jobs of the {njobs}-job stream for up to {per_step:.1f} s on {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "scenario-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": _dtype(cfg),
            "data": "synthetic", "config": {"workload": f"{args.workload}: {desc}"},
            "leaf_expansions_per_s": tot_jobs / tot_t,
            "cpu_baseline": {"value": value, "unit": "scenario-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "scenario-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def source_digest(kind):
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kind]:
        with open(os.path.join(ROOT, "paper_1802_06215_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(workload, kind):
    """DRAM bytes per launch of this workload's expansion kernels from the
    committed ncu summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path):
        return None
    digest = source_digest(kind)
    for line in open(path):
        m = re.match(r"\|\s*(\w+)\s*\|\s*([0-9.eE+]+)\s*\|\s*(\w+)\s*\|", line)
        if m and m.group(1) == workload and m.group(3) == digest:
            return float(m.group(2))
    return None


def root_states(cfg, rng):
    if cfg.kind == inputs.CAR:
        base = (rng.uniform(0, 40, cfg.P), rng.uniform(0, 40, cfg.P))
        b = inputs.car_block(cfg, cfg.K, rng, s=0.0, v=0, base=base, jitter=0.0)
        return b
    if cfg.kind == inputs.NAV:
        return inputs.nav_block(cfg, cfg.K, rng)
    pos = [(0, cfg.n // 2), (0, cfg.n // 2 - 1)][: (2 if cfg.kind == inputs.MULTIGRID else 1)]
    return inputs.rs_block(cfg, cfg.K, rng, pos=pos)


def planning_step(_dsp, m, cfg, plan, reps=5, batch=0):
    """`reps` planning steps from the benchmark's root belief, each on its own
    random streams (plan step), with the WEU exit (xi = 0.95) and the time
    limit: totals over the steps (a free-running search's tree, and so when
    its exit rule ends it, varies with the threads' timing), the per-step
    spread, and the first step's root bounds and action."""
    threads, seconds, use_queue = plan
    b = root_states(cfg, np.random.default_rng(99))
    p = _dsp.dsp_search_params(threads=threads, rounds=10 ** 7, time_limit_s=seconds, c_a=1.0, c_o=0.5, xi=0.95,
                               target_gap=0.0, deterministic=0, use_queue=use_queue, batch=batch)
    rows = []
    for r in range(reps):
        _dsp.dsp_set_plan_step(m.h, 0x50000000 + r)
        rows.append(_dsp.dsp_plan(m.h, b, None, p, m.num_actions))
    _dsp.dsp_set_plan_step(m.h, 0)
    g = rows[0]
    exps = sum(x["expansions"] for x in rows)
    secs = sum(x["seconds"] for x in rows)
    rates = [x["expansions"] / x["seconds"] for x in rows]
    return {"root_u": g["root_u"], "root_l": g["root_l"], "root_gap": g["root_u"] - g["root_l"],
            "threads": threads, "planning_time_s": seconds, "through_queue": bool(use_queue),
            "batched_launches_of": batch if batch > 1 else None,
            "planning_steps": reps, "expansions": exps, "nodes": sum(x["nodes"] for x in rows), "seconds": secs,
            "expansions_per_s": exps / secs,
            "expansions_per_s_min": min(rates), "expansions_per_s_max": max(rates),
            "scenario_steps_per_s": sum(x["scenario_steps"] for x in rows) / secs, "action": g["action"]}


def learned_step(_dsp, batch, m, cfg, jobs, seconds, n_beliefs=32):
    """The learned default policy (shipped weights) against the heuristic one:
    root gap after planning steps of equal time (xi = 0 and target gap 0, so
    that both searches run to the time limit) from held-out beliefs along
    heuristic-planner episodes, and the tensor-core rate of the in-rollout
    network over a learned-policy expansion of the first 256 jobs."""
    import torch
    from paper_1802_06215_b300 import learn
    car = cfg.kind == inputs.CAR
    path = os.path.join(ROOT, "paper_1802_06215_b300", "weights", "car50_pi0.npz" if car else "rs15_15_pi0.npz")
    h, meta = learn.load_weights(path)
    if car:
        roots = learn.car_roots(cfg, n_beliefs, 9000)
    else:
        roots = learn.eval_roots(cfg, range(9000, 9000 + (n_beliefs + 1) // 2), 2, 0.05)[:n_beliefs]
    cmp_ = learn.compare(cfg, h, roots, seconds, xi=0.0, target_gap=0.0)
    sub = batch.JobBatch(m, jobs[:256])
    _dsp.dsp_set_policy(m.h, h)
    sub.run()
    torch.cuda.synchronize()
    m.reset_counters()
    _dsp.dsp_kernel_timing(m.h, True)
    for _ in range(3):
        sub.run()
    torch.cuda.synchronize()
    kms, calls = _dsp.dsp_kernel_timing(m.h, False)
    steps, status = m.counters()
    _dsp.dsp_set_policy(m.h, None)
    _dsp.dsp_mlp_destroy(h)
    if status != 0:
        raise RuntimeError(f"device status word {status}")
    na = m.num_actions
    flop = 2 * (64 * 256 + 256 * 256 + 256 * (na + 1))
    tflops = steps * flop / (kms / 1000.0) / 1e12
    kname = ("car_expand_kernel + car_rollout_tc_kernel (learned-policy expansion of 256 jobs; tcgen05.mma BF16, "
             "TMEM accumulators)" if car else
             "rs_group_kernel + rs_rollout_tc_kernel (learned-policy expansion of 256 jobs; tcgen05.mma BF16, TMEM "
             "accumulators)")
    peak = MEASURED.get("bf16_tflops")
    if not car:
        cmp_["training"] = training_step_rate(_dsp, na, peak)
    cmp_["weights"] = os.path.relpath(path, ROOT)
    cmp_["tensor_roofline"] = {
        "bound": "tensor", "achieved": tflops, "unit": "TFLOP/s", "peak": peak,
        "frac": tflops / peak if peak else None, "peak_source": "MEASURED_PEAKS bf16_tflops (burst, of measured)",
        "flop_per_scenario_step": flop, "scenario_steps": steps / 3, "kernel_ms_per_launch": kms / max(calls, 1),
        "kernel": kname}
    return cmp_


def training_step_rate(_dsp, na, peak, batch=16384, steps=20):
    """The policy network's training step (dsp_mlp_train_step: BF16 forward
    and backward GEMMs with FP32 accumulation, softmax cross-entropy, Adam)
    on random features and labels: samples/s and the GEMMs' rate against the
    BF16 peak (6 B (64*256 + 256*256 + 256*32) flop per step)."""
    import torch
    h = _dsp.dsp_mlp_create(batch, 7)
    X = torch.rand((batch, 64), dtype=torch.float32, device="cuda")
    y = torch.randint(0, na + 1, (batch,), dtype=torch.int32, device="cuda")
    for _ in range(3):
        _dsp.dsp_mlp_train_step(h, X.data_ptr(), y.data_ptr(), batch, na + 1, 1e-3)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        _dsp.dsp_mlp_train_step(h, X.data_ptr(), y.data_ptr(), batch, na + 1, 1e-3)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    _dsp.dsp_mlp_destroy(h)
    flop = 6 * batch * (64 * 256 + 256 * 256 + 256 * 32)
    return {"batch": batch, "ms_per_step": dt * 1000.0, "samples_per_s": batch / dt,
            "tflops": flop / dt / 1e12, "frac_of_bf16_peak": flop / dt / 1e12 / peak if peak else None,
            "note": "wall time per step (the loss is read back every step); tcgen05 GEMMs, 128-row tiles, FP32 "
                    "accumulators in tensor memory, weight gradients split over the batch"}


def combine_ranks(t_ms, steps, dist, device):
    """Max over ranks of the timed region, sum over ranks of the scenario-
    steps (each rank expands its own job stream: weak scaling, no exchange of
    data between ranks)."""
    if dist is None:
        return float(t_ms), float(steps)
    import torch
    tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    st = torch.tensor([float(steps)], dtype=torch.float64, device=device)
    dist.all_reduce(st, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(st.item())


def episodes(args):
    """Whole-planner episodes (the Rock Sample 15x15 task, 4 search threads,
    --plan-seconds per decision, up to --episode-steps decisions, worlds
    9000.. held out from training): heuristic against learned default policy."""
    from paper_1802_06215_b300 import build, learn
    build.build()
    cfg = inputs.rs15_15()
    seeds = list(range(9000, 9000 + args.episodes))
    heur = learn.run_episodes(cfg, seeds, args.episode_steps, args.plan_seconds)
    h, _ = learn.load_weights(os.path.join(ROOT, "paper_1802_06215_b300", "weights", "rs15_15_pi0.npz"))
    lrn = learn.run_episodes(cfg, seeds, args.episode_steps, args.plan_seconds, policy=h)
    print(json.dumps({"metric": "planner episodes (discounted return, decisions/s, root gap)", "workload":
                      f"rs15_15: {len(seeds)} worlds x up to {args.episode_steps} decisions of "
                      f"{args.plan_seconds} s, 4 threads", "heuristic": heur, "learned": lrn}), flush=True)


def learned_rollouts(args):
    """The learned-policy rollout kernel alone (dsp_rollout_logged) on N
    Rock Sample 15x15 start states with the shipped weights: tensor rate of
    the in-rollout network against the measured BF16 peak."""
    import torch
    from paper_1802_06215_b300 import _dsp, batch, build, learn
    build.build()
    cfg = inputs.rs15_15()
    m = batch.Model(cfg)
    n = args.learned_rollouts
    b = inputs.rs_block(cfg, n, np.random.default_rng(0), pos=[(0, cfg.n // 2)])
    bd = torch.tensor(b.view(np.int32), device="cuda")
    hd = torch.zeros((n, 32), dtype=torch.int8, device="cuda")
    val = torch.zeros(n, dtype=torch.float32, device="cuda")
    h, _ = learn.load_weights(os.path.join(ROOT, "paper_1802_06215_b300", "weights", "rs15_15_pi0.npz"))
    _dsp.dsp_set_policy(m.h, h)
    st = torch.cuda.current_stream()
    for _ in range(max(1, args.warmup)):
        _dsp.dsp_rollout_logged(m.h, bd.data_ptr(), n, n, hd.data_ptr(), 1, val.data_ptr(), 0, st.cuda_stream)
    torch.cuda.synchronize()
    m.reset_counters()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        _dsp.dsp_rollout_logged(m.h, bd.data_ptr(), n, n, hd.data_ptr(), 1, val.data_ptr(), 0, st.cuda_stream)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    steps, status = m.counters()
    if status != 0:
        raise RuntimeError(f"device status word {status}")
    flop = 2 * (64 * 256 + 256 * 256 + 256 * (m.num_actions + 1))
    tflops = steps / args.steps * flop / (ms / 1000.0) / 1e12
    peak = MEASURED.get("bf16_tflops")
    print(json.dumps({"metric": "learned-policy rollout tensor rate", "value": tflops, "unit": "TFLOP/s",
                      "rollouts": n, "ms_per_launch": ms, "scenario_steps_per_launch": steps / args.steps,
                      "flop_per_scenario_step": flop, "peak": peak, "frac": tflops / peak if peak else None,
                      "mean_value": float(val.mean().item()), "kernel": "rs_rollout_tc_kernel<false>"}), flush=True)
    _dsp.dsp_mlp_destroy(h)
    m.close()


def measure(args, name, rank, world, dist, local, headline=True):
    """One workload: device-resident rate (L2 flushed before every timed step),
    end-to-end rate through pinned host buffers, kernel time and ALU roofline,
    the oracle's CPU baseline, and (rank 0) planning and learned-policy
    comparisons. Returns the JSON line's fields (None on ranks > 0)."""
    import torch
    from paper_1802_06215_b300 import _dsp, batch
    mk, njobs, desc, plan = WORKLOADS[name]
    cfg = mk()
    njobs = (args.jobs or njobs) if headline else njobs
    jobs = inputs.job_stream(cfg, njobs, 1000 + rank)
    m = batch.Model(cfg)
    jb = batch.JobBatch(m, jobs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        jb.run()
    torch.cuda.synchronize()
    kernels_per_step = 1 if cfg.kind == inputs.CAR else 2

    # the launch shape the timed region runs: the autotuner's choice on this
    # job batch (kept per model, K, |A| and GPU; the default shape is timed
    # beside it afterwards)
    autotuned = None
    if args.shape:
        fields = dict(kv.split("=") for kv in args.shape.split(","))
        unknown = set(fields) - set(_dsp.SHAPE_FIELDS)
        if unknown:
            raise SystemExit(f"--shape: unknown fields {sorted(unknown)}")
        _dsp.dsp_set_launch_shape(m.h, **{k: int(v) for k, v in fields.items()})
    elif not args.no_autotune:
        from paper_1802_06215_b300 import autotune as AT
        cache = os.environ.get("DSP_TUNE_CACHE") or None
        best = AT.autotune(m, jb, torch.cuda.get_device_name(), cache, reps=3)
        autotuned = {"shape": {k: best[k] for k in _dsp.SHAPE_FIELDS}, "cached": best["cached"],
                     "tuning_ms_per_call": best.get("ms"), "default_tuning_ms_per_call": best.get("default_ms"),
                     "candidates_timed": best.get("tried"), "jobs": njobs,
                     "search_space": {
                         inputs.CAR: "tps {4,8,16,32} x ctas_car {fit,3,2}",
                         inputs.NAV: "ctas_b {fit,6,4,2}"}.get(
                             cfg.kind, "block_b {128,256,512} x ctas_b {fit,6,4} x warps_a {default,5,10} "
                                       "(two robots {default,8,16}); one robot x rs_form {blocks,items}"),
                     "note": "0 = the field's default; the timed region runs this shape"}
        for _ in range(2):
            jb.run()
        torch.cuda.synchronize()

    # device-resident timing (L2 flushed before every step, outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    m.reset_counters()
    _dsp.dsp_kernel_timing(m.h, True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    with ClockSampler(local) as clk:
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            jb.run()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    kernel_ms, kernel_calls = _dsp.dsp_kernel_timing(m.h, False)
    times = [a.elapsed_time(b) for a, b in ev]
    steps_total, status = m.counters()
    if status != 0:
        raise RuntimeError(f"device status word {status}")
    t_ms, steps_all = combine_ranks(sum(times), steps_total, dist, "cuda")
    value = steps_all / (t_ms / 1000.0)
    steps_per_launch = steps_total / args.steps
    if autotuned is not None:
        # the default shape on the same jobs, for comparison (not the headline)
        tuned_shape = _dsp.dsp_get_launch_shape(m.h)
        _dsp.dsp_set_launch_shape(m.h)
        nd = max(20, args.steps // 4)
        for _ in range(max(3, args.warmup)):
            jb.run()
        torch.cuda.synchronize()
        _dsp.dsp_kernel_timing(m.h, True)
        d_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nd)]
        for k in range(nd):
            flush.zero_()
            d_ev[k][0].record(stream)
            jb.run()
            d_ev[k][1].record(stream)
        torch.cuda.synchronize()
        d_kms, d_calls = _dsp.dsp_kernel_timing(m.h, False)
        _dsp.dsp_set_launch_shape(m.h, **tuned_shape)
        autotuned["default_shape_ms_per_step"] = sum(a.elapsed_time(b) for a, b in d_ev) / nd
        autotuned["tuned_shape_ms_per_step"] = t_ms / args.steps
        autotuned["default_shape_kernel_ms_per_launch"] = d_kms / max(1, d_calls)
        autotuned["tuned_shape_kernel_ms_per_launch"] = kernel_ms / max(1, kernel_calls)

    # end to end through the public call: every step copies its inputs in from
    # pinned host memory and the results a host search reads out (each
    # child's count, offsets, key and sums; the leaf states and grouped
    # positions stay on the device for the children's expansions, as in
    # dsp_plan), inside the timed region. Three
    # job arenas on three streams take the steps in turn, so that one step's
    # transfers overlap the others' kernels; the time is the wall time of all
    # steps, first copy to last result.
    n_lanes = max(1, args.e2e_lanes)
    lanes = [(stream, jb)] + [(torch.cuda.Stream(), batch.JobBatch(m, jobs)) for _ in range(n_lanes - 1)]
    for s_, b_ in lanes:  # warm every arena and stream
        with torch.cuda.stream(s_):
            b_.upload_inputs()
            b_.run(s_)
            b_.download_outputs()
    torch.cuda.synchronize()
    e2s, e2e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2s.record(stream)
    for s_, _ in lanes[1:]:
        s_.wait_event(e2s)
    h0 = time.perf_counter()
    for k in range(args.steps):
        s_, b_ = lanes[k % len(lanes)]
        with torch.cuda.stream(s_):
            flush.zero_()
            b_.upload_inputs()
            b_.run(s_)
            b_.download_outputs()
    host_ms = (time.perf_counter() - h0) * 1000.0  # the host's enqueueing, before the last result
    for s_, _ in lanes[1:]:
        tail = torch.cuda.Event()
        tail.record(s_)
        stream.wait_event(tail)
    e2e_.record(stream)
    torch.cuda.synchronize()
    e2_ms, _ = combine_ranks(e2s.elapsed_time(e2e_), 0, dist, "cuda")
    e2_value = steps_all / (e2_ms / 1000.0)

    # integer issue-rate probe (context for the roofline denominator)
    sink = torch.zeros(4, dtype=torch.int32, device="cuda")
    _dsp.dsp_alu_probe(sink.data_ptr(), 64, stream.cuda_stream)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    probe_ops = _dsp.dsp_alu_probe(sink.data_ptr(), 2048, stream.cuda_stream)
    p1.record(stream)
    torch.cuda.synchronize()
    probe_tops = probe_ops / (p0.elapsed_time(p1) / 1000.0) / 1e12

    if rank != 0:
        m.close()
        return None
    clocks = clk.summary()
    planning = None
    if not args.no_plan:
        # a plan through the device queue: the model creates the queue (and its
        # kernel's graph) on the first such step and keeps it, so that step is
        # reported on its own and the steps after it are what replanning sees
        first = planning_step(_dsp, m, cfg, plan, reps=1) if plan[2] else None
        planning = planning_step(_dsp, m, cfg, plan)
        if first is not None:
            planning["first_step_with_queue_creation"] = {k: first[k] for k in ("expansions", "seconds",
                                                                                "expansions_per_s")}
    # the same planning step with the leaves going through the device job queue;
    # the model creates its queue (and the kernel's graph) on the first such
    # step and keeps it, so the second step is what a replanning loop sees
    planning_queue = None
    planning_batched = None
    if not args.no_plan and cfg.kind in (inputs.GRID, inputs.MULTIGRID) and not plan[2]:
        # the threads' claimed leaves handed to one dispatcher that expands up
        # to 64 of them per dsp_expand_leaves call
        planning_batched = planning_step(_dsp, m, cfg, plan, batch=64)
        first = planning_step(_dsp, m, cfg, (plan[0], plan[1], 1), reps=1)
        planning_queue = planning_step(_dsp, m, cfg, (plan[0], plan[1], 1))
        planning_queue["first_step_with_queue_creation"] = {k: first[k] for k in ("expansions", "seconds",
                                                                                   "expansions_per_s")}
    # the planning workload of the 15x15 task as stated: 16 seeded worlds, up
    # to 100 planning steps each (the episode ends when the robot exits), 4
    # search threads, each step 50 rounds of 4 trials (no time limit), the
    # belief updated by Bayes' rule after every real step
    planning_episodes = None
    if not args.no_plan and name == "rs15_15" and args.plan_worlds > 0:
        from paper_1802_06215_b300 import learn
        t0 = time.perf_counter()
        planning_episodes = learn.run_episodes(cfg, range(9000, 9000 + args.plan_worlds), 100, 0.0, threads=4,
                                               rounds=50)
        planning_episodes.update({"steps_per_world_max": 100, "threads": 4, "trials_per_step": 200,
                                  "wall_seconds": time.perf_counter() - t0, "world_seeds": "9000.."})
    learned = None
    if not args.no_learned and name in ("rs15_15", "car50"):
        learned = learned_step(_dsp, batch, m, cfg, jobs, plan[1])
    cpu = None
    ops_per_step = None
    if not args.no_cpu_baseline:
        secs = args.cpu_seconds if headline else args.cpu_seconds / 2
        r1 = cpu_oracle_run(cfg, jobs, secs, 1)
        ops_per_step = r1["ops"] / max(1, r1["steps"])
        cores = os.cpu_count() or 1
        rn = cpu_oracle_run(cfg, jobs, secs / 2, cores)
        cpu = {"value": r1["steps"] / r1["seconds"], "unit": "scenario-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"first {r1['jobs']} of the {njobs} jobs of this workload, single-threaded, "
                         f"{r1['seconds']:.1f} s", "ops_per_scenario_step": ops_per_step,
               "all_cores": {"value": rn["steps"] / rn["seconds"], "cores": cores,
                             "sample": f"first {rn['jobs']} jobs on {cores} threads, {rn['seconds']:.1f} s"}}
    kind = {inputs.CAR: "car", inputs.NAV: "nav"}.get(cfg.kind, "rs")
    avg_kernel_s = kernel_ms / max(1, kernel_calls) / 1000.0
    peak_tops = SMS * LANES_PER_SM * MAX_SM_MHZ * 1e6 / 1e12
    roof = None
    if ops_per_step:
        achieved = ops_per_step * steps_per_launch / avg_kernel_s / 1e12
        # one-robot Rock Sample's block form has its own row
        blocks = cfg.kind == inputs.GRID and _dsp.dsp_get_launch_shape(m.h)["rs_form"] == 1
        traffic = measured_traffic(name + ("_blocks" if blocks else ""), kind)
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s",
                "frac": achieved / peak_tops, "traffic": traffic,
                "peak_source": "derived: 148 SMs x 128 lanes x 2032 MHz (one 32-bit op per lane per clock)",
                "probe_tops": probe_tops, "ops_per_scenario_step": ops_per_step,
                "kernel": {"rs": "rs_group_kernel + " + ("rs_rollout_blocks_kernel" if blocks else
                                                          ("rs_rollout_slices_kernel" if cfg.kind == inputs.GRID
                                                           else "rs_rollout_items_kernel")) + " (one expansion)",
                           "car": "car_expand_kernel",
                           "nav": "nav_group_kernel + nav_rollout_items_kernel (one expansion)"}[kind],
                "kernel_ms_per_launch": avg_kernel_s * 1000.0,
                "achieved_hbm_gbs": jb.total_bytes / avg_kernel_s / 1e9}
        if kind == "rs":
            roof["note"] = ("achieved counts the definition's operations (the oracle's count: a policy scan "
                            "at every rollout step); the kernels carry the heuristic's target between samples, "
                            "jump over move-only steps and walk one trajectory for each slice of up to 128 of a "
                            "child's items, with bit-exact results, so they execute fewer operations and frac can "
                            "exceed 1; the phases' issue-slot use under ncu is in profiles/ (phase A 65 %, phase B "
                            "83 % for one robot)")
    line = {
        "metric": METRIC, "value": value, "unit": "scenario-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(cfg), "data": "synthetic",
        "config": {"workload": f"{name}: {desc}", "jobs_per_step": njobs,
                   "l2": "256 MiB buffer written before every timed step (outside the events)"},
        "leaf_expansions_per_s": njobs * world * args.steps / (t_ms / 1000.0),
        "scenario_steps_per_step": steps_per_launch,
        "e2e": {"value": e2_value, "unit": "scenario-steps/s", "h2d_bytes_per_step": jb.input_bytes,
                "d2h_bytes_per_step": jb.output_bytes, "ms_per_step": e2_ms / args.steps,
                "host_enqueue_ms_per_step": host_ms / args.steps,
                "method": f"dsp_expand_leaves on {n_lanes} job arenas and {n_lanes} streams taking the steps in turn; "
                          "wall time from the first upload to the last result, L2 flush in each step; "
                          "read back: each child's count, offsets, key and reward/u/l sums (what dsp_plan's "
                          "search reads); the leaf states and grouped positions stay on the device",
                "device_resident_bytes_per_step": jb.device_out_bytes},
        "gpu_launches": args.steps * kernels_per_step,
        "launch_shape": _dsp.dsp_get_launch_shape(m.h),
        "roofline": roof,
        "cpu_baseline": cpu,
        "planning": planning,
        "planning_batched": planning_batched,
        "planning_queue": planning_queue,
        "planning_episodes": planning_episodes,
        "autotune": autotuned,
        "learned_pi0": learned,
        "clocks": clocks,
    }
    m.close()
    return line


# Workloads measured beside the headline one in a default run (the driving
# task among 50 pedestrians beside Rock Sample 15x15), each under its own key.
COMPANIONS = {"rs15_15": ["car50", "mars15_15"]}


def run_ours(args, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1802_06215_b300 import build
    build.build()
    line = measure(args, args.workload, rank, world, dist, local)
    extra = {}
    if not args.no_companions:
        for name in COMPANIONS.get(args.workload, []):
            extra[name] = measure(args, name, rank, world, dist, local, headline=False)
    if rank == 0:
        for name, sub in extra.items():
            sub.pop("metric", None)
            sub.pop("n_gpus", None)
            line[name] = sub
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def sweep(args):
    """Variants of the same kernels (crowd sizes, map sizes and joint action
    counts, numbers of scenarios): one JSON line per workload with its
    device-resident rate, kernel time and ALU roofline fraction. Each point
    runs the autotuner's launch shape for its batch (unless --shape or
    --no-autotune), times `--steps` expansions after `--warmup` (L2 flushed
    before each) and counts algorithmic ops with the oracle on the leading
    jobs for 2 s."""
    import torch
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    peak_tops = SMS * LANES_PER_SM * MAX_SM_MHZ * 1e6 / 1e12
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    names = args.sweep.split(",") if args.sweep != "all" else SWEEP
    for name in names:
        mk, njobs, desc, _ = WORKLOADS[name]
        cfg = mk()
        m = batch.Model(cfg)
        jobs = inputs.job_stream(cfg, args.jobs or njobs, 1000)
        jb = batch.JobBatch(m, jobs)
        tuned = None
        if args.shape:  # fields that do not apply to the workload's model keep their defaults
            fields = {k: int(v) for k, v in (kv.split("=") for kv in args.shape.split(","))}
            _dsp.dsp_set_launch_shape(m.h, **fields)
        elif not args.no_autotune:
            # the autotuner's shape for this batch; its default-shape time beside it
            from paper_1802_06215_b300 import autotune as AT
            best = AT.autotune(m, jb, torch.cuda.get_device_name(), None, reps=3)
            tuned = {"shape": {k: best[k] for k in _dsp.SHAPE_FIELDS}, "tuning_ms_per_call": best.get("ms"),
                     "default_tuning_ms_per_call": best.get("default_ms"),
                     "note": "0 = the field's default; the line's times are this shape's"}
        for _ in range(args.warmup):
            jb.run()
        torch.cuda.synchronize()
        m.reset_counters()
        _dsp.dsp_kernel_timing(m.h, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record()
            jb.run()
            ev[k][1].record()
        torch.cuda.synchronize()
        kms, calls = _dsp.dsp_kernel_timing(m.h, False)
        steps, status = m.counters()
        if status != 0:
            raise RuntimeError(f"{name}: device status word {status}")
        t_ms = sum(a.elapsed_time(b) for a, b in ev)
        r1 = cpu_oracle_run(cfg, jobs, 2.0, 1)
        ops = r1["ops"] / max(1, r1["steps"])
        achieved = ops * (steps / args.steps) / (kms / calls / 1000.0) / 1e12
        print(json.dumps({"sweep": name, "config": desc, "value": steps / (t_ms / 1000.0),
                          "unit": "scenario-steps/s", "ms_per_step": t_ms / args.steps,
                          "kernel_ms_per_launch": kms / calls, "scenario_steps_per_step": steps / args.steps,
                          "leaf_expansions_per_s": len(jobs) / (t_ms / args.steps / 1000.0),
                          "ops_per_scenario_step": ops, "roofline": {"bound": "alu", "achieved": achieved,
                                                                     "peak": peak_tops, "unit": "Tops/s",
                                                                     "frac": achieved / peak_tops},
                          "autotune": tuned, "cpu_oracle_1core": r1["steps"] / r1["seconds"]}), flush=True)
        m.close()
        del jb


def plan_scaling(args):
    """Planning throughput against search threads: per-leaf launches, batched
    launches and the device job queue on per-node atomics (with --plan-locks
    also under one tree lock): three planning steps of 0.3 s per (threads,
    path) from the benchmark's root belief, xi < 0 so that no trial ends
    without a leaf (the machinery's rate, not the planner's). One JSON line per
    point: median, min and max expansions/s."""
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    mk = WORKLOADS[args.plan_scaling][0]
    cfg = mk()
    m = batch.Model(cfg)
    b = root_states(cfg, np.random.default_rng(99))

    def plan(threads, q, lock, bsz, secs):
        p = _dsp.dsp_search_params(threads=threads, rounds=10 ** 7, time_limit_s=secs, c_a=1.0, c_o=0.5, xi=-1.0,
                                   target_gap=-1.0, deterministic=0, use_queue=q, tree_lock=lock, batch=bsz)
        return _dsp.dsp_plan(m.h, b, None, p, m.num_actions)

    paths = [(0, 0, 0, "per-leaf launches"), (0, 0, 64, "batched launches (up to 64 leaves)"),
             (1, 0, 0, "device queue")]
    if args.plan_locks:
        paths += [(0, 1, 0, "per-leaf launches"), (1, 1, 0, "device queue")]
    for q, lock, bsz, _ in paths:
        plan(4, q, lock, bsz, 0.2)
    for threads in (1, 2, 4, 8, 16, 32):
        for q, lock, bsz, name in paths:
            r = []
            for _ in range(3):
                g = plan(threads, q, lock, bsz, 0.3)
                r.append(g["expansions"] / g["seconds"])
            print(json.dumps({"plan_scaling": args.plan_scaling, "threads": threads, "path": name,
                              "tree": "one tree lock" if lock else "per-node atomics",
                              "expansions_per_s": statistics.median(r), "min": min(r), "max": max(r)}),
                  flush=True)
    m.close()


def pomcp_rate(args):
    """The POMCP-style planner (dsp_pomcp_plan) with the GPU as its rollout
    service, against the oracle's planner on one host core over the same
    rounds from the benchmark's root belief: simulations, rollouts and
    scenario-steps per second, and whether both planned the same tree."""
    import oracle
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    mk = WORKLOADS[args.pomcp][0]
    cfg = mk()
    m = batch.Model(cfg)
    b = root_states(cfg, np.random.default_rng(99))
    for bsz in (256, 1024, 4096):
        p = _dsp.dsp_pomcp_params(rounds=2, batch=bsz, c=10.0, time_limit_s=0.0)
        _dsp.dsp_pomcp_plan(m.h, b, None, p, m.num_actions)  # warm
        rounds = max(2, 16384 // bsz)
        p = _dsp.dsp_pomcp_params(rounds=rounds, batch=bsz, c=10.0, time_limit_s=0.0)
        g = _dsp.dsp_pomcp_plan(m.h, b, None, p, m.num_actions)
        t0 = time.perf_counter()
        o = oracle.Model(cfg).pomcp(b, None, rounds=rounds, batch=bsz, c=10.0)
        to = time.perf_counter() - t0
        print(json.dumps({"pomcp": args.pomcp, "batch": bsz, "rounds": g["rounds"], "seconds": g["seconds"],
                          "simulations_per_s": g["simulations"] / g["seconds"],
                          "rollouts_per_s": g["rollouts"] / g["seconds"],
                          "scenario_steps_per_s": g["scenario_steps"] / g["seconds"],
                          "nodes": g["nodes"], "root_value": g["value"], "action": g["action"],
                          "same_tree_as_oracle": bool(o["signature"] == g["signature"] and
                                                      np.array_equal(o["root_q"], g["root_q"])),
                          "oracle_1core": {"seconds": to, "simulations_per_s": o["simulations"] / to,
                                           "scenario_steps_per_s": o["steps"] / to}}), flush=True)
    m.close()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.episodes:
        if rank == 0:
            episodes(args)
    elif args.learned_rollouts:
        if rank == 0:
            learned_rollouts(args)
    elif args.sweep:
        if rank == 0:
            sweep(args)
    elif args.plan_scaling:
        if rank == 0:
            plan_scaling(args)
    elif args.pomcp:
        if rank == 0:
            pomcp_rate(args)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
