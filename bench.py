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
inputs copied in and every result copied out inside the timed region.
"""
import argparse
import json
import os
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
    # name: (config factory, jobs per step, description)
    "rs15_15": (inputs.rs15_15, 4096, "Rock Sample 15x15, 15 rocks, |A|=20, K=500, D=90; 4096 leaf jobs, "
                                      "|Phi_b|~U{1..500}, depth~U{0..10}"),
    "rs7_8": (inputs.rs7_8, 4096, "Rock Sample 7x7, 8 rocks, |A|=13, K=100, D=90; 4096 leaf jobs, "
                                  "|Phi_b|~U{1..100}, depth~U{0..10}"),
    "mars15_15": (inputs.mars15_15, 512, "two-robot Rock Sample 15x15, 15 rocks, |A|=400, K=500, D=90; 512 leaf "
                                         "jobs, |Phi_b|~U{1..500}, depth~U{0..10}"),
    "car50": (inputs.car50, 1024, "car among 50 pedestrians, |A|=3, K=500, D=50; 1024 leaf jobs, "
                                  "|Phi_b|~U{1..500}, depth~U{0..10}"),
}
SMS, LANES_PER_SM, MAX_SM_MHZ = 148, 128, 2032.0
METRIC = "scenario-steps/sec and leaf expansions/sec at K=500, D=90 (fraction of roofline); root gap"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="rs15_15", choices=list(WORKLOADS))
    p.add_argument("--jobs", type=int, default=0, help="override jobs per step")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU baseline sample budget")
    p.add_argument("--no-cpu-baseline", action="store_true")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def run_reference(args, rank, world):
    if rank != 0:
        return
    mk, njobs, desc = WORKLOADS[args.workload]
    cfg = mk()
    njobs = args.jobs or njobs
    jobs = inputs.job_stream(cfg, njobs, 1000)
    cores = os.cpu_count() or 1
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_oracle_run(cfg, jobs, min(per_step, 2.0), cores)
    tot_steps, tot_jobs, tot_t = 0, 0, 0.0
    for _ in range(args.steps):
        r = cpu_oracle_run(cfg, jobs, per_step, cores)
        tot_steps += r["steps"]
        tot_jobs += r["jobs"]
        tot_t += r["seconds"]
    value = tot_steps / tot_t
    sample = f"each step: leading jobs of the {njobs}-job stream for ~{per_step:.1f} s on {cores} threads"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "scenario-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": _dtype(cfg),
            "data": "synthetic", "config": {"workload": f"{args.workload}: {desc}"},
            "leaf_expansions_per_s": tot_jobs / tot_t,
            "cpu_baseline": {"value": value, "unit": "scenario-steps/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "scenario-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _dtype(cfg):
    return "f32" if cfg.kind == inputs.CAR else "int32"


def run_ours(args, rank, world):
    import torch
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    mk, njobs, desc = WORKLOADS[args.workload]
    cfg = mk()
    njobs = args.jobs or njobs
    jobs = inputs.job_stream(cfg, njobs, 1000 + rank)
    m = batch.Model(cfg)
    jb = batch.JobBatch(m, jobs)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(3, args.warmup)):
        jb.run()
    torch.cuda.synchronize()

    # device-resident timing (L2 flushed before every step, outside the events)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    m.reset_counters()
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
    times = [a.elapsed_time(b) for a, b in ev]
    steps_total, status = m.counters()
    if status != 0:
        raise RuntimeError(f"device status word {status}")
    t_ms = sum(times)
    if dist:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        st = torch.tensor([float(steps_total)], device="cuda")
        dist.all_reduce(st, op=dist.ReduceOp.SUM)
        steps_all = float(st.item())
    else:
        steps_all = float(steps_total)
    value = steps_all / (t_ms / 1000.0)
    steps_per_launch = steps_total / args.steps

    # end to end: pinned inputs in, every result out, inside the timed region
    e2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        flush.zero_()
        e2[k][0].record(stream)
        jb.upload_inputs()
        jb.run()
        jb.download_outputs()
        e2[k][1].record(stream)
    torch.cuda.synchronize()
    e2_ms = sum(a.elapsed_time(b) for a, b in e2)
    if dist:
        tt = torch.tensor([e2_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2_ms = float(tt.item())
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
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    cpu = None
    ops_per_step = None
    if not args.no_cpu_baseline:
        r1 = cpu_oracle_run(cfg, jobs, args.cpu_seconds, 1)
        ops_per_step = r1["ops"] / max(1, r1["steps"])
        cpu = {"value": r1["steps"] / r1["seconds"], "unit": "scenario-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"first {r1['jobs']} of the {njobs} jobs of this workload, single-threaded, "
                         f"{r1['seconds']:.1f} s", "ops_per_scenario_step": ops_per_step}
    avg_launch_s = t_ms / args.steps / 1000.0
    max_mhz = clocks.get("sm_max_mhz") or MAX_SM_MHZ
    peak_tops = SMS * LANES_PER_SM * MAX_SM_MHZ * 1e6 / 1e12
    roof = None
    if ops_per_step:
        achieved = ops_per_step * steps_per_launch / avg_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak_tops, "unit": "Tops/s", "frac": achieved / peak_tops,
                "traffic": None, "peak_source": "148 SMs x 128 lanes x 2032 MHz (issue rate, one 32-bit op per lane "
                                                 "per clock)", "probe_tops": probe_tops,
                "ops_per_scenario_step": ops_per_step, "kernel": "rs_expand_kernel" if cfg.kind != inputs.CAR
                else "car_expand_kernel"}
    line = {
        "metric": METRIC, "value": value, "unit": "scenario-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": _dtype(cfg), "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "jobs_per_step": njobs,
                   "l2": "256 MiB buffer written before every timed step (outside the events)"},
        "leaf_expansions_per_s": njobs * world / (t_ms / 1000.0),
        "scenario_steps_per_step": steps_per_launch,
        "e2e": {"value": e2_value, "unit": "scenario-steps/s", "h2d_bytes_per_step": jb.input_bytes,
                "d2h_bytes_per_step": jb.output_bytes},
        "gpu_launches": args.steps,
        "roofline": roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", args.gpus if args.gpus else 1))
    if world != args.gpus and "WORLD_SIZE" not in os.environ:
        world = 1
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
