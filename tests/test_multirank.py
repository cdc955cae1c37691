"""The N > 1 launch of the benchmark on CPU ranks (gloo): every rank expands
its own job stream, and only the timed region's maximum and the step count's
sum cross ranks; the reference arm runs on rank 0 alone."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    from paper_1802_06215_b300 import inputs
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    t, s = bench.combine_ranks(10.0 + rank, 100 * (rank + 1), dist, "cpu")
    cfg = inputs.rs7_8()
    jobs = inputs.job_stream(cfg, 8, 1000 + rank)
    out.put((rank, t, s, int(jobs[0].parent[:, 0].sum()), len(jobs)))
    dist.barrier()
    dist.destroy_process_group()


def test_rank_reduction_and_sharding_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(r[1] == 11.0 and r[2] == 300.0 for r in res)
    assert res[0][4] == res[1][4] == 8
    assert res[0][3] != res[1][3]  # the ranks' job streams differ


def test_reference_arm_two_ranks():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps",
           "1", "--warmup", "0", "--workload", "rs7_8", "--jobs", "16", "--ref-step-seconds", "0.3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
