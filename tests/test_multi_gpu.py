"""Node-level parallelism over several GPUs (Sec. III-D): leaf expansions of
one planning step routed over one model per GPU (dsp_plan_multi).

On the host (no GPU): the routing rule dsp_route_leaves, alone and applied by
two gloo ranks that each stand for a GPU and must together cover every
expansion exactly once. On one GPU: two or three models on the same device
stand in for a device list; deterministic rounds must build the tree of
dsp_plan on one model bit for bit (and the oracle's), since an expansion's
results do not depend on the GPU that computes it."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_route_rule_round_robin_and_copies():
    from paper_1802_06215_b300 import _dsp, build
    build.build()
    parents = np.array([0, 0, 1, 1, 2, 0, 2], np.int32)
    tgt, cp = _dsp.dsp_route_leaves(3, 5, parents)
    assert tgt.tolist() == [(5 + k) % 3 for k in range(7)]
    assert cp.tolist() == [int(t != p) for t, p in zip(tgt, parents)]
    tgt1, cp1 = _dsp.dsp_route_leaves(1, 123, np.zeros(4, np.int32))
    assert tgt1.tolist() == [0, 0, 0, 0] and cp1.tolist() == [0, 0, 0, 0]
    with pytest.raises(_dsp.DspError):
        _dsp.dsp_route_leaves(2, 0, np.array([0, 2], np.int32))  # parent model out of range
    with pytest.raises(_dsp.DspError):
        _dsp.dsp_route_leaves(0, 0, np.zeros(1, np.int32))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1802_06215_b300 import _dsp
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    # both ranks route the same 3 batches of a step (rank r stands for GPU r)
    mine, copies = [], 0
    first = 0
    rng = np.random.default_rng(7)
    for size in (5, 1, 8):
        parents = rng.integers(0, 2, size).astype(np.int32)
        tgt, cp = _dsp.dsp_route_leaves(2, first, parents)
        for k in range(size):
            if tgt[k] == rank:
                mine.append(first + k)
                copies += int(cp[k])
        first += size
    t = torch.zeros(first, dtype=torch.int64)
    t[mine] = 1
    dist.all_reduce(t)
    c = torch.tensor([copies], dtype=torch.int64)
    dist.all_reduce(c)
    q.put((rank, t.tolist(), int(c.item()), len(mine)))
    dist.barrier()
    dist.destroy_process_group()


def test_route_rule_partitions_expansions_over_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, cover0, c0, n0), (_, cover1, c1, n1) = out
    assert cover0 == cover1 == [1] * 14          # every expansion on exactly one rank
    assert n0 == 7 and n1 == 7                     # round robin
    assert c0 == c1


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1802_06215_b300 import _dsp, batch, build
    build.build()
    return torch, _dsp, batch


@pytest.mark.gpu
@pytest.mark.parametrize("mk,G", [("rs15_15", 2), ("mars15_15", 3), ("car50", 2)])
def test_multi_model_rounds_equal_one_model(gpu, mk, G):
    import oracle
    from paper_1802_06215_b300 import inputs as I
    torch, _dsp, batch = gpu
    cfg = getattr(I, mk)()
    if cfg.kind == I.MULTIGRID:
        cfg = cfg.with_(K=120)
    models = [batch.Model(cfg) for _ in range(G)]
    rng = np.random.default_rng(3)
    if cfg.kind == I.CAR:
        root = I.car_block(cfg, 100, rng, s=0.0, v=0)
    else:
        pos = [(0, cfg.n // 2), (0, cfg.n // 2 - 1)][: (2 if cfg.kind == I.MULTIGRID else 1)]
        root = I.rs_block(cfg, min(cfg.K, 200), rng, pos=pos)
    p = _dsp.dsp_search_params(threads=4, rounds=6, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0,
                               deterministic=1, use_queue=0)
    one = _dsp.dsp_plan(models[0].h, root, None, p, models[0].num_actions)
    multi = _dsp.dsp_plan_multi([m.h for m in models], root, None, p, models[0].num_actions)
    for f in ("signature", "root_u", "root_l", "action", "nodes", "expansions", "scenario_steps"):
        assert one[f] == multi[f], f
    assert np.array_equal(one["root_visits"], multi["root_visits"])
    o = oracle.Model(cfg).plan(root, None, threads=4, rounds=6, c_a=1.0, c_o=0.5, xi=0.95)
    assert o["signature"] == multi["signature"] and o["root_u"] == multi["root_u"]
    for m in models:
        m.close()


@pytest.mark.gpu
def test_multi_model_free_running(gpu):
    from paper_1802_06215_b300 import inputs as I
    torch, _dsp, batch = gpu
    cfg = I.rs15_15()
    models = [batch.Model(cfg) for _ in range(2)]
    root = I.rs_block(cfg, cfg.K, np.random.default_rng(1), pos=[(0, 7)])
    p = _dsp.dsp_search_params(threads=8, rounds=40, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0,
                               deterministic=0, use_queue=0)
    r = _dsp.dsp_plan_multi([m.h for m in models], root, None, p, models[0].num_actions)
    assert r["expansions"] >= 2 and r["root_l"] <= r["root_u"] + 1e-9 and 0 <= r["action"] < models[0].num_actions
    q = _dsp.dsp_search_params(threads=4, rounds=10, time_limit_s=0.0, c_a=1.0, c_o=0.5, xi=0.95, target_gap=0.0,
                               deterministic=0, use_queue=1)
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_plan_multi([m.h for m in models], root, None, q, models[0].num_actions)
    assert e.value.status == _dsp.DSP_E_UNSUPPORTED
    other = batch.Model(cfg.with_(seed=5))
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_plan_multi([models[0].h, other.h], root, None, p, models[0].num_actions)
    assert e.value.status == _dsp.DSP_E_INVALID
    other.close()
    for m in models:
        m.close()
