"""Learned default policy pi0 for one-robot Rock Sample: harvest, imitation
training and the comparison with the heuristic pi0.

The paper's leaf initialisation rolls out a hand-written default policy to get
l0 (Sec. III-A, Eq. lb). Here a network may take its place:

1. Planner episodes on fresh world seeds. At each step `dsp_plan_nodes` plans
   from the current belief (K scenarios drawn from per-rock posteriors), the
   world takes the chosen action (`dsp_step` of the same model on the world's
   own random stream, a plan-step counter no planning call uses) and the belief
   is updated by Bayes' rule with the sensor accuracy 0.5 + 0.5 * 2^(-d/20) of
   the Rock Sample model (Sec. IV-A).
2. Every expanded tree node with enough scenarios gives one pair: the features
   of its state and belief counters (`dsp_features`, the same map the learned
   rollout evaluates) and argmax_a L(b, a), the action the tree's lower bound
   takes there. With the heuristic pi0 in the rollouts that label is one step
   of policy improvement over it.
3. Minibatch Adam on softmax cross-entropy with `dsp_mlp_train_step` (BF16
   tensor-core forward and backward, FP32 master weights).
4. `dsp_set_policy` installs the network. Every rollout still steps g, so l0
   stays the value of a policy and a valid lower bound.

PyTorch only holds device buffers here; every step of the computation runs in
the library's kernels.

    python -m paper_1802_06215_b300.learn train --out weights.npz
    python -m paper_1802_06215_b300.learn compare --weights weights.npz
"""
import argparse
import json
import math
import time

import numpy as np

from . import _dsp, batch, inputs

WORLD_STEP_BASE = 1 << 31  # plan-step counters of the world's own random streams
SENSE0 = 5                 # first Sense action of one-robot Rock Sample
SAMPLE = 4


def sensor_accuracy(d):
    return 0.5 + 0.5 * 2.0 ** (-d / 20.0)


class Belief:
    """Belief of one-robot Rock Sample: observed position and sampled mask,
    independent posteriors P(rock i good), and the belief counters (sensed good
    minus sensed bad per rock) that the planner and the policies read."""

    def __init__(self, cfg, pos_word, sampled=0):
        self.cfg = cfg
        self.pos = int(pos_word)
        self.sampled = int(sampled)
        self.p = np.full(cfg.m, 0.5)
        self.hist = np.zeros(32, np.int8)

    def scenarios(self, rng, K):
        m = self.cfg.m
        good = ((rng.random((K, m)) < self.p[None, :]).astype(np.uint32) << np.arange(m, dtype=np.uint32)).sum(
            axis=1, dtype=np.uint32)
        b = np.zeros((5, K), np.uint32)
        b[0] = self.pos
        b[2] = good & np.uint32(~self.sampled & 0xFFFFFFFF)
        b[3] = self.sampled
        b[4] = np.arange(K, dtype=np.uint32)
        return b

    def update(self, a, key, next_pos, next_sampled):
        if a >= SENSE0:
            r = a - SENSE0
            z = int(key) & 3
            if z in (1, 2):
                x, y = self.pos & 0xFF, (self.pos >> 8) & 0xFF
                c = int(self.cfg.rock_cells[r])
                q = sensor_accuracy(math.hypot((c & 0xFF) - x, (c >> 8) - y))
                like_good, like_bad = (q, 1 - q) if z == 1 else (1 - q, q)
                p = self.p[r]
                self.p[r] = p * like_good / (p * like_good + (1 - p) * like_bad)
                self.hist[r] = np.int8(max(-127, min(127, int(self.hist[r]) + (1 if z == 1 else -1))))
        self.pos = int(next_pos)
        self.sampled = int(next_sampled)


def start_word(cfg):
    return np.uint32(0 | ((cfg.n // 2) << 8))


def search_params(seconds, threads=4):
    return _dsp.dsp_search_params(threads=threads, rounds=10 ** 7, time_limit_s=seconds, c_a=1.0, c_o=0.5,
                                  xi=0.95, target_gap=0.0, deterministic=0, use_queue=0)


def episode(model, cfg, world_seed, steps, seconds, threads=4, min_scen=16, node_cap=1 << 15, harvest=True):
    """One planner episode. Returns the discounted return, the visited roots
    (state block, counters) and, when harvesting, the exported nodes."""
    rng = np.random.default_rng([world_seed, 0xBE11EF])
    world = inputs.rs_block(cfg, 1, rng, pos=[(0, cfg.n // 2)])
    world[4] = 0
    belief = Belief(cfg, world[0, 0])
    ret, disc = 0.0, 1.0
    roots, states, hists, labels, decisions = [], [], [], [], 0
    t_plan = 0.0
    for t in range(steps):
        K = cfg.K
        root = belief.scenarios(rng, K)
        roots.append((root, belief.hist.copy()))
        model.set_plan_step((world_seed * 1000 + t) & 0x7FFFFFFF)
        p = search_params(seconds, threads)
        if harvest:
            res, rec, st = _dsp.dsp_plan_nodes(model.h, root, belief.hist, p, model.num_actions, min_scen,
                                               node_cap, model.words)
            if len(rec):
                states.append(st)
                hists.append(rec["hist"])
                labels.append(rec["action"].astype(np.int32))
        else:
            res = _dsp.dsp_plan(model.h, root, belief.hist, p, model.num_actions)
        t_plan += res["seconds"]
        decisions += 1
        a = int(res["action"])
        model.set_plan_step(WORLD_STEP_BASE + (world_seed & 0x3FFFFFFF))
        nxt, key, rew = model.step(world, np.array([a], np.int32), t)
        ret += disc * float(rew[0])
        disc *= cfg.gamma
        belief.update(a, key[0], nxt[0, 0], nxt[3, 0])
        world = nxt
        if (int(key[0]) >> 62) & 1 or (int(nxt[0, 0]) >> 16) & 1:
            break
    out = {"return": ret, "roots": roots, "decisions": decisions, "plan_seconds": t_plan}
    if harvest and states:
        out["states"] = np.concatenate(states, axis=1)
        out["hist"] = np.concatenate(hists, axis=0)
        out["labels"] = np.concatenate(labels)
    return out


def features(model, states, hist):
    """Features of a (words, count) block with (count, 32) counters, computed
    by dsp_features on the device."""
    import torch
    count = states.shape[1]
    if count == 0:
        return np.zeros((0, 64), np.float32)
    b = torch.as_tensor(np.ascontiguousarray(states).view(np.int32), device="cuda")
    h = torch.as_tensor(np.ascontiguousarray(hist, np.int8), device="cuda")
    f = torch.empty((count, 64), dtype=torch.float32, device="cuda")
    _dsp.dsp_features(model.h, b.data_ptr(), count, count, h.data_ptr(), f.data_ptr(),
                      torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def harvest(cfg, world_seeds, steps, seconds, policy=None, threads=4, min_scen=16, log=print):
    """(features, labels) from planner episodes on the given world seeds; with
    `policy` (a dsp_mlp handle) the planner's rollouts use it."""
    model = batch.Model(cfg)
    if policy is not None:
        _dsp.dsp_set_policy(model.h, policy)
    X, Y, rets = [], [], []
    t0 = time.time()
    for s in world_seeds:
        ep = episode(model, cfg, s, steps, seconds, threads, min_scen)
        rets.append(ep["return"])
        if "states" in ep:
            X.append(features(model, ep["states"], ep["hist"]))
            Y.append(ep["labels"])
        log(f"world {s}: return {ep['return']:.2f}, {ep['decisions']} decisions, "
            f"{sum(len(y) for y in Y)} pairs, {time.time() - t0:.0f} s")
    model.close()
    return np.concatenate(X), np.concatenate(Y), rets


def train(X, Y, n_actions, epochs=30, batch_size=2048, lr=1e-3, seed=0, val_frac=0.1, log=print, init=None):
    """Imitation training with the library's kernels; returns the dsp_mlp
    handle and the validation accuracy."""
    import torch
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(Y))
    nval = int(len(Y) * val_frac)
    vi, ti = perm[:nval], perm[nval:]
    h = _dsp.dsp_mlp_create(batch_size, seed)
    if init is not None:
        _dsp.dsp_mlp_set_weights(h, init)
    Xt = torch.as_tensor(X[ti], device="cuda")
    Yt = torch.as_tensor(Y[ti].astype(np.int32), device="cuda")
    nb = len(ti) // batch_size
    stream = torch.cuda.current_stream().cuda_stream
    acc = float("nan")
    for ep in range(epochs):
        order = torch.as_tensor(rng.permutation(len(ti)), device="cuda")
        Xs, Ys = Xt[order].contiguous(), Yt[order].contiguous()
        lr_ep = lr * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        tot = 0.0
        for b in range(nb):
            sl = slice(b * batch_size, (b + 1) * batch_size)
            tot += _dsp.dsp_mlp_train_step(h, Xs[sl].data_ptr(), Ys[sl].data_ptr(), batch_size, n_actions, lr_ep,
                                           stream)
        if nval and (ep % 5 == 4 or ep == epochs - 1):
            acc = accuracy(h, X[vi], Y[vi], n_actions, batch_size)
            log(f"epoch {ep + 1}: loss {tot / max(nb, 1):.4f}, validation accuracy {acc:.3f}")
    return h, acc


def accuracy(h, X, Y, n_actions, batch_size):
    import torch
    hits = 0
    for s in range(0, len(Y), batch_size):
        xb = torch.as_tensor(np.ascontiguousarray(X[s:s + batch_size]), device="cuda")
        lg = torch.empty((len(xb), 32), dtype=torch.float32, device="cuda")
        _dsp.dsp_mlp_forward(h, xb.data_ptr(), len(xb), lg.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        pred = lg.cpu().numpy()[:, :n_actions].argmax(axis=1)
        hits += int((pred == Y[s:s + batch_size]).sum())
    return hits / max(len(Y), 1)


def compare(cfg, policy, roots, seconds, threads=4):
    """Root gap u - l after one planning step of `seconds` from each root
    belief, heuristic pi0 then learned pi0, on the same random streams."""
    model = batch.Model(cfg)
    rows = []
    for k, (root, hist) in enumerate(roots):
        row = {}
        for name, pol in (("heuristic", None), ("learned", policy)):
            _dsp.dsp_set_policy(model.h, pol)
            model.set_plan_step(0x40000000 + k)
            r = _dsp.dsp_plan(model.h, root, hist, search_params(seconds, threads), model.num_actions)
            row[name] = {"gap": r["root_u"] - r["root_l"], "u": r["root_u"], "l": r["root_l"],
                         "action": int(r["action"]), "expansions": r["expansions"], "seconds": r["seconds"]}
        rows.append(row)
    model.close()
    out = {"beliefs": len(rows), "planning_time_s": seconds, "threads": threads}
    for name in ("heuristic", "learned"):
        out[name] = {"mean_root_gap": float(np.mean([r[name]["gap"] for r in rows])),
                     "mean_root_l": float(np.mean([r[name]["l"] for r in rows])),
                     "mean_root_u": float(np.mean([r[name]["u"] for r in rows])),
                     "mean_expansions": float(np.mean([r[name]["expansions"] for r in rows])),
                     "decisions_per_s": len(rows) / sum(r[name]["seconds"] for r in rows)}
    out["decision_agreement"] = float(np.mean([r["heuristic"]["action"] == r["learned"]["action"] for r in rows]))
    out["learned_tighter"] = float(np.mean([r["learned"]["gap"] < r["heuristic"]["gap"] for r in rows]))
    return out


def save_weights(path, h, meta):
    np.savez_compressed(path, params=_dsp.dsp_mlp_get_weights(h).astype(np.float32), meta=json.dumps(meta))


def load_weights(path):
    z = np.load(path)
    h = _dsp.dsp_mlp_create(64, 0)
    _dsp.dsp_mlp_set_weights(h, z["params"])
    return h, json.loads(str(z["meta"]))


def eval_roots(cfg, world_seeds, steps, seconds, threads=4):
    """Root beliefs along heuristic-planner episodes on held-out worlds."""
    model = batch.Model(cfg)
    roots = []
    for s in world_seeds:
        roots += episode(model, cfg, s, steps, seconds, threads, harvest=False)["roots"]
    model.close()
    return roots


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "compare"])
    ap.add_argument("--worlds", type=int, default=32)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--plan-seconds", type=float, default=0.1)
    ap.add_argument("--iterations", type=int, default=2, help="harvest/train rounds (later ones roll out the net)")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--weights", default="paper_1802_06215_b300/weights/rs15_15_pi0.npz")
    ap.add_argument("--out", default=None)
    ap.add_argument("--eval-worlds", type=int, default=8)
    ap.add_argument("--eval-steps", type=int, default=8)
    ap.add_argument("--eval-seconds", type=float, default=1.0)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    cfg = inputs.rs15_15()
    if a.cmd == "train":
        policy, init, meta = None, None, {"iterations": []}
        X_all, Y_all = [], []
        for it in range(a.iterations):
            seeds = list(range(1000 + it * a.worlds, 1000 + (it + 1) * a.worlds))
            X, Y, rets = harvest(cfg, seeds, a.steps, a.plan_seconds, policy=policy)
            X_all.append(X)
            Y_all.append(Y)
            h, acc = train(np.concatenate(X_all), np.concatenate(Y_all), 20, epochs=a.epochs, seed=it)
            meta["iterations"].append({"worlds": seeds, "pairs": int(sum(len(y) for y in Y_all)),
                                       "mean_return": float(np.mean(rets)), "val_accuracy": acc})
            print(json.dumps(meta["iterations"][-1]))
            if policy is not None:
                _dsp.dsp_mlp_destroy(policy)
            policy = h
        meta.update({"config": "rs15_15", "steps": a.steps, "plan_seconds": a.plan_seconds, "epochs": a.epochs})
        save_weights(a.out or a.weights, policy, meta)
    else:
        policy, meta = load_weights(a.weights)
        roots = eval_roots(cfg, range(9000, 9000 + a.eval_worlds), a.eval_steps, 0.05)
        print(json.dumps(compare(cfg, policy, roots, a.eval_seconds)))


if __name__ == "__main__":
    main()
