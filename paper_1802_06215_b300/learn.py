"""Learned default policy pi0 for one-robot Rock Sample: training data,
training, and the comparison with the heuristic pi0.

The paper's leaf initialisation rolls out a hand-written default policy to get
l0 (Sec. III-A, Eq. lb). Here a network may take its place. Its logits cover
the |A| actions plus one more column, "defer", which takes the heuristic
policy's action; the rollout takes the argmax over the actions allowed in the
observable state and defer (the rule of `allowed_mask`). Every rollout still
steps g, so l0 stays the value of a policy and a valid lower bound.

Approximate policy iteration (`policy_iteration`, the `api` command, which
made the shipped weights): pi_0 is the heuristic. At iteration k, states are
drawn uniformly over the observable space plus from pi_k's own rollouts
(logged actions replayed with `dsp_step`); each gets Q^{pi_k}(s, a) from one
leaf expansion (`dsp_expand_leaves`, rollouts running pi_k) over scenarios
drawn from the belief its counters imply; the label is the best allowed action
where it beats the heuristic's action by a margin, else defer. The network is
trained on all labels so far (`dsp_mlp_train_step`: BF16 tensor-core forward
and backward, FP32 master weights, Adam) and installed (`dsp_set_policy`) as
pi_{k+1}.

Planner imitation (`harvest`, the `train` command; NOT how the shipped weights
were made): planner episodes on fresh world seeds, with Bayes belief updates
(sensor accuracy 0.5 + 0.5 * 2^(-d/20), Sec. IV-A); every expanded tree node
exported by `dsp_plan_nodes` gives its features (`dsp_features`) and
argmax_a L(b, a). A network trained this way, without the allowed-action rule
or defer, looped on illegal or useless actions and gave a lower l0 than the
heuristic, so `train` writes only to the file given by `--out` and never to
the shipped weights.

PyTorch only holds device buffers here; every step of the computation runs in
the library's kernels.

    python -m paper_1802_06215_b300.learn api --iterations 4 --epochs 30
    python -m paper_1802_06215_b300.learn compare
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


class Belief:
    """Belief of one-robot Rock Sample: observed position and sampled mask,
    independent posteriors P(rock i good), and the belief counters (sensed good
    minus sensed bad per rock) that the planner and the policies read. The
    sensor's accuracy at squared distance d2 is thresh[d2] / 2^32, from the
    sensor table the model's kernels read (dsp_get_table)."""

    def __init__(self, cfg, pos_word, thresh, sampled=0):
        self.cfg = cfg
        self.pos = int(pos_word)
        self.sampled = int(sampled)
        self.thresh = np.asarray(thresh)
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
                d2 = ((c & 0xFF) - x) ** 2 + ((c >> 8) - y) ** 2
                q = float(self.thresh[d2]) / 4294967296.0
                like_good, like_bad = (q, 1 - q) if z == 1 else (1 - q, q)
                p = self.p[r]
                self.p[r] = p * like_good / (p * like_good + (1 - p) * like_bad)
                self.hist[r] = np.int8(max(-127, min(127, int(self.hist[r]) + (1 if z == 1 else -1))))
        self.pos = int(next_pos)
        self.sampled = int(next_sampled)


def start_word(cfg):
    return np.uint32(0 | ((cfg.n // 2) << 8))


def search_params(seconds, threads=4, xi=0.95, target_gap=0.0, rounds=10 ** 7):
    """Free-running search: `threads` x `rounds` trials at most, `seconds` of
    planning (0 = no time limit)."""
    return _dsp.dsp_search_params(threads=threads, rounds=rounds, time_limit_s=seconds, c_a=1.0, c_o=0.5,
                                  xi=xi, target_gap=target_gap, deterministic=0, use_queue=0)


def episode(model, cfg, world_seed, steps, seconds, threads=4, min_scen=16, node_cap=1 << 15, harvest=True,
            rounds=10 ** 7):
    """One planner episode. Returns the discounted return, the visited roots
    (state block, counters) and, when harvesting, the exported nodes."""
    rng = np.random.default_rng([world_seed, 0xBE11EF])
    world = inputs.rs_block(cfg, 1, rng, pos=[(0, cfg.n // 2)])
    world[4] = 0
    belief = Belief(cfg, world[0, 0], model.table(0))
    ret, disc = 0.0, 1.0
    roots, states, hists, labels, decisions, gaps = [], [], [], [], 0, []
    t_plan, expansions, scen_steps = 0.0, 0, 0
    for t in range(steps):
        K = cfg.K
        root = belief.scenarios(rng, K)
        roots.append((root, belief.hist.copy()))
        model.set_plan_step((world_seed * 1000 + t) & 0x7FFFFFFF)
        p = search_params(seconds, threads, rounds=rounds)
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
        expansions += res["expansions"]
        scen_steps += res["scenario_steps"]
        gaps.append(res["root_u"] - res["root_l"])
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
    out = {"return": ret, "roots": roots, "decisions": decisions, "plan_seconds": t_plan, "gaps": gaps,
           "expansions": expansions, "scenario_steps": scen_steps}
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


def imitation_labels(model, cfg, states, hist, actions):
    """The planner's chosen actions at tree nodes as training labels: |A|
    (defer to the heuristic) where the planner chose the heuristic's action,
    else the action. Returns (keep, labels): keep marks the pairs whose action
    the learned policy may take (the library's allowed-action rule)."""
    pos, sampled = states[0], states[3]
    keep = allowed_mask(model, cfg, pos, sampled, hist)[np.arange(len(actions)), actions]
    heur = heuristic_action(model, pos, sampled, hist)
    return keep, np.where(actions == heur, model.num_actions, actions).astype(np.int32)


def harvest(cfg, world_seeds, steps, seconds, policy=None, threads=4, min_scen=16, defer=True, log=print):
    """(features, labels) from planner episodes on the given world seeds: at
    every exported tree node (a belief with at least `min_scen` scenarios),
    the action the planner's search chose there. With `defer` the label is
    |A| ("defer to the heuristic") where the planner chose the heuristic's
    action, and pairs whose action the learned policy may not take (the
    library's allowed-action rule, which the learned rollout applies) are
    dropped. With `policy` (a dsp_mlp handle) the planner's rollouts use it."""
    model = batch.Model(cfg)
    if policy is not None:
        _dsp.dsp_set_policy(model.h, policy)
    X, Y, rets = [], [], []
    kept = seen = 0
    t0 = time.time()
    for s in world_seeds:
        ep = episode(model, cfg, s, steps, seconds, threads, min_scen)
        rets.append(ep["return"])
        if "states" in ep:
            y = ep["labels"].astype(np.int32)
            x = features(model, ep["states"], ep["hist"])
            if defer:
                ok, y = imitation_labels(model, cfg, ep["states"], ep["hist"], y)
                seen += len(y)
                kept += int(ok.sum())
                x, y = x[ok], y[ok]
            X.append(x)
            Y.append(y)
        log(f"world {s}: return {ep['return']:.2f}, {ep['decisions']} decisions, "
            f"{sum(len(y) for y in Y)} pairs, {time.time() - t0:.0f} s")
    model.close()
    if defer and seen:
        log(f"allowed pairs kept: {kept} of {seen}")
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


def _rs_block(pos, sampled):
    """State block of one-robot Rock Sample states given their positions and
    sampled masks (the other fields do not enter the policies)."""
    b = np.zeros((5, len(pos)), np.uint32)
    b[0] = pos
    b[3] = sampled
    return b


def allowed_mask(model, cfg, pos, sampled, hist):
    """(count, |A| + 1) bool: the actions the learned policy may take (the
    library's own rule, as the learned rollout applies it; column |A| defers
    to the heuristic)."""
    _, bits = _dsp.default_policy(model.h, _rs_block(pos, sampled), hist, want_allowed=True)
    return ((bits[:, None].astype(np.uint64) >> np.arange(6 + cfg.m, dtype=np.uint64)) & 1).astype(bool)


def heuristic_action(model, pos, sampled, hist):
    """The hand-written default policy's action (one robot), computed by the
    library's rollout policy."""
    return _dsp.default_policy(model.h, _rs_block(pos, sampled), hist)


def counter_posterior(c, q=0.85):
    """P(rock good) implied by a belief counter c (readings of a sensor of
    accuracy q): q^c / (q^c + (1-q)^c)."""
    c = np.clip(np.asarray(c, np.float64), -30, 30)
    return 1.0 / (1.0 + ((1 - q) / q) ** c)


def q_labels(model, cfg, pos, sampled, hist, depth, rng, Kq=128, chunk=2048, thr=0.25):
    """Conservative greedy labels of Q(s, a), estimated by one leaf expansion
    per state over Kq scenarios drawn from the belief the counters imply:
    Q(s, a) = sum over children of (reward sum + gamma * l0 sum) per scenario,
    the rollouts running the model's current default policy (common random
    numbers across actions). The label is |A| (defer to the heuristic) unless
    the best allowed action beats the heuristic's action by more than thr;
    then it is that action. Returns labels and that advantage."""
    m_ = cfg.m
    na = 5 + m_
    labels = np.zeros(len(pos), np.int32)
    margin = np.zeros(len(pos))
    al = allowed_mask(model, cfg, pos, sampled, hist)[:, :na]
    ha = heuristic_action(model, pos, sampled, hist)
    bits = np.arange(m_, dtype=np.uint32)
    for s0 in range(0, len(pos), chunk):
        jobs = []
        for i in range(s0, min(len(pos), s0 + chunk)):
            p = counter_posterior(hist[i, :m_])
            good = ((rng.random((Kq, m_)) < p).astype(np.uint32) << bits).sum(axis=1, dtype=np.uint32)
            b = np.zeros((5, Kq), np.uint32)
            b[0] = pos[i]
            b[2] = good & np.uint32(~int(sampled[i]) & 0xFFFFFFFF)
            b[3] = sampled[i]
            b[4] = rng.choice(cfg.K, Kq, replace=False).astype(np.uint32)
            jobs.append(inputs.Job(parent=b, idx=np.arange(Kq, dtype=np.uint16), last_action=-1,
                                   depth=int(depth[i]), hist=hist[i].astype(np.int8)))
        jb = batch.JobBatch(model, jobs)
        jb.run()
        res = jb.all_results()
        for k, r in enumerate(res):
            i = s0 + k
            q = np.full(model.num_actions, -np.inf)
            for a in range(model.num_actions):
                nc = int(r["child_count"][a])
                q[a] = (float(np.sum(r["rew"][a][:nc], dtype=np.float64)) +
                        cfg.gamma * float(np.sum(r["l"][a][:nc], dtype=np.float64))) / (2.0 ** 32 * Kq)
            q[~al[i]] = -np.inf
            best = int(np.argmax(q))
            margin[i] = q[best] - q[ha[i]]
            labels[i] = best if margin[i] > thr else na
    return labels, margin


def random_states(cfg, count, rng):
    """Observable Rock Sample states spread over the whole space: position
    uniform, each rock sampled with a per-state probability, counters zero or
    uniform in -3..3, depth uniform in 0..10."""
    x = rng.integers(0, cfg.n, count)
    y = rng.integers(0, cfg.n, count)
    pos = (x | (y << 8)).astype(np.uint32)
    ps = rng.random(count)[:, None]
    sampled = ((rng.random((count, cfg.m)) < ps).astype(np.uint32) << np.arange(cfg.m, dtype=np.uint32)).sum(
        axis=1, dtype=np.uint32)
    hist = np.zeros((count, 32), np.int8)
    c = rng.integers(-3, 4, (count, cfg.m)) * (rng.random((count, cfg.m)) < 0.5)
    hist[:, :cfg.m] = c
    depth = rng.integers(0, 11, count).astype(np.int32)
    return pos, sampled, hist, depth


def on_policy_states(model, cfg, pos, sampled, hist, depth, rng, per_rollout=6):
    """States the model's learned policy visits: one logged rollout from each
    given state (good rocks drawn from the counters' belief), replayed step by
    step with dsp_step to recover positions, sampled masks and counters, then
    per_rollout of the visited states chosen at random."""
    import torch
    N = len(pos)
    b = np.zeros((5, N), np.uint32)
    p = counter_posterior(hist[:, :cfg.m])
    b[0] = pos
    b[2] = ((rng.random((N, cfg.m)) < p).astype(np.uint32) << np.arange(cfg.m, dtype=np.uint32)).sum(
        axis=1, dtype=np.uint32) & ~sampled
    b[3] = sampled
    b[4] = rng.integers(0, cfg.K, N).astype(np.uint32)
    out = [[] for _ in range(4)]
    for d0 in np.unique(depth):
        sel = np.nonzero(depth == d0)[0]
        blk = np.ascontiguousarray(b[:, sel])
        n = len(sel)
        bd = torch.as_tensor(blk.view(np.int32), device="cuda")
        hd = torch.as_tensor(np.ascontiguousarray(hist[sel]), device="cuda")
        val = torch.empty(n, dtype=torch.float32, device="cuda")
        act = torch.full((n, cfg.D), -1, dtype=torch.int32, device="cuda")
        _dsp.dsp_rollout_logged(model.h, bd.data_ptr(), n, n, hd.data_ptr(), int(d0), val.data_ptr(),
                                act.data_ptr(), torch.cuda.current_stream().cuda_stream)
        acts = act.cpu().numpy()
        cur, h = blk, hist[sel].copy()
        visited = [[] for _ in range(n)]
        for t in range(cfg.D - int(d0)):
            live = np.nonzero(acts[:, t] >= 0)[0]
            if len(live) == 0:
                break
            for i in live:
                visited[i].append((cur[0, i], cur[3, i], h[i].copy(), int(d0) + t))
            nxt, keys, _ = model.step(np.ascontiguousarray(cur[:, live]), acts[live, t], int(d0) + t)
            a = acts[live, t]
            z = (keys & np.uint64(3)).astype(np.int64)
            sense = a >= SENSE0
            for j in np.nonzero(sense & (z > 0))[0]:
                r = a[j] - SENSE0
                i = live[j]
                h[i, r] = np.int8(max(-127, min(127, int(h[i, r]) + (1 if z[j] == 1 else -1))))
            cur = cur.copy()
            cur[:, live] = nxt
        for v in visited:
            if not v:
                continue
            for k in rng.choice(len(v), min(per_rollout, len(v)), replace=False):
                for o, e in zip(out, v[k]):
                    o.append(e)
    return (np.array(out[0], np.uint32), np.array(out[1], np.uint32), np.array(out[2], np.int8).reshape(-1, 32),
            np.array(out[3], np.int32))


def mean_rollout_value(model, cfg, pos, sampled, hist, depth, rng, reps=1):
    """Mean default-policy rollout value from the given states (good rocks
    drawn from the counters' belief) under the model's current policy."""
    import torch
    vals = []
    for _ in range(reps):
        N = len(pos)
        b = np.zeros((5, N), np.uint32)
        p = counter_posterior(hist[:, :cfg.m])
        b[0] = pos
        b[2] = ((rng.random((N, cfg.m)) < p).astype(np.uint32) << np.arange(cfg.m, dtype=np.uint32)).sum(
            axis=1, dtype=np.uint32) & ~sampled
        b[3] = sampled
        b[4] = rng.integers(0, cfg.K, N).astype(np.uint32)
        for d0 in np.unique(depth):
            sel = np.nonzero(depth == d0)[0]
            vals.append(model.rollout(np.ascontiguousarray(b[:, sel]), hist[sel], int(d0)))
    return float(np.mean(np.concatenate(vals)))


def policy_iteration(cfg, iterations=4, n_random=60000, n_onpolicy=4000, Kq=64, epochs=30, seed=0, init=None,
                     log=print):
    """Approximate policy iteration: at iteration k the labels are the greedy
    actions of Q^{pi_k} (pi_0 the heuristic) on random states plus the states
    pi_k's own rollouts visit; the network is trained on all labels so far
    and becomes pi_{k+1}."""
    rng = np.random.default_rng([seed, 0xA91])
    model = batch.Model(cfg)
    policy = None
    if init is not None:
        policy = _dsp.dsp_mlp_create(64, 0)
        _dsp.dsp_mlp_set_weights(policy, init)
        _dsp.dsp_set_policy(model.h, policy)
    Xs, Ys, hist_log = [], [], []
    ev = random_states(cfg, 4000, np.random.default_rng([seed, 0xE7A1]))
    start = (np.full(2000, start_word(cfg), np.uint32), np.zeros(2000, np.uint32), np.zeros((2000, 32), np.int8),
             np.zeros(2000, np.int32))
    _dsp.dsp_set_policy(model.h, None)
    base = {"random_states": mean_rollout_value(model, cfg, *ev, np.random.default_rng(1)),
            "start": mean_rollout_value(model, cfg, *start, np.random.default_rng(2))}
    log(json.dumps({"heuristic_value": base}))
    _dsp.dsp_set_policy(model.h, policy)
    for it in range(iterations):
        t0 = time.time()
        pos, sampled, hist, depth = random_states(cfg, n_random, rng)
        if policy is not None:
            seeds = random_states(cfg, n_onpolicy, rng)
            s2 = (np.concatenate([seeds[0], start[0][:n_onpolicy // 4]]),
                  np.concatenate([seeds[1], start[1][:n_onpolicy // 4]]),
                  np.concatenate([seeds[2], start[2][:n_onpolicy // 4]]),
                  np.concatenate([seeds[3], start[3][:n_onpolicy // 4]]))
            op = on_policy_states(model, cfg, *s2, rng)
            pos, sampled = np.concatenate([pos, op[0]]), np.concatenate([sampled, op[1]])
            hist, depth = np.concatenate([hist, op[2]]), np.concatenate([depth, op[3]])
        y, margin = q_labels(model, cfg, pos, sampled, hist, depth, rng, Kq=Kq)
        X = features(model, np.stack([pos, np.zeros_like(pos), np.zeros_like(pos), sampled, np.zeros_like(pos)]),
                     hist)
        Xs.append(X)
        Ys.append(y)
        t1 = time.time()
        h, acc = train(np.concatenate(Xs), np.concatenate(Ys), model.num_actions + 1, epochs=epochs,
                       seed=seed + it, log=lambda *_: None)
        if policy is not None:
            _dsp.dsp_mlp_destroy(policy)
        policy = h
        _dsp.dsp_set_policy(model.h, policy)
        val = {"random_states": mean_rollout_value(model, cfg, *ev, np.random.default_rng(1)),
               "start": mean_rollout_value(model, cfg, *start, np.random.default_rng(2))}
        rec = {"iteration": it + 1, "states": int(len(y)), "pairs": int(sum(len(v) for v in Ys)),
               "override_frac": float(np.mean(y != model.num_actions)),
               "val_accuracy": acc, "label_seconds": t1 - t0, "train_seconds": time.time() - t1,
               "learned_value": val, "heuristic_value": base}
        hist_log.append(rec)
        log(json.dumps(rec))
    model.close()
    return policy, hist_log


def run_episodes(cfg, world_seeds, steps, seconds, policy=None, threads=4, rounds=10 ** 7):
    """Planner episodes on the given worlds (Sec. IV-A task, belief updated by
    Bayes' rule after every real step): mean discounted return, decisions per
    second of planning time and mean root gap at decision time; `policy` (a
    dsp_mlp handle) replaces the heuristic default policy in the rollouts.
    Each decision plans for `seconds` (0 = no limit) and at most `threads` x
    `rounds` trials."""
    model = batch.Model(cfg)
    _dsp.dsp_set_policy(model.h, policy)
    rets, dec, secs, gaps, exps, ssteps = [], 0, 0.0, [], 0, 0
    for s in world_seeds:
        ep = episode(model, cfg, s, steps, seconds, threads, harvest=False, rounds=rounds)
        rets.append(ep["return"])
        dec += ep["decisions"]
        secs += ep["plan_seconds"]
        gaps += ep["gaps"]
        exps += ep["expansions"]
        ssteps += ep["scenario_steps"]
    model.close()
    return {"worlds": len(rets), "mean_return": float(np.mean(rets)), "min_return": float(np.min(rets)),
            "decisions": dec, "plan_seconds": secs, "decisions_per_s": dec / max(secs, 1e-9),
            "mean_root_gap": float(np.mean(gaps)), "expansions": exps,
            "expansions_per_s": exps / max(secs, 1e-9), "scenario_steps_per_s": ssteps / max(secs, 1e-9)}


# ---------------------------------------------------------------- the car ----

def car_heuristic_action(model, block):
    """The car's hand-written default policy on a state block, computed by
    the library's rollout policy."""
    return _dsp.default_policy(model.h, block)


def car_states(cfg, count, rng):
    """Car states spread over the task: s uniform on [0, 58) m, speed uniform
    on 0..3, pedestrians uniform on the 40 x 40 m region, goals drawn per
    scenario later; depth uniform in 0..10."""
    b = inputs.car_block(cfg, count, rng)
    b[0] = rng.uniform(0.0, 58.0, count).astype(np.float32).view(np.uint32)
    depth = rng.integers(0, 11, count).astype(np.int32)
    return b, depth


def car_belief_block(cfg, state_col, Kq, rng):
    """Kq scenarios of one car state: position, speed and pedestrian positions
    as observed, hidden goals drawn uniformly (the belief over them)."""
    P = cfg.P
    s = float(state_col[0:1].view(np.float32)[0])
    v = int(state_col[1] & 0xFF)
    base = (state_col[4:4 + P].view(np.float32).astype(np.float64), state_col[4 + P:4 + 2 * P].view(np.float32)
            .astype(np.float64))
    b = inputs.car_block(cfg, Kq, rng, s=s, v=v, base=base, jitter=0.0,
                         scen=rng.choice(cfg.K, Kq, replace=False))
    b[0] = state_col[0]
    b[4:4 + 2 * P] = state_col[4:4 + 2 * P, None]
    return b


def car_q_labels(model, cfg, block, depth, rng, Kq=64, chunk=1024, thr=2.0):
    """Conservative greedy labels for car states, as q_labels: Q(s, a) from one
    leaf expansion over Kq goal-belief scenarios (rollouts with the model's
    current default policy); label 3 (defer) unless the best action beats the
    heuristic's by more than thr."""
    n = block.shape[1]
    labels = np.zeros(n, np.int32)
    ha = car_heuristic_action(model, block)
    na = model.num_actions
    for s0 in range(0, n, chunk):
        jobs = []
        for i in range(s0, min(n, s0 + chunk)):
            b = car_belief_block(cfg, block[:, i], Kq, rng)
            jobs.append(inputs.Job(parent=b, idx=np.arange(Kq, dtype=np.uint16), last_action=-1, depth=int(depth[i]),
                                   hist=np.zeros(32, np.int8)))
        jb = batch.JobBatch(model, jobs)
        jb.run()
        for k, r in enumerate(jb.all_results()):
            i = s0 + k
            q = np.zeros(na)
            for a in range(na):
                nc = int(r["child_count"][a])
                q[a] = (float(np.sum(r["rew"][a][:nc], dtype=np.float64)) +
                        cfg.gamma * float(np.sum(r["l"][a][:nc], dtype=np.float64))) / (2.0 ** 32 * Kq)
            best = int(np.argmax(q))
            labels[i] = best if q[best] - q[ha[i]] > thr else na
    return labels


def car_features(model, block):
    import torch
    n = block.shape[1]
    b = torch.as_tensor(np.ascontiguousarray(block).view(np.int32), device="cuda")
    f = torch.empty((n, 64), dtype=torch.float32, device="cuda")
    _dsp.dsp_features(model.h, b.data_ptr(), n, n, 0, f.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return f.cpu().numpy()


def car_on_policy_states(model, cfg, block, depth, rng, per_rollout=4):
    """States the model's learned car policy visits: logged rollouts from the
    given states, replayed with dsp_step, per_rollout visited states each."""
    import torch
    out_cols, out_depth = [], []
    for d0 in np.unique(depth):
        sel = np.nonzero(depth == d0)[0]
        cur = np.ascontiguousarray(block[:, sel])
        n = len(sel)
        bd = torch.as_tensor(cur.view(np.int32), device="cuda")
        val = torch.empty(n, dtype=torch.float32, device="cuda")
        act = torch.full((n, cfg.D), -1, dtype=torch.int32, device="cuda")
        _dsp.dsp_rollout_logged(model.h, bd.data_ptr(), n, n, 0, int(d0), val.data_ptr(), act.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        acts = act.cpu().numpy()
        visited = [[] for _ in range(n)]
        for t in range(cfg.D - int(d0)):
            live = np.nonzero(acts[:, t] >= 0)[0]
            if len(live) == 0:
                break
            for i in live:
                visited[i].append(t)
            nxt, _, _ = model.step(np.ascontiguousarray(cur[:, live]), acts[live, t], int(d0) + t)
            cur = cur.copy()
            for col, i in enumerate(live):
                if len(visited[i]) and rng.random() < per_rollout / max(1, cfg.D - int(d0)):
                    out_cols.append(cur[:, i].copy())
                    out_depth.append(int(d0) + t)
            cur[:, live] = nxt
    if not out_cols:
        return np.zeros((block.shape[0], 0), np.uint32), np.zeros(0, np.int32)
    return np.stack(out_cols, axis=1), np.array(out_depth, np.int32)


def car_mean_value(model, cfg, block, depth, rng):
    vals = []
    for d0 in np.unique(depth):
        sel = np.nonzero(depth == d0)[0]
        b = np.ascontiguousarray(block[:, sel]).copy()
        # hidden goals as the belief draws them
        b[4 + 2 * cfg.P:] = inputs.car_block(cfg, len(sel), rng)[4 + 2 * cfg.P:]
        vals.append(model.rollout(b, None, int(d0)))
    return float(np.mean(np.concatenate(vals)))


def car_policy_iteration(cfg, iterations=3, n_random=12000, n_onpolicy=2000, Kq=64, epochs=30, seed=0,
                         log=print):
    """Approximate policy iteration for the car (as policy_iteration)."""
    rng = np.random.default_rng([seed, 0xCA2])
    model = batch.Model(cfg)
    policy = None
    Xs, Ys, hist_log = [], [], []
    ev_b, ev_d = car_states(cfg, 3000, np.random.default_rng([seed, 0xE7A2]))
    base = {"random_states": car_mean_value(model, cfg, ev_b, ev_d, np.random.default_rng(1))}
    log(json.dumps({"heuristic_value": base}))
    for it in range(iterations):
        t0 = time.time()
        b, d = car_states(cfg, n_random, rng)
        if policy is not None:
            sb, sd = car_states(cfg, n_onpolicy, rng)
            ob, od = car_on_policy_states(model, cfg, sb, sd, rng)
            b, d = np.concatenate([b, ob], axis=1), np.concatenate([d, od])
        y = car_q_labels(model, cfg, b, d, rng, Kq=Kq)
        X = car_features(model, b)
        Xs.append(X)
        Ys.append(y)
        t1 = time.time()
        h, acc = train(np.concatenate(Xs), np.concatenate(Ys), model.num_actions + 1, epochs=epochs, seed=seed + it,
                       log=lambda *_: None)
        if policy is not None:
            _dsp.dsp_mlp_destroy(policy)
        policy = h
        _dsp.dsp_set_policy(model.h, policy)
        val = {"random_states": car_mean_value(model, cfg, ev_b, ev_d, np.random.default_rng(1))}
        rec = {"iteration": it + 1, "states": int(len(y)), "pairs": int(sum(len(v) for v in Ys)),
               "override_frac": float(np.mean(y != model.num_actions)), "val_accuracy": acc,
               "label_seconds": t1 - t0, "train_seconds": time.time() - t1, "learned_value": val,
               "heuristic_value": base}
        hist_log.append(rec)
        log(json.dumps(rec))
    model.close()
    return policy, hist_log


def car_roots(cfg, count, seed):
    """Planning roots of the car: at the start of the path, at rest, each with
    its own pedestrian layout and K goal-belief scenarios."""
    roots = []
    for k in range(count):
        rng = np.random.default_rng([seed, k])
        base = (rng.uniform(0, 40, cfg.P), rng.uniform(0, 40, cfg.P))
        roots.append((inputs.car_block(cfg, cfg.K, rng, s=0.0, v=0, base=base, jitter=0.0), None))
    return roots


def compare(cfg, policy, roots, seconds, threads=4, xi=0.95, target_gap=0.0):
    """Root gap u - l after one planning step of `seconds` from each root
    belief, heuristic pi0 then learned pi0, on the same random streams. With
    xi = 0 and target_gap = 0 a search stops at its time limit only (a path
    ends at a zero-gap node or depth D), so both policies plan for the same
    time; each arm reports the seconds it took."""
    model = batch.Model(cfg)
    rows = []
    for k, (root, hist) in enumerate(roots):
        row = {}
        for name, pol in (("heuristic", None), ("learned", policy)):
            _dsp.dsp_set_policy(model.h, pol)
            model.set_plan_step(0x40000000 + k)
            r = _dsp.dsp_plan(model.h, root, hist, search_params(seconds, threads, xi, target_gap),
                              model.num_actions)
            row[name] = {"gap": r["root_u"] - r["root_l"], "u": r["root_u"], "l": r["root_l"],
                         "action": int(r["action"]), "expansions": r["expansions"], "seconds": r["seconds"]}
        rows.append(row)
    model.close()
    out = {"beliefs": len(rows), "planning_time_s": seconds, "threads": threads, "xi": xi,
           "target_gap": target_gap}
    for name in ("heuristic", "learned"):
        secs = [r[name]["seconds"] for r in rows]
        out[name] = {"mean_root_gap": float(np.mean([r[name]["gap"] for r in rows])),
                     "mean_root_l": float(np.mean([r[name]["l"] for r in rows])),
                     "mean_root_u": float(np.mean([r[name]["u"] for r in rows])),
                     "mean_expansions": float(np.mean([r[name]["expansions"] for r in rows])),
                     "mean_seconds": float(np.mean(secs)), "min_seconds": float(np.min(secs)),
                     "max_seconds": float(np.max(secs)),
                     # searches that ended before 95 % of the budget: with the root gap
                     # closed (nothing left to plan), or for another reason
                     "ended_early_gap_closed": int(sum(r[name]["seconds"] < 0.95 * seconds and
                                                       r[name]["gap"] <= 1e-9 for r in rows)),
                     "ended_early_other": int(sum(r[name]["seconds"] < 0.95 * seconds and
                                                  r[name]["gap"] > 1e-9 for r in rows)),
                     "decisions_per_s": len(rows) / sum(secs)}
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
    ap.add_argument("cmd", choices=["train", "api", "compare", "api-car", "compare-car"])
    ap.add_argument("--worlds", type=int, default=32)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--plan-seconds", type=float, default=0.1)
    ap.add_argument("--iterations", type=int, default=2, help="harvest/train rounds (later ones roll out the net)")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--weights", default=None, help="weights file (default: the shipped one of the task)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--init", default=None, help="api: start from these weights (e.g. the imitation network)")
    ap.add_argument("--eval-worlds", type=int, default=8)
    ap.add_argument("--eval-steps", type=int, default=8)
    ap.add_argument("--eval-seconds", type=float, default=1.0)
    a = ap.parse_args(argv)
    from . import build
    build.build()
    cfg = inputs.rs15_15()
    if a.cmd == "api-car":
        ccfg = inputs.car50()
        policy, hl = car_policy_iteration(ccfg, iterations=a.iterations, epochs=a.epochs)
        save_weights(a.out or "paper_1802_06215_b300/weights/car50_pi0.npz", policy,
                     {"config": "car50", "method": "approximate policy iteration", "iterations": hl})
        return
    if a.cmd == "compare-car":
        ccfg = inputs.car50()
        policy, meta = load_weights(a.weights or "paper_1802_06215_b300/weights/car50_pi0.npz")
        print(json.dumps(compare(ccfg, policy, car_roots(ccfg, a.eval_worlds, 9000), a.eval_seconds)))
        return
    if a.cmd == "api":
        init, init_meta = None, None
        if a.init:
            z = np.load(a.init)
            init, init_meta = z["params"], json.loads(str(z["meta"]))
        policy, hl = policy_iteration(cfg, iterations=a.iterations, epochs=a.epochs, init=init)
        meta = {"config": "rs15_15", "method": "approximate policy iteration", "iterations": hl}
        if init_meta is not None:
            meta.update({"method": "planner imitation, then approximate policy iteration", "init": init_meta})
        save_weights(a.out or a.weights or "paper_1802_06215_b300/weights/rs15_15_pi0.npz", policy, meta)
    elif a.cmd == "train":
        if not a.out:
            ap.error("train (planner imitation) needs --out")
        policy, init, meta = None, None, {"iterations": []}
        X_all, Y_all = [], []
        for it in range(a.iterations):
            seeds = list(range(1000 + it * a.worlds, 1000 + (it + 1) * a.worlds))
            X, Y, rets = harvest(cfg, seeds, a.steps, a.plan_seconds, policy=policy)
            X_all.append(X)
            Y_all.append(Y)
            # 20 actions and the defer label
            h, acc = train(np.concatenate(X_all), np.concatenate(Y_all), 21, epochs=a.epochs, seed=it)
            meta["iterations"].append({"worlds": seeds, "pairs": int(sum(len(y) for y in Y_all)),
                                       "mean_return": float(np.mean(rets)), "val_accuracy": acc})
            print(json.dumps(meta["iterations"][-1]))
            if policy is not None:
                _dsp.dsp_mlp_destroy(policy)
            policy = h
        meta.update({"config": "rs15_15", "method": "planner imitation (defer labels, allowed actions)",
                     "steps": a.steps,
                     "plan_seconds": a.plan_seconds, "epochs": a.epochs})
        save_weights(a.out, policy, meta)
    else:
        policy, meta = load_weights(a.weights or "paper_1802_06215_b300/weights/rs15_15_pi0.npz")
        roots = eval_roots(cfg, range(9000, 9000 + a.eval_worlds), a.eval_steps, 0.05)
        print(json.dumps(compare(cfg, policy, roots, a.eval_seconds)))


if __name__ == "__main__":
    main()
