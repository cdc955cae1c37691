// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// Plain, single-threaded restatement of DESPOT leaf expansion and of the
// HyP-DESPOT tree search, step by step in the paper's order:
//  * leaf initialisation (Sec. III-A, Sec. III-D): gather the leaf's scenarios
//    from its parent and apply the last action ("update"), step every
//    (action, scenario) pair with g (Eq. expand), split each action's scenarios
//    by observation into children (Eq. newnodes), and give each child the
//    heuristic upper bound (Eq. ub) and the default-policy lower bound rolled
//    out to depth D with a tail heuristic (Eq. lb);
//  * forward search with scenario-based PO-UCT for actions (Eq. UCT),
//    weighted excess uncertainty minus virtual loss for observations
//    (Eq. select_lb, Eq. augmented_WEU), and the Bellman backup (Eq. backup);
//  * exhaustive expansion to depth D of the same scenario tree, the optimal
//    value the bounds must bracket.
//
// Readings where the paper is silent: per-scenario values are in the model's Real
// type in time order; sums over scenarios are exact int64 fixed point with
// scale 2^-32; children are ordered by the first position at which their
// observation occurs, members in their original order; node values are kept
// weighted by |Phi_b|/K; a trial descends to one leaf, expands it and backs
// up; "deterministic rounds" run the selection of T trials in thread order,
// then their expansions, then their backups in thread order.
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <limits>
#include <memory>
#include <utility>
#include <vector>

#include "car.hpp"
#include "rocksample.hpp"
#include "nav.hpp"

namespace orc {

inline int64_t to_fixed(double x) { return (int64_t)std::llrint(x * 4294967296.0); }
inline double from_fixed(int64_t f) { return (double)f / 4294967296.0; }

// Observation equality beyond the key: exact for Rock Sample (the key is the
// observation), the full cell vector for the car.
template <class R>
bool same_obs(const RockSample<R>&, const RSState&, const RSState&) {
  return true;
}
template <class R>
bool same_obs(const Car<R>& m, const CarState<R>& a, const CarState<R>& b) {
  return m.observe_state(a) == m.observe_state(b);
}
template <class R>
bool same_obs(const Nav<R>&, const NavState&, const NavState&) {
  return true;
}

// Eq. lb for one scenario: roll the default policy from depth t0 until the
// state is terminal or depth D, discounting rewards by gamma^(t - t0), then add
// gamma^(D - t0) times the tail heuristic if the horizon was reached.
template <class M, class S>
auto rollout(const M& m, S s, Hist h, int t0, uint64_t* steps) -> decltype(m.upper(s)) {
  using Real = decltype(m.upper(s));
  Real v = (Real)0;
  int t = t0;
  while (t < m.D && !m.terminal(s)) {
    int a = m.policy(s, h);
    S next;
    uint64_t key;
    Real r = m.step(s, a, t, next, &key);
    *steps += 1;
    m.observe(h, a, key);
    count_ops(6);  // loop and terminal tests, discount lookup, multiply, add, depth increment
    v = v + m.G[t - t0] * r;
    s = next;
    t += 1;
  }
  if (!m.terminal(s)) v = v + m.G[m.D - t0] * m.tail(s);
  return v;
}

template <class S>
struct ExpandOut {
  int n = 0, na = 0, cap = 0;
  std::vector<S> leaf;                // the leaf's own (updated) scenario states
  std::vector<int32_t> child_count;   // [na]
  std::vector<int32_t> child_off;     // [na][cap + 1]
  std::vector<uint64_t> key;          // [na][cap]
  std::vector<int64_t> rew, u, l;     // [na][cap], fixed point 2^-32
  std::vector<uint16_t> perm;         // [na][n], positions in the leaf, grouped by child
  uint64_t steps = 0;                 // g calls on live scenarios
};

// Leaf initialisation of one leaf b at depth `depth` (Sec. III-D).
template <class M, class S>
void expand_leaf(const M& m, const std::vector<S>& parent, const uint16_t* idx, int n, int last_action,
                 int depth, const Hist& h, int a0, int na, int cap, ExpandOut<S>& out) {
  using Real = decltype(m.upper(parent[0]));
  out.n = n;
  out.na = na;
  out.cap = cap;
  out.steps = 0;
  // gather + update (the leaf stores only indexes into its parent's list)
  out.leaf.resize(n);
  for (int p = 0; p < n; ++p) {
    S s = parent[idx[p]];
    if (last_action >= 0) {
      S next;
      uint64_t key;
      if (!m.terminal(s)) out.steps += 1;
      m.step(s, last_action, depth - 1, next, &key);
      s = next;
    }
    out.leaf[p] = s;
  }
  out.child_count.assign(na, 0);
  out.child_off.assign((size_t)na * (cap + 1), 0);
  out.key.assign((size_t)na * cap, 0);
  out.rew.assign((size_t)na * cap, 0);
  out.u.assign((size_t)na * cap, 0);
  out.l.assign((size_t)na * cap, 0);
  out.perm.assign((size_t)na * n, 0);
  std::vector<S> next(n);
  std::vector<uint64_t> keys(n);
  std::vector<Real> rew(n);
  for (int ai = 0; ai < na; ++ai) {
    int a = a0 + ai;
    // Eq. expand: s', z = g(s, a, phi) for every scenario of the leaf
    for (int p = 0; p < n; ++p) {
      if (!m.terminal(out.leaf[p])) out.steps += 1;
      rew[p] = m.step(out.leaf[p], a, depth, next[p], &keys[p]);
    }
    // Eq. newnodes: one child per distinct observation, in order of first
    // occurrence; members keep their original order
    std::vector<int> first;             // first position of each child
    std::vector<std::vector<int>> members;
    for (int p = 0; p < n; ++p) {
      int c = -1;
      for (size_t k = 0; k < first.size(); ++k) {
        int q = first[k];
        if (keys[q] == keys[p] && same_obs(m, next[q], next[p])) {
          c = (int)k;
          break;
        }
      }
      if (c < 0) {
        first.push_back(p);
        members.push_back({});
        c = (int)first.size() - 1;
      }
      members[c].push_back(p);
    }
    int nc = (int)first.size();
    out.child_count[ai] = nc;
    int off = 0;
    for (int c = 0; c < nc; ++c) {
      out.child_off[(size_t)ai * (cap + 1) + c] = off;
      out.key[(size_t)ai * cap + c] = keys[first[c]];
      int64_t sr = 0, su = 0, sl = 0;
      for (int p : members[c]) {
        out.perm[(size_t)ai * n + off] = (uint16_t)p;
        off += 1;
        // Eq. ub: the heuristic of the child's state (the tail at depth D)
        Real uval = (depth + 1 >= m.D) ? m.tail(next[p]) : m.upper(next[p]);
        if (m.terminal(next[p])) uval = (Real)0;
        // Eq. lb: default-policy rollout from the child's depth
        Hist h2 = h;
        m.observe(h2, a, keys[p]);
        Real lval = rollout(m, next[p], h2, depth + 1, &out.steps);
        sr += to_fixed((double)rew[p]);
        su += to_fixed((double)uval);
        sl += to_fixed((double)lval);
      }
      out.rew[(size_t)ai * cap + c] = sr;
      out.u[(size_t)ai * cap + c] = su;
      out.l[(size_t)ai * cap + c] = sl;
    }
    out.child_off[(size_t)ai * (cap + 1) + nc] = off;
  }
}

// ---------------------------------------------------------------- search ---

struct SearchParams {
  int threads = 1;        // T search threads (trials per round)
  int rounds = 100;       // trial rounds (budget)
  double c_a = 0.0;       // PO-UCT exploration scale (Eq. UCT)
  double c_o = 0.0;       // virtual-loss scale (Eq. augmented_WEU)
  double xi = 0.95;       // target uncertainty ratio (Eq. select_lb)
  double target_gap = 0;  // stop when the root gap is at most this
};

template <class S>
struct VNode;

template <class S>
struct QNode {
  double R = 0, U = 0, L = 0;  // weighted step reward and bounds
  std::vector<VNode<S>*> children;
};

template <class S>
struct VNode {
  int depth = 0;
  double W = 1;  // |Phi_b| / K
  int n = 0;     // |Phi_b|
  VNode* parent = nullptr;
  int parent_action = -1;
  std::vector<uint16_t> pos;  // positions in the parent's scenario list
  std::vector<S> states;      // own states, present once expanded (root: given)
  Hist hist{};
  uint64_t key = 0;
  bool term = false;
  double U = 0, L = 0;  // weighted bounds
  int N = 0;
  std::vector<int> Na;
  bool expanded = false;
  bool claimed = false;
  int vl = 0;
  std::vector<QNode<S>> q;
};

struct SearchResult {
  double root_u = 0, root_l = 0;
  int action = -1;
  int nodes = 0, expansions = 0, rounds = 0;
  uint64_t steps = 0;
  uint64_t signature = 0;  // digest of the tree in creation order
  std::vector<int> root_na;
};

template <class M, class S>
struct Despot {
  const M& m;
  SearchParams prm;
  std::vector<std::unique_ptr<VNode<S>>> pool;
  VNode<S>* root = nullptr;
  uint64_t steps = 0;
  int expansions = 0;

  Despot(const M& model, const SearchParams& p) : m(model), prm(p) {}

  VNode<S>* new_node() {
    pool.emplace_back(new VNode<S>());
    return pool.back().get();
  }

  void expand(VNode<S>* b) {
    int na = m.num_actions();
    int cap = b->n;
    ExpandOut<S> e;
    if (b->parent == nullptr) {
      std::vector<uint16_t> ident(b->n);
      for (int i = 0; i < b->n; ++i) ident[i] = (uint16_t)i;
      expand_leaf(m, b->states, ident.data(), b->n, -1, b->depth, b->hist, 0, na, cap, e);
    } else {
      expand_leaf(m, b->parent->states, b->pos.data(), b->n, b->parent_action, b->depth, b->hist, 0, na,
                  cap, e);
    }
    steps += e.steps;
    expansions += 1;
    b->states = e.leaf;
    b->expanded = true;
    b->q.assign(na, QNode<S>());
    b->Na.assign(na, 0);
    double K = (double)m.K;
    double gamma = (double)m.gamma;
    for (int a = 0; a < na; ++a) {
      QNode<S>& q = b->q[a];
      int nc = e.child_count[a];
      int64_t rsum = 0;
      for (int c = 0; c < nc; ++c) rsum += e.rew[(size_t)a * cap + c];
      q.R = from_fixed(rsum) / K;
      double su = 0, sl = 0;
      for (int c = 0; c < nc; ++c) {
        VNode<S>* ch = new_node();
        int o0 = e.child_off[(size_t)a * (cap + 1) + c], o1 = e.child_off[(size_t)a * (cap + 1) + c + 1];
        ch->depth = b->depth + 1;
        ch->n = o1 - o0;
        ch->W = (double)ch->n / K;
        ch->parent = b;
        ch->parent_action = a;
        ch->pos.assign(e.perm.begin() + (size_t)a * b->n + o0, e.perm.begin() + (size_t)a * b->n + o1);
        ch->key = e.key[(size_t)a * cap + c];
        ch->term = (ch->key >> 62) & 1u;
        ch->hist = b->hist;
        m.observe(ch->hist, a, ch->key);
        ch->U = from_fixed(e.u[(size_t)a * cap + c]) / K;
        ch->L = from_fixed(e.l[(size_t)a * cap + c]) / K;
        q.children.push_back(ch);
        su += ch->U;
        sl += ch->L;
      }
      q.U = q.R + gamma * su;
      q.L = q.R + gamma * sl;
    }
    refresh(b);
  }

  // Eq. backup for one node from its action values.
  void refresh(VNode<S>* b) {
    double bu = -std::numeric_limits<double>::infinity(), bl = bu;
    for (auto& q : b->q) {
      bu = std::max(bu, q.U);
      bl = std::max(bl, q.L);
    }
    b->U = bu;
    b->L = bl;
  }
  void refresh_action(VNode<S>* b, int a) {
    QNode<S>& q = b->q[a];
    double su = 0, sl = 0;
    for (auto* c : q.children) {
      su += c->U;
      sl += c->L;
    }
    double gamma = (double)m.gamma;
    q.U = q.R + gamma * su;
    q.L = q.R + gamma * sl;
  }

  // Eq. UCT: scenario-based PO-UCT over normalised action upper bounds.
  int choose_action(VNode<S>* b) {
    int best = 0;
    double bestv = -std::numeric_limits<double>::infinity();
    for (int a = 0; a < (int)b->q.size(); ++a) {
      double v = b->q[a].U / b->W;
      if (prm.c_a != 0) {
        if (b->Na[a] == 0)
          v = std::numeric_limits<double>::infinity();
        else
          v += prm.c_a * std::sqrt(std::log((double)b->n * b->N) / ((double)b->n * b->Na[a]));
      }
      if (v > bestv) {
        bestv = v;
        best = a;
      }
    }
    return best;
  }

  struct Trial {
    std::vector<VNode<S>*> path;
    std::vector<int> acts;
    VNode<S>* leaf = nullptr;
  };

  // Forward search of one trial (Sec. III-C).
  Trial select() {
    Trial t;
    VNode<S>* b = root;
    t.path.push_back(b);
    while (true) {
      if (!b->expanded) {
        if (b->depth < m.D && !b->term && !b->claimed) {
          b->claimed = true;
          t.leaf = b;
        }
        return t;
      }
      b->N += 1;
      int a = choose_action(b);
      b->Na[a] += 1;
      double eps0 = root->U - root->L;
      VNode<S>* best = nullptr;
      double beste = -std::numeric_limits<double>::infinity();
      for (auto* c : b->q[a].children) {
        // Eq. select_lb minus the virtual loss of Eq. augmented_WEU
        double e = (c->U - c->L) - c->W * prm.xi * eps0 - prm.c_o * eps0 * (double)c->vl;
        if (e > beste) {
          beste = e;
          best = c;
        }
      }
      t.acts.push_back(a);
      if (best == nullptr || !(beste > 0)) return t;
      best->vl += 1;
      t.path.push_back(best);
      b = best;
    }
  }

  void backup(Trial& t) {
    // the path's last node is either the expanded leaf (already refreshed) or
    // the node where the trial stopped
    for (int i = (int)t.path.size() - 1; i >= 0; --i) {
      VNode<S>* b = t.path[i];
      if (i < (int)t.acts.size() && b->expanded) {
        refresh_action(b, t.acts[i]);
        refresh(b);
      }
      if (i > 0) b->vl -= 1;
    }
  }

  SearchResult plan(const std::vector<S>& root_states, const Hist& root_hist) {
    root = new_node();
    root->n = (int)root_states.size();
    root->W = (double)root->n / (double)m.K;
    root->states = root_states;
    root->hist = root_hist;
    int rounds = 0;
    for (int r = 0; r < prm.rounds; ++r) {
      std::vector<Trial> trials;
      for (int th = 0; th < prm.threads; ++th) trials.push_back(select());
      bool any = false;
      for (auto& t : trials)
        if (t.leaf) {
          expand(t.leaf);
          any = true;
        }
      for (auto& t : trials) backup(t);
      for (auto& t : trials)
        if (t.leaf) t.leaf->claimed = false;
      rounds += 1;
      if (root->expanded && root->U - root->L <= prm.target_gap) break;
      if (!any) break;
    }
    SearchResult res;
    res.root_u = root->U;
    res.root_l = root->L;
    res.nodes = (int)pool.size();
    res.expansions = expansions;
    res.rounds = rounds;
    res.steps = steps;
    int best = -1;
    double bl = -std::numeric_limits<double>::infinity();
    for (int a = 0; a < (int)root->q.size(); ++a)
      if (root->q[a].L > bl) {
        bl = root->q[a].L;
        best = a;
      }
    res.action = best;
    res.root_na = root->Na;
    uint64_t sig = 0x12345678ull;
    for (auto& up : pool) {
      VNode<S>* v = up.get();
      uint64_t ub, lb;
      std::memcpy(&ub, &v->U, 8);
      std::memcpy(&lb, &v->L, 8);
      sig = splitmix64_mix(sig ^ (uint64_t)v->depth) ^ v->key;
      sig = splitmix64_mix(sig ^ ub) ^ lb;
      sig = splitmix64_mix(sig ^ (uint64_t)v->n ^ ((uint64_t)v->N << 32));
    }
    res.signature = sig;
    return res;
  }
};

// Optimal value of the D-horizon scenario tree (every action, every observed
// branch), in the model's Real type for steps and FP64 for the recursion.
template <class M, class S>
double exhaustive_value(const M& m, const std::vector<S>& states, const Hist& h, int depth) {
  int n = (int)states.size();
  bool all_term = true;
  for (auto& s : states)
    if (!m.terminal(s)) all_term = false;
  if (all_term) return 0.0;
  if (depth >= m.D) {
    double l = 0;
    for (auto& s : states)
      if (!m.terminal(s)) l += (double)m.tail(s);
    return l / n;
  }
  double best = -std::numeric_limits<double>::infinity();
  for (int a = 0; a < m.num_actions(); ++a) {
    std::vector<S> next(n);
    std::vector<uint64_t> keys(n);
    double rsum = 0;
    for (int p = 0; p < n; ++p) rsum += (double)m.step(states[p], a, depth, next[p], &keys[p]);
    std::vector<int> first;
    std::vector<std::vector<S>> groups;
    for (int p = 0; p < n; ++p) {
      int c = -1;
      for (size_t k = 0; k < first.size(); ++k)
        if (keys[first[k]] == keys[p] && same_obs(m, next[first[k]], next[p])) {
          c = (int)k;
          break;
        }
      if (c < 0) {
        first.push_back(p);
        groups.push_back({});
        c = (int)first.size() - 1;
      }
      groups[c].push_back(next[p]);
    }
    double v = rsum / n;
    for (size_t c = 0; c < groups.size(); ++c) {
      Hist h2 = h;
      m.observe(h2, a, keys[first[c]]);
      v += (double)m.gamma * ((double)groups[c].size() / n) * exhaustive_value(m, groups[c], h2, depth + 1);
    }
    best = std::max(best, v);
  }
  return best;
}

}  // namespace orc
