// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// A POMCP-style planner (the single-scenario-per-path variant the paper names
// among its future directions, Sec. V) over the same models and scenario
// streams: UCT over histories, each simulation carrying one scenario down the
// tree and a default-policy rollout at the first new node.
//
// Batched reading (where the paper is silent; it is what lets rollouts go to a GPU
// in batches): a round runs `batch` simulations level by level. Simulation i
// of the plan takes root scenario i mod n. At each level the live simulations,
// in index order, choose an action at their node by UCB1 on the action values
// as they stood at the round's start plus one virtual visit per earlier
// choice of the same action at the same node in this round (an unvisited
// action first, lowest index on ties), step their scenario with g at that
// depth, and go to the child of (action, observation), creating it if new. A
// simulation stops at a terminal outcome (value 0 below it), at depth D (value
// 0), or at a node created in this round, where it rolls out the default
// policy from its scenario with the node's history. Then, in index order, each
// simulation backs up its discounted return along its path:
// N(h) += 1, N(h, a) += 1, Q(h, a) += (G - Q(h, a)) / N(h, a).
// Nodes are numbered in creation order (level, then simulation index).
#pragma once
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

#include "despot.hpp"

namespace orc {

struct PomcpParams {
  int rounds = 10;
  int batch = 64;
  double c = 1.0;  // UCB1 exploration constant
};

struct PomcpResult {
  int action = -1;
  double value = 0;
  int nodes = 0, simulations = 0, rollouts = 0;
  uint64_t steps = 0;
  uint64_t signature = 0;
  std::vector<double> root_q;
  std::vector<int> root_na;
};

template <class M, class S>
struct Pomcp {
  struct Child {
    uint64_t key;
    int node;
  };
  struct Node {
    int depth = 0;
    int born = -1;  // round that created it
    bool term = false;
    Hist hist{};
    uint64_t key = 0;
    long long N = 0;
    std::vector<long long> Na;
    std::vector<double> Q;
    std::vector<std::vector<Child>> ch;  // per action
  };
  struct Sim {
    S s;
    int node = 0;
    bool live = true;
    bool rollout = false;
    std::vector<int> nodes, acts;
    std::vector<double> rew;
    double leaf = 0;
  };

  const M& m;
  PomcpParams prm;
  std::vector<Node> tree;
  uint64_t steps = 0;

  Pomcp(const M& model, const PomcpParams& p) : m(model), prm(p) {}

  int new_node(int depth, int born, const Hist& h, uint64_t key, bool term) {
    Node nd;
    nd.depth = depth;
    nd.born = born;
    nd.hist = h;
    nd.key = key;
    nd.term = term;
    const int na = m.num_actions();
    nd.Na.assign(na, 0);
    nd.Q.assign(na, 0.0);
    nd.ch.assign(na, {});
    tree.push_back(nd);
    return (int)tree.size() - 1;
  }

  int ucb(const Node& h, const std::vector<long long>& virt) const {
    const int na = (int)h.Q.size();
    long long n = h.N;
    for (int a = 0; a < na; ++a) n += virt[a];
    int best = 0;
    double bestv = -std::numeric_limits<double>::infinity();
    for (int a = 0; a < na; ++a) {
      const long long k = h.Na[a] + virt[a];
      double v;
      if (k == 0)
        v = std::numeric_limits<double>::infinity();
      else
        v = h.Q[a] + prm.c * std::sqrt(std::log((double)n) / (double)k);
      if (v > bestv) {
        bestv = v;
        best = a;
      }
    }
    return best;
  }

  PomcpResult plan(const std::vector<S>& root, const Hist& h0) {
    using Real = decltype(m.upper(root[0]));
    tree.clear();
    new_node(0, -1, h0, 0, false);
    const int n = (int)root.size();
    const double gamma = (double)m.gamma;
    long long sim_count = 0;
    int rollouts = 0;
    for (int r = 0; r < prm.rounds; ++r) {
      std::vector<Sim> sims(prm.batch);
      for (int i = 0; i < prm.batch; ++i) {
        sims[i].s = root[(size_t)(sim_count % n)];
        sim_count += 1;
      }
      // virtual visits of this round per (node, action)
      std::vector<std::vector<long long>> virt(tree.size());
      for (int d = 0; d < m.D; ++d) {
        bool any = false;
        for (int i = 0; i < prm.batch; ++i) {
          Sim& x = sims[i];
          if (!x.live) continue;
          any = true;
          const int hn = x.node;
          if ((int)virt.size() < (int)tree.size()) virt.resize(tree.size());
          if (virt[hn].empty()) virt[hn].assign(m.num_actions(), 0);
          const int a = ucb(tree[hn], virt[hn]);
          virt[hn][a] += 1;
          S next;
          uint64_t key;
          if (!m.terminal(x.s)) steps += 1;
          const Real rr = m.step(x.s, a, d, next, &key);
          x.s = next;
          x.nodes.push_back(hn);
          x.acts.push_back(a);
          x.rew.push_back((double)rr);
          int c = -1;
          for (const Child& k : tree[hn].ch[a])
            if (k.key == key) c = k.node;
          const bool term = (key >> 62) & 1u;
          bool fresh = false;
          if (c < 0) {
            Hist hc = tree[hn].hist;
            m.observe(hc, a, key);
            c = new_node(d + 1, r, hc, key, term);
            tree[hn].ch[a].push_back(Child{key, c});
            fresh = true;
          } else if (tree[c].born == r) {
            fresh = true;
          }
          x.node = c;
          if (term || d + 1 >= m.D) {
            x.live = false;  // value 0 below
          } else if (fresh) {
            x.live = false;
            x.rollout = true;
          }
        }
        if (!any) break;
      }
      // the default policy from every simulation that stopped at a new node
      for (int i = 0; i < prm.batch; ++i) {
        Sim& x = sims[i];
        if (!x.rollout) continue;
        const Node& leaf = tree[x.node];
        x.leaf = (double)rollout(m, x.s, leaf.hist, leaf.depth, &steps);
        rollouts += 1;
      }
      // backups in simulation order
      for (int i = 0; i < prm.batch; ++i) {
        Sim& x = sims[i];
        double G = x.leaf;
        for (int k = (int)x.nodes.size() - 1; k >= 0; --k) {
          G = x.rew[k] + gamma * G;
          Node& h = tree[x.nodes[k]];
          const int a = x.acts[k];
          h.N += 1;
          h.Na[a] += 1;
          h.Q[a] += (G - h.Q[a]) / (double)h.Na[a];
        }
      }
    }
    PomcpResult res;
    const Node& root_node = tree[0];
    int best = -1;
    for (int a = 0; a < (int)root_node.Q.size(); ++a)
      if (root_node.Na[a] > 0 && (best < 0 || root_node.Q[a] > root_node.Q[best])) best = a;
    res.action = best;
    res.value = best >= 0 ? root_node.Q[best] : 0.0;
    res.nodes = (int)tree.size();
    res.simulations = (int)sim_count;
    res.rollouts = rollouts;
    res.steps = steps;
    res.root_q = root_node.Q;
    res.root_na.assign(root_node.Na.begin(), root_node.Na.end());
    uint64_t sig = 0x243F6A8885A308D3ull;
    for (const Node& nd : tree) {
      sig = (sig ^ (uint64_t)nd.depth) * 0x100000001B3ull;
      sig = (sig ^ nd.key) * 0x100000001B3ull;
      sig = (sig ^ (uint64_t)nd.N) * 0x100000001B3ull;
    }
    res.signature = sig;
    return res;
  }
};

}  // namespace orc
