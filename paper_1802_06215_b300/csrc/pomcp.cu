// POMCP-style planning with the GPU as the rollout service (dsp_pomcp_plan,
// include/dsp.h): the single-scenario-per-path variant the paper names among
// its future directions (Sec. V), on the same models and scenario streams.
//
// The tree of histories lives on the host. A round carries `batch`
// simulations, each with one root scenario, down the tree level by level:
// the host chooses every live simulation's action by UCB1 (with virtual
// visits for the round's earlier choices), one dsp_step call steps them all on
// the GPU, and the host moves each to the child of its observation. The
// simulations that reach a node created in this round are rolled out by the
// GPU, one dsp_rollout call per start depth, and the host backs up their
// returns in simulation order.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "model.hpp"

namespace dsp {
namespace {

struct PChild {
  uint64_t key;
  int node;
};

struct PNode {
  int depth = 0;
  int born = -1;
  uint64_t key = 0;
  int8_t hist[32] = {};
  long long N = 0;
  std::vector<long long> Na;
  std::vector<double> Q;
  std::vector<std::vector<PChild>> ch;
};

struct PSim {
  int node = 0;
  bool live = true, rollout = false, term = false;
  std::vector<int> nodes, acts;
  std::vector<double> rew;
  double leaf = 0;
};

// Device buffers of one call: two state blocks of `batch` scenarios, the
// actions, keys and rewards of a level, and the rollouts' inputs and values.
struct PBuffers {
  uint32_t* cur = nullptr;
  uint32_t* next = nullptr;
  int32_t* acts = nullptr;
  uint64_t* keys = nullptr;
  float* rew = nullptr;
  uint32_t* roll = nullptr;
  int8_t* hist = nullptr;
  float* vals = nullptr;
  ~PBuffers() {
    cudaFree(cur);
    cudaFree(next);
    cudaFree(acts);
    cudaFree(keys);
    cudaFree(rew);
    cudaFree(roll);
    cudaFree(hist);
    cudaFree(vals);
  }
};

class Pomcp {
 public:
  Pomcp(dsp_model* m, const dsp_pomcp_params& p) : m_(m), p_(p) {
    na_ = m->host->num_actions;
    words_ = m->host->words;
    D_ = m->host->D;
    kind_ = m->host->kind;
    per_ = m->host->per_robot;
    gamma_ = (double)m->host->gamma;
  }

  dsp_status run(const uint32_t* root, int n, const int8_t* hist, dsp_pomcp_result* out, double* root_q,
                 int32_t* root_na);

 private:
  int new_node(int depth, int born, const int8_t* h, uint64_t key) {
    PNode nd;
    nd.depth = depth;
    nd.born = born;
    nd.key = key;
    std::memcpy(nd.hist, h, 32);
    nd.Na.assign(na_, 0);
    nd.Q.assign(na_, 0.0);
    nd.ch.assign(na_, {});
    tree_.push_back(std::move(nd));
    return (int)tree_.size() - 1;
  }

  // UCB1 with the round's virtual visits; an unvisited action first, lowest
  // index on ties.
  int choose(const PNode& h, const std::vector<long long>& virt) const {
    long long total = h.N;
    for (int a = 0; a < na_; ++a) total += virt[a];
    int best = 0;
    double bestv = -std::numeric_limits<double>::infinity();
    for (int a = 0; a < na_; ++a) {
      const long long k = h.Na[a] + virt[a];
      const double v = k == 0 ? std::numeric_limits<double>::infinity()
                              : h.Q[a] + p_.c * std::sqrt(std::log((double)total) / (double)k);
      if (v > bestv) {
        bestv = v;
        best = a;
      }
    }
    return best;
  }

  dsp_model* m_;
  dsp_pomcp_params p_;
  int na_, words_, D_, kind_, per_;
  double gamma_;
  std::vector<PNode> tree_;
};

dsp_status Pomcp::run(const uint32_t* root, int n, const int8_t* hist, dsp_pomcp_result* out, double* root_q,
                      int32_t* root_na) {
  const auto t0 = std::chrono::steady_clock::now();
  const int B = p_.batch;
  const size_t blk = (size_t)words_ * B;
  PBuffers d;
  cudaError_t e = cudaMalloc(&d.cur, blk * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.next, blk * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.acts, (size_t)B * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.keys, (size_t)B * 8);
  if (e == cudaSuccess) e = cudaMalloc(&d.rew, (size_t)B * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.roll, blk * 4);
  if (e == cudaSuccess) e = cudaMalloc(&d.hist, (size_t)B * 32);
  if (e == cudaSuccess) e = cudaMalloc(&d.vals, (size_t)B * 4);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: buffers");
  cudaStream_t st;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: stream");
  struct StreamGuard {
    cudaStream_t s;
    ~StreamGuard() { cudaStreamDestroy(s); }
  } guard{st};

  std::vector<uint32_t> hblk(blk), hnext(blk), hroll(blk);
  std::vector<int32_t> hacts(B);
  std::vector<uint64_t> hkeys(B);
  std::vector<float> hrew(B), hvals(B);
  std::vector<int8_t> hhist((size_t)B * 32);
  int8_t h0[32] = {};
  if (hist) std::memcpy(h0, hist, 32);
  tree_.clear();
  new_node(0, -1, h0, 0);
  uint64_t steps0 = 0, steps1 = 0, tree_steps = 0;
  uint32_t status = 0;
  dsp_status s = dsp_read_counters(m_, &steps0, &status);
  if (s != DSP_OK) return s;
  long long sims_done = 0;
  int rollouts = 0, rounds = 0;
  for (int r = 0; r < p_.rounds; ++r) {
    std::vector<PSim> sims(B);
    // each simulation's root scenario, column by column
    for (int i = 0; i < B; ++i) {
      const int k = (int)((sims_done + i) % n);
      for (int w = 0; w < words_; ++w) hblk[(size_t)w * B + i] = root[(size_t)w * n + k];
      sims[i].term = false;
    }
    sims_done += B;
    e = cudaMemcpyAsync(d.cur, hblk.data(), blk * 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: root scenarios");
    std::vector<std::vector<long long>> virt;
    for (int dd = 0; dd < D_; ++dd) {
      bool any = false;
      for (int i = 0; i < B; ++i) {
        PSim& x = sims[i];
        hacts[i] = 0;
        if (!x.live) continue;
        any = true;
        if (virt.size() < tree_.size()) virt.resize(tree_.size());
        if (virt[x.node].empty()) virt[x.node].assign(na_, 0);
        const int a = choose(tree_[x.node], virt[x.node]);
        virt[x.node][a] += 1;
        hacts[i] = a;
      }
      if (!any) break;
      // g for every simulation (the stopped ones are stepped too and ignored)
      e = cudaMemcpyAsync(d.acts, hacts.data(), (size_t)B * 4, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: actions");
      s = dsp_step(m_, d.cur, B, B, d.acts, dd, d.next, B, d.keys, d.rew, st);
      if (s != DSP_OK) return s;
      e = cudaMemcpyAsync(hkeys.data(), d.keys, (size_t)B * 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hrew.data(), d.rew, (size_t)B * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(hnext.data(), d.next, blk * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: level results");
      for (int i = 0; i < B; ++i) {
        PSim& x = sims[i];
        if (!x.live) continue;
        const int a = hacts[i];
        const uint64_t key = hkeys[i];
        if (!x.term) tree_steps += 1;
        const int h = x.node;
        x.nodes.push_back(h);
        x.acts.push_back(a);
        x.rew.push_back((double)hrew[i]);
        int c = -1;
        for (const PChild& k : tree_[h].ch[a])
          if (k.key == key) c = k.node;
        const bool term = (key >> 62) & 1u;
        bool fresh = false;
        if (c < 0) {
          int8_t hc[32];
          std::memcpy(hc, tree_[h].hist, 32);
          host_observe(kind_, per_, hc, a, key);
          c = new_node(dd + 1, r, hc, key);
          tree_[h].ch[a].push_back(PChild{key, c});
          fresh = true;
        } else if (tree_[c].born == r) {
          fresh = true;
        }
        x.node = c;
        x.term = term;
        if (term || dd + 1 >= D_) {
          x.live = false;
        } else if (fresh) {
          x.live = false;
          x.rollout = true;
          // keep its scenario for the rollout
          for (int w = 0; w < words_; ++w) hroll[(size_t)w * B + i] = hnext[(size_t)w * B + i];
        }
      }
      std::swap(d.cur, d.next);
    }
    // rollouts, one call per start depth
    std::vector<int> by_depth;
    for (int dd = 1; dd < D_; ++dd) {
      std::vector<int> idx;
      for (int i = 0; i < B; ++i)
        if (sims[i].rollout && tree_[sims[i].node].depth == dd) idx.push_back(i);
      if (idx.empty()) continue;
      const int cnt = (int)idx.size();
      for (int j = 0; j < cnt; ++j) {
        const int i = idx[j];
        for (int w = 0; w < words_; ++w) hblk[(size_t)w * cnt + j] = hroll[(size_t)w * B + i];
        std::memcpy(&hhist[(size_t)32 * j], tree_[sims[i].node].hist, 32);
      }
      e = cudaMemcpyAsync(d.roll, hblk.data(), (size_t)words_ * cnt * 4, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(d.hist, hhist.data(), (size_t)cnt * 32, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: rollout inputs");
      s = dsp_rollout(m_, d.roll, cnt, cnt, d.hist, dd, d.vals, st);
      if (s != DSP_OK) return s;
      e = cudaMemcpyAsync(hvals.data(), d.vals, (size_t)cnt * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_pomcp_plan: rollout values");
      for (int j = 0; j < cnt; ++j) sims[idx[j]].leaf = (double)hvals[j];
      rollouts += cnt;
    }
    // backups in simulation order
    for (int i = 0; i < B; ++i) {
      PSim& x = sims[i];
      double G = x.leaf;
      for (int k = (int)x.nodes.size() - 1; k >= 0; --k) {
        G = x.rew[k] + gamma_ * G;
        PNode& h = tree_[x.nodes[k]];
        const int a = x.acts[k];
        h.N += 1;
        h.Na[a] += 1;
        h.Q[a] += (G - h.Q[a]) / (double)h.Na[a];
      }
    }
    rounds += 1;
    if (p_.time_limit_s > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() >= p_.time_limit_s)
      break;
  }
  s = dsp_read_counters(m_, &steps1, &status);
  if (s != DSP_OK) return s;
  if (status != 0) return fail(DSP_E_DEVICE, "dsp_pomcp_plan: device status word %u", status);
  const PNode& rt = tree_[0];
  int best = -1;
  for (int a = 0; a < na_; ++a)
    if (rt.Na[a] > 0 && (best < 0 || rt.Q[a] > rt.Q[best])) best = a;
  out->action = best;
  out->value = best >= 0 ? rt.Q[best] : 0.0;
  out->nodes = (int32_t)tree_.size();
  out->simulations = (int32_t)sims_done;
  out->rollouts = rollouts;
  out->rounds = rounds;
  out->scenario_steps = tree_steps + (steps1 - steps0);
  uint64_t sig = 0x243F6A8885A308D3ull;
  for (const PNode& nd : tree_) {
    sig = (sig ^ (uint64_t)nd.depth) * 0x100000001B3ull;
    sig = (sig ^ nd.key) * 0x100000001B3ull;
    sig = (sig ^ (uint64_t)nd.N) * 0x100000001B3ull;
  }
  out->signature = sig;
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int a = 0; a < na_; ++a) {
    if (root_q) root_q[a] = rt.Q[a];
    if (root_na) root_na[a] = (int32_t)rt.Na[a];
  }
  return DSP_OK;
}

}  // namespace
}  // namespace dsp

using namespace dsp;

extern "C" dsp_status dsp_pomcp_plan(dsp_model* m, const uint32_t* root_states, int32_t n, const int8_t* hist,
                                     const dsp_pomcp_params* params, dsp_pomcp_result* result, double* root_q,
                                     int32_t* root_na) {
  if (!m || !root_states || !params || !result) return fail(DSP_E_INVALID, "dsp_pomcp_plan: NULL argument");
  if (n < 1) return fail(DSP_E_INVALID, "dsp_pomcp_plan: n=%d", n);
  if (params->rounds < 1 || params->batch < 1 || params->batch > 65536)
    return fail(DSP_E_INVALID, "dsp_pomcp_plan: rounds %d, batch %d", params->rounds, params->batch);
  if (!(params->c >= 0.0)) return fail(DSP_E_INVALID, "dsp_pomcp_plan: exploration constant");
  if (m->policy_on) return fail(DSP_E_UNSUPPORTED, "dsp_pomcp_plan: rolls out the heuristic policy");
  Pomcp pc(m, *params);
  return pc.run(root_states, n, hist, result, root_q, root_na);
}
