// Host tree search of HyP-DESPOT (Sec. III-C) around the GPU leaf expansion.
//
// T CPU threads search one DESPOT tree (Sec. III-A): each trial descends from
// the root choosing actions by scenario-based PO-UCT (Eq. UCT) and
// observation branches by weighted excess uncertainty minus virtual loss
// (Eq. select_lb, Eq. augmented_WEU), expands the leaf it reaches on the GPU
// (dsp_expand_leaves: Eq. expand, newnodes, ub, lb), creates the children on
// the host and backs the bounds up to the root (Eq. backup). Node values are
// kept weighted by |Phi_b|/K; a node's scenario list lives on the device as
// the leaf states its expansion wrote, and its children refer to it through
// the grouped positions (perm) the kernel wrote, so scenario data never comes
// back to the host.
//
// Two schedules:
//  - deterministic rounds: the T trials of a round select in thread order,
//    their leaves are expanded as one batch, and they back up in thread
//    order, so the tree is reproducible bit for bit;
//  - free running: T std::threads, each with its own CUDA stream
//    (Sec. III-D, node-level parallelism), expanding concurrently. They select
//    and back up either on per-node atomics, without a lock (the default: a
//    leaf is claimed by compare-and-swap, visit and virtual-loss counts are
//    atomic increments, bounds are atomic stores recomputed from the children,
//    children are published with release ordering), or under one tree lock.
//    Without the lock two backups through a node may interleave and leave it
//    a bound computed from an older child value: still a bound (the older
//    value is looser), and the next backup through the node refreshes it; a
//    bottom-up pass over the tree after the threads join makes every node
//    exact again.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "model.hpp"

namespace dsp {
namespace {

uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Device memory for one plan on one GPU: bump allocation from 256 MB chunks.
class Arena {
 public:
  explicit Arena(int device) : device_(device) {}
  ~Arena() {
    if (!chunks_.empty()) cudaSetDevice(device_);
    for (void* p : chunks_) cudaFree(p);
  }
  cudaError_t alloc(size_t bytes, void** out) {
    std::lock_guard<std::mutex> lock(mu_);
    bytes = (bytes + 255) & ~(size_t)255;
    if (chunks_.empty() || off_ + bytes > cap_) {
      size_t cap = std::max(bytes, (size_t)256 << 20);
      void* p = nullptr;
      cudaError_t e = cudaSetDevice(device_);
      if (e == cudaSuccess) e = cudaMalloc(&p, cap);
      if (e != cudaSuccess) return e;
      chunks_.push_back(p);
      cap_ = cap;
      off_ = 0;
    }
    *out = (char*)chunks_.back() + off_;
    off_ += bytes;
    return cudaSuccess;
  }

 private:
  int device_;
  std::mutex mu_;
  std::vector<void*> chunks_;
  size_t cap_ = 0, off_ = 0;
};

template <class T>
T ld(const std::atomic<T>& x) {
  return x.load(std::memory_order_relaxed);
}
template <class T>
void wr(std::atomic<T>& x, T v) {
  x.store(v, std::memory_order_relaxed);
}

struct Node;
// An action's children: consecutive nodes of their expansion's node array.
struct Children {
  Node* first = nullptr;
  int n = 0;
  struct It {
    Node* p;
    Node* operator*() const { return p; }
    It& operator++();
    bool operator!=(const It& o) const { return p != o.p; }
  };
  It begin() const;
  It end() const;
};
struct QBranch {
  double R = 0;                 // set before the node is published
  std::atomic<double> U{0.0}, L{0.0};
  Children ch;                  // set before the node is published, then read-only
};
struct Node {
  int depth = 0, n = 0;
  double W = 1;
  Node* parent = nullptr;
  int pa = -1;                     // action into this node
  const uint16_t* d_idx = nullptr; // positions in the parent's states (device)
  uint32_t* d_states = nullptr;    // own states once expanded (root: the given ones)
  int dev = 0;                     // model (GPU) that holds d_states and d_perm
  uint16_t* d_perm = nullptr;      // grouped positions written by the expansion
  int8_t hist[32] = {};
  uint64_t key = 0;
  bool term = false;
  std::atomic<bool> expanded{false};  // children published (release / acquire)
  std::atomic<bool> claimed{false};   // a thread is expanding this leaf
  std::atomic<double> U{0.0}, L{0.0};
  std::atomic<long long> N{0};
  std::unique_ptr<std::atomic<long long>[]> Na;
  std::atomic<int> vl{0};
  std::unique_ptr<QBranch[]> q;
  int nq = 0;
};
inline Children::It& Children::It::operator++() {
  ++p;
  return *this;
}
inline Children::It Children::begin() const { return It{first}; }
inline Children::It Children::end() const { return It{first + n}; }

// Pinned host buffer of one search thread, grown on demand.
struct Pinned {
  char* p = nullptr;
  size_t cap = 0;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
  cudaError_t reserve(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = nullptr;
    cap = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMallocHost((void**)&p, want);
    if (e == cudaSuccess) cap = want;
    return e;
  }
};

// Small per-job results, contiguous so one copy brings them to the host.
struct JobOut {
  int na = 0, cap = 0;
  size_t bytes = 0;
  size_t o_cnt = 0, o_off = 0, o_key = 0, o_rew = 0, o_u = 0, o_l = 0;
  void layout(int na_, int cap_) {
    na = na_;
    cap = cap_;
    size_t o = 0;
    auto take = [&](size_t b) {
      size_t r = o;
      o += (b + 15) & ~(size_t)15;
      return r;
    };
    o_cnt = take(4 * (size_t)na);
    o_off = take(4 * (size_t)na * (cap + 1));
    o_key = take(8 * (size_t)na * cap);
    o_rew = take(8 * (size_t)na * cap);
    o_u = take(8 * (size_t)na * cap);
    o_l = take(8 * (size_t)na * cap);
    bytes = o;
  }
};

// One CUDA stream per model (GPU) for one search thread.
struct Streams {
  std::vector<cudaStream_t> st;
  std::vector<int> dev;
  ~Streams() {
    for (size_t g = 0; g < st.size(); ++g) {
      cudaSetDevice(dev[g]);
      cudaStreamDestroy(st[g]);
    }
  }
  cudaError_t make(const std::vector<dsp_model*>& models) {
    for (dsp_model* m : models) {
      cudaStream_t x = nullptr;
      cudaError_t e = cudaSetDevice(m->device);
      if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
      if (e != cudaSuccess) return e;
      st.push_back(x);
      dev.push_back(m->device);
    }
    return cudaSetDevice(models[0]->device);
  }
};

class Search {
 public:
  // models: one per GPU, built from one description; leaf expansions are
  // routed over them (node-level parallelism, Sec. III-D). models[0] holds
  // the root's states.
  Search(const std::vector<dsp_model*>& models, const dsp_search_params& p)
      : models_(models), m_(models[0]), p_(p) {
    na_ = m_->host->num_actions;
    K_ = (double)m_->host->K;
    gamma_ = (double)m_->host->gamma;
    D_ = m_->host->D;
    words_ = m_->host->words;
    kind_ = m_->host->kind;
    per_ = m_->host->per_robot;
    for (dsp_model* m : models_) arenas_.emplace_back(new Arena(m->device));
    ident_.assign(models_.size(), nullptr);
  }

  dsp_status run(const uint32_t* root_host, int n, const int8_t* hist, dsp_search_result* out, int32_t* visits);
  dsp_status export_nodes(int min_scen, int cap, dsp_plan_node* nodes, uint32_t* states, int32_t* count);

 private:
  struct Trial {
    std::vector<Node*> path;
    std::vector<int> acts;
    Node* leaf = nullptr;
    long long epoch = 0;  // leaves published when the trial was selected
  };

  // count new nodes, one array allocated outside the pool lock, listed in
  // creation order under one acquisition of it
  Node* new_nodes(int count) {
    if (count <= 0) return nullptr;
    std::unique_ptr<Node[]> blk(new Node[count]);
    Node* p = blk.get();
    std::lock_guard<std::mutex> lock(pool_mu_);
    blocks_.push_back({std::move(blk), count});
    n_nodes_ += count;
    return p;
  }
  // every node in creation order (after the search threads have joined)
  template <class F>
  void for_each_node(F&& f) const {
    for (const NodeBlock& b : blocks_)
      for (int k = 0; k < b.n; ++k) f(b.p.get() + k);
  }
  Node* new_node() { return new_nodes(1); }

  void observe(int8_t* h, int a, uint64_t key) const { host_observe(kind_, per_, h, a, key); }

  void refresh(Node* b) {
    double bu = -std::numeric_limits<double>::infinity(), bl = bu;
    for (int a = 0; a < b->nq; ++a) {
      bu = std::max(bu, ld(b->q[a].U));
      bl = std::max(bl, ld(b->q[a].L));
    }
    wr(b->U, bu);
    wr(b->L, bl);
  }
  void refresh_action(Node* b, int a) {
    QBranch& q = b->q[a];
    double su = 0, sl = 0;
    for (Node* c : q.ch) {
      su += ld(c->U);
      sl += ld(c->L);
    }
    wr(q.U, q.R + gamma_ * su);
    wr(q.L, q.R + gamma_ * sl);
  }

  int choose_action(Node* b) const {
    int best = 0;
    double bestv = -std::numeric_limits<double>::infinity();
    const long long N = ld(b->N);
    for (int a = 0; a < b->nq; ++a) {
      double v = ld(b->q[a].U) / b->W;
      if (p_.c_a != 0) {
        const long long na = ld(b->Na[a]);
        if (na == 0)
          v = std::numeric_limits<double>::infinity();
        else
          v += p_.c_a * std::sqrt(std::log((double)b->n * (double)N) / ((double)b->n * (double)na));
      }
      if (v > bestv) {
        bestv = v;
        best = a;
      }
    }
    return best;
  }

  // Forward search of one trial from the root (under the tree lock, or on
  // the nodes' atomics). A leaf is taken by compare-and-swap on its claim
  // flag; in_flight_ counts it before the claim can be seen.
  Trial select() {
    Trial t;
    t.epoch = published_.load();
    Node* b = root_;
    t.path.push_back(b);
    while (true) {
      if (!b->expanded.load(std::memory_order_acquire)) {
        if (b->depth < D_ && !b->term && !ld(b->claimed)) {
          in_flight_.fetch_add(1);
          bool free = false;
          if (b->claimed.compare_exchange_strong(free, true))
            t.leaf = b;
          else
            in_flight_.fetch_sub(1);
        }
        return t;
      }
      b->N.fetch_add(1, std::memory_order_relaxed);
      int a = choose_action(b);
      b->Na[a].fetch_add(1, std::memory_order_relaxed);
      double eps0 = ld(root_->U) - ld(root_->L);
      Node* best = nullptr;
      double beste = -std::numeric_limits<double>::infinity();
      for (Node* c : b->q[a].ch) {
        double e = (ld(c->U) - ld(c->L)) - c->W * p_.xi * eps0 - p_.c_o * eps0 * (double)ld(c->vl);
        if (e > beste) {
          beste = e;
          best = c;
        }
      }
      t.acts.push_back(a);
      if (best == nullptr || !(beste > 0)) return t;
      best->vl.fetch_add(1, std::memory_order_relaxed);
      t.path.push_back(best);
      b = best;
    }
  }

  // Whether a descent without any virtual loss would reach a leaf worth
  // expanding (read-only). With several threads the stop rule asks it, so
  // that the virtual loss of trials still selecting on other threads, which
  // can make every branch look not worth it for a moment, never ends the
  // search. (One thread has no such trials and keeps the plain rule, the
  // rounds search's.)
  bool leaf_left() const {
    Node* b = root_;
    while (true) {
      if (!b->expanded.load(std::memory_order_acquire)) return b->depth < D_ && !b->term && !ld(b->claimed);
      const int a = choose_action(b);
      const double eps0 = ld(root_->U) - ld(root_->L);
      Node* best = nullptr;
      double beste = -std::numeric_limits<double>::infinity();
      for (Node* c : b->q[a].ch) {
        const double e = (ld(c->U) - ld(c->L)) - c->W * p_.xi * eps0;
        if (e > beste) {
          beste = e;
          best = c;
        }
      }
      if (best == nullptr || !(beste > 0)) return false;
      b = best;
    }
  }

  void backup(Trial& t) {
    for (int i = (int)t.path.size() - 1; i >= 0; --i) {
      Node* b = t.path[i];
      if (i < (int)t.acts.size() && b->expanded.load(std::memory_order_acquire)) {
        refresh_action(b, t.acts[i]);
        refresh(b);
      }
      if (i > 0) b->vl.fetch_sub(1, std::memory_order_relaxed);
    }
  }

  // Every expanded node's bounds recomputed from its children, children first
  // (a node is created after its parent): after lock-free threads, whose
  // interleaved backups may have left a node an older (looser) bound.
  void settle() {
    for (auto it = blocks_.rbegin(); it != blocks_.rend(); ++it)
      for (int k = it->n - 1; k >= 0; --k) {
        Node* b = it->p.get() + k;
        if (!b->expanded.load(std::memory_order_acquire)) continue;
        for (int a = 0; a < b->nq; ++a) refresh_action(b, a);
        refresh(b);
      }
  }

  // Device buffers and the job descriptor of one leaf on model g (caller
  // prepares `jo`, with model g's GPU current). With `copy` the states its
  // scenarios come from (the parent's, or the root's given ones) and its
  // scenario positions are first copied from the GPU that holds them, on `st`.
  dsp_status prepare(Node* b, int g, bool copy, dsp_leaf_job& J, const JobOut& jo, char* dsmall, cudaStream_t st) {
    int n = b->n;
    std::memset(&J, 0, sizeof(J));
    Arena& ar = *arenas_[g];
    const Node* src = b->parent != nullptr ? b->parent : b;
    const uint32_t* pstates = src->d_states;
    const uint16_t* idx = b->parent != nullptr ? b->d_idx : ident_[g];
    void* p = nullptr;
    cudaError_t e = cudaSuccess;
    if (copy) {
      const size_t sb = (size_t)words_ * src->n * 4;
      e = ar.alloc(sb, &p);
      if (e == cudaSuccess)
        e = cudaMemcpyPeerAsync(p, models_[g]->device, pstates, models_[src->dev]->device, sb, st);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: parent states to the leaf's GPU");
      pstates = (const uint32_t*)p;
      if (b->parent != nullptr) {
        e = ar.alloc((size_t)n * 2, &p);
        if (e == cudaSuccess)
          e = cudaMemcpyPeerAsync(p, models_[g]->device, idx, models_[src->dev]->device, (size_t)n * 2, st);
        if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: scenario positions to the leaf's GPU");
        idx = (const uint16_t*)p;
      }
    }
    J.parent = pstates;
    J.parent_cap = src->n;
    J.idx = idx;
    J.last_action = b->parent != nullptr ? b->pa : -1;
    J.n_scen = n;
    J.depth = b->depth;
    std::memcpy(J.hist, b->hist, 32);
    J.first_action = 0;
    J.n_actions = na_;
    J.child_cap = jo.cap;
    e = ar.alloc((size_t)words_ * n * 4, &p);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: node states");
    J.leaf_states = (uint32_t*)p;
    e = ar.alloc((size_t)na_ * n * 2, &p);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: grouped positions");
    J.perm = (uint16_t*)p;
    J.child_count = (int32_t*)(dsmall + jo.o_cnt);
    J.child_off = (int32_t*)(dsmall + jo.o_off);
    J.child_key = (uint64_t*)(dsmall + jo.o_key);
    J.rew_sum = (int64_t*)(dsmall + jo.o_rew);
    J.u_sum = (int64_t*)(dsmall + jo.o_u);
    J.l_sum = (int64_t*)(dsmall + jo.o_l);
    return DSP_OK;
  }

  // Children of an expanded leaf from its copied results. The leaf is claimed
  // by the calling thread, and other threads stop at an unexpanded leaf, so
  // this runs without the tree lock; publish() then marks the leaf expanded.
  // The nodes of one expansion come from the pool in one batch.
  void create_children(Node* b, int dev, const dsp_leaf_job& J, const JobOut& jo, const char* hsmall) {
    const int32_t* cnt = (const int32_t*)(hsmall + jo.o_cnt);
    const int32_t* off = (const int32_t*)(hsmall + jo.o_off);
    const uint64_t* key = (const uint64_t*)(hsmall + jo.o_key);
    const int64_t* rew = (const int64_t*)(hsmall + jo.o_rew);
    const int64_t* us = (const int64_t*)(hsmall + jo.o_u);
    const int64_t* ls = (const int64_t*)(hsmall + jo.o_l);
    b->d_states = J.leaf_states;
    b->d_perm = J.perm;
    b->dev = dev;
    b->q.reset(new QBranch[na_]);
    b->nq = na_;
    b->Na.reset(new std::atomic<long long>[na_]);
    for (int a = 0; a < na_; ++a) wr(b->Na[a], 0LL);
    const int cap = jo.cap, n = b->n;
    int total = 0;
    for (int a = 0; a < na_; ++a) total += std::min(cnt[a], cap);
    Node* made = new_nodes(total);
    int next = 0;
    for (int a = 0; a < na_; ++a) {
      QBranch& q = b->q[a];
      int nc = std::min(cnt[a], cap);
      int64_t rsum = 0;
      for (int c = 0; c < nc; ++c) rsum += rew[(size_t)a * cap + c];
      q.R = ((double)rsum / 4294967296.0) / K_;
      double su = 0, sl = 0;
      q.ch.first = made + next;
      q.ch.n = nc;
      for (int c = 0; c < nc; ++c) {
        Node* ch = made + next++;
        int o0 = off[(size_t)a * (cap + 1) + c], o1 = off[(size_t)a * (cap + 1) + c + 1];
        ch->depth = b->depth + 1;
        ch->n = o1 - o0;
        ch->W = (double)ch->n / K_;
        ch->parent = b;
        ch->pa = a;
        ch->d_idx = J.perm + (size_t)a * n + o0;
        ch->key = key[(size_t)a * cap + c];
        ch->term = (ch->key >> 62) & 1u;
        std::memcpy(ch->hist, b->hist, 32);
        observe(ch->hist, a, ch->key);
        const double cu = ((double)us[(size_t)a * cap + c] / 4294967296.0) / K_;
        const double cl = ((double)ls[(size_t)a * cap + c] / 4294967296.0) / K_;
        wr(ch->U, cu);
        wr(ch->L, cl);
        su += cu;
        sl += cl;
      }
      wr(q.U, q.R + gamma_ * su);
      wr(q.L, q.R + gamma_ * sl);
    }
  }

  // Makes a leaf whose children exist visible to the search (under the tree
  // lock when the threads use it): bounds first, then the flag with release
  // ordering, so that a thread that sees the flag sees the children.
  void publish(Node* b) {
    refresh(b);
    b->expanded.store(true, std::memory_order_release);
    published_.fetch_add(1);
  }

  // Expands leaves as one batch on `st` and creates their children in order.
  // The GPU part of a batch (job tables, launch or queue, result copy into
  // `pinned`) and the host part (children, publishing), separable so that a
  // dispatcher can let the next batch launch while it makes this one's nodes.
  struct BatchOut {
    std::vector<dsp_leaf_job> jobs;
    std::vector<JobOut> jo;
    std::vector<size_t> base;
    std::vector<int32_t> dev;  // the model each leaf was expanded on
    const char* host = nullptr;
  };
  dsp_status expand_batch(const std::vector<Node*>& leaves, Streams& st, Pinned& pinned) {
    BatchOut bo;
    dsp_status s = expand_gpu(leaves, st, pinned, bo);
    if (s != DSP_OK) return s;
    finish_batch(leaves, bo);
    return DSP_OK;
  }
  void finish_batch(const std::vector<Node*>& leaves, const BatchOut& bo) {
    const int L = (int)leaves.size();
    for (int k = 0; k < L; ++k)
      create_children(leaves[k], bo.dev[k], bo.jobs[k], bo.jo[k], bo.host + bo.base[k]);
    {
      std::unique_lock<std::mutex> lock(tree_mu_, std::defer_lock);
      if (p_.deterministic == 0 && p_.tree_lock != 0) lock.lock();
      for (int k = 0; k < L; ++k) publish(leaves[k]);
    }
    expansions_ += L;
  }
  // The GPU part of a batch: the leaves are routed over the models (the
  // expansion with global index e goes to model e mod G, dsp_route_leaves);
  // each model expands its leaves in one dsp_expand_leaves call on its own
  // stream (or through the device queue), and every model's small results
  // come back into one pinned host buffer.
  dsp_status expand_gpu(const std::vector<Node*>& leaves, Streams& st, Pinned& pinned, BatchOut& bo) {
    const int L = (int)leaves.size(), G = (int)models_.size();
    std::vector<dsp_leaf_job>& jobs = bo.jobs;
    std::vector<JobOut>& jo = bo.jo;
    std::vector<size_t>& base = bo.base;
    jobs.resize(L);
    jo.resize(L);
    base.resize(L);
    bo.dev.resize(L);
    std::vector<int32_t> pdev(L), copy(L);
    for (int k = 0; k < L; ++k) pdev[k] = leaves[k]->parent != nullptr ? leaves[k]->parent->dev : leaves[k]->dev;
    const long long e0 = routed_.fetch_add(L);
    dsp_status s = dsp_route_leaves(L, e0, G, pdev.data(), bo.dev.data(), copy.data());
    if (s != DSP_OK) return s;
    std::vector<size_t> dev_total(G, 0), local(L), host_off(G, 0);
    for (int k = 0; k < L; ++k) {
      jo[k].layout(na_, dsp_max_children(m_, leaves[k]->n));
      local[k] = dev_total[bo.dev[k]];
      dev_total[bo.dev[k]] += jo[k].bytes;
    }
    size_t total = 0;
    for (int g = 0; g < G; ++g) {
      host_off[g] = total;
      total += dev_total[g];
    }
    std::vector<char*> dsmall(G, nullptr);
    cudaError_t e = cudaSuccess;
    for (int g = 0; g < G; ++g) {
      if (dev_total[g] == 0) continue;
      void* p = nullptr;
      e = arenas_[g]->alloc(dev_total[g], &p);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: results");
      dsmall[g] = (char*)p;
    }
    for (int k = 0; k < L; ++k) {
      const int g = bo.dev[k];
      base[k] = host_off[g] + local[k];
      e = cudaSetDevice(models_[g]->device);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: device");
      s = prepare(leaves[k], g, copy[k] != 0, jobs[k], jo[k], dsmall[g] + local[k], st.st[g]);
      if (s != DSP_OK) return s;
    }
    if (queue_ != nullptr) {
      // through the device job queue (one model): publish, wait (bounded), then copy
      std::vector<uint64_t> tickets(L);
      for (int k = 0; k < L && s == DSP_OK; ++k) s = dsp_queue_submit(queue_, &jobs[k], 10000000000ull, &tickets[k]);
      for (int k = 0; k < L && s == DSP_OK; ++k) s = dsp_queue_wait(queue_, tickets[k], 60000000000ull);
    } else if (G == 1) {
      s = dsp_expand_leaves(m_, jobs.data(), L, st.st[0]);
    } else {
      std::vector<dsp_leaf_job> mine;
      for (int g = 0; g < G && s == DSP_OK; ++g) {
        mine.clear();
        for (int k = 0; k < L; ++k)
          if (bo.dev[k] == g) mine.push_back(jobs[k]);
        if (mine.empty()) continue;
        e = cudaSetDevice(models_[g]->device);
        if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: device");
        s = dsp_expand_leaves(models_[g], mine.data(), (int)mine.size(), st.st[g]);
      }
    }
    if (s != DSP_OK) return s;
    e = pinned.reserve(total);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: pinned results");
    char* host = pinned.p;
    for (int g = 0; g < G && e == cudaSuccess; ++g)
      if (dev_total[g] > 0) e = cudaMemcpyAsync(host + host_off[g], dsmall[g], dev_total[g], cudaMemcpyDeviceToHost,
                                                st.st[g]);
    for (int g = 0; g < G && e == cudaSuccess; ++g)
      if (dev_total[g] > 0) e = cudaStreamSynchronize(st.st[g]);
    if (e == cudaSuccess && G > 1) e = cudaSetDevice(m_->device);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: results copy");
    bo.host = host;
    return DSP_OK;
  }

  dsp_status run_rounds();
  dsp_status run_threads();

  std::vector<dsp_model*> models_;
  dsp_model* m_;
  dsp_search_params p_;
  int na_, D_, words_, kind_, per_;
  double K_, gamma_;
  std::vector<std::unique_ptr<Arena>> arenas_;  // per model: the tree's device memory on its GPU
  struct NodeBlock {
    std::unique_ptr<Node[]> p;
    int n;
  };
  std::vector<NodeBlock> blocks_;  // every node, one array per expansion, in creation order
  long long n_nodes_ = 0;
  Node* root_ = nullptr;
  std::vector<uint16_t*> ident_;                // per model: positions 0..n-1 of the root's scenarios
  std::atomic<long long> routed_{0};            // expansions routed so far
  std::mutex tree_mu_;   // free running with tree_lock: selection and backup
  std::mutex pool_mu_;   // the node pool (children are made outside the tree lock)
  std::atomic<long long> published_{0};  // leaves made visible
  std::atomic<int> in_flight_{0};        // leaves claimed and not yet backed up
  std::atomic<long long> started_{0};    // expansions begun (free running)
  std::atomic<int> expansions_{0};
  dsp_queue* queue_ = nullptr;  // free running with use_queue: the shared device job queue
  int rounds_ = 0;
};

dsp_status Search::run_rounds() {
  Streams st;
  cudaError_t e = st.make(models_);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: stream");
  Pinned staging;
  dsp_status s = DSP_OK;
  for (int r = 0; r < p_.rounds; ++r) {
    std::vector<Trial> trials;
    for (int t = 0; t < p_.threads; ++t) trials.push_back(select());
    std::vector<Node*> leaves;
    for (auto& t : trials)
      if (t.leaf) leaves.push_back(t.leaf);
    if (!leaves.empty()) {
      s = expand_batch(leaves, st, staging);
      if (s != DSP_OK) break;
    }
    for (auto& t : trials) backup(t);
    for (Node* l : leaves) wr(l->claimed, false);
    in_flight_.fetch_sub((int)leaves.size());
    rounds_ += 1;
    if (root_->expanded.load() && ld(root_->U) - ld(root_->L) <= p_.target_gap) break;
    if (leaves.empty()) break;
  }
  return s;
}

dsp_status Search::run_threads() {
  auto t0 = std::chrono::steady_clock::now();
  std::atomic<bool> stop{false};
  std::vector<dsp_status> status(p_.threads, DSP_OK);
  const long long budget = (long long)p_.threads * p_.rounds;
  const bool locked = p_.tree_lock != 0;
  auto gap_reached = [&]() {
    return root_->expanded.load(std::memory_order_acquire) && ld(root_->U) - ld(root_->L) <= p_.target_gap;
  };
  // Batched launches (batch > 1, no queue): a thread that claims a leaf hands
  // its trial to the pending list and tries to become the dispatcher; the
  // dispatcher expands everything pending (up to `batch` leaves per launch) in
  // one dsp_expand_leaves call on its own stream, creates and publishes the
  // children, and backs the trials up, while the other threads go on
  // selecting. After releasing the role it looks again, so no trial is left
  // behind by a push that met a busy dispatcher.
  const bool batched = p_.batch > 1 && queue_ == nullptr;
  std::mutex pend_mu, disp_mu;
  std::vector<Trial> pending;
  auto dispatch = [&](Streams& stream, Pinned& staging, int tid) {
    while (true) {
      if (!disp_mu.try_lock()) return;  // the dispatcher will look again after it lets go
      std::vector<Trial> take;
      {
        std::lock_guard<std::mutex> lock(pend_mu);
        const size_t k = std::min(pending.size(), (size_t)p_.batch);
        for (size_t i = 0; i < k; ++i) take.push_back(std::move(pending[i]));
        pending.erase(pending.begin(), pending.begin() + (long)k);
      }
      if (take.empty()) {
        disp_mu.unlock();
        std::lock_guard<std::mutex> lock(pend_mu);
        if (pending.empty()) return;
        continue;
      }
      std::vector<Node*> leaves;
      for (auto& x : take) leaves.push_back(x.leaf);
      BatchOut bo;
      dsp_status s = expand_gpu(leaves, stream, staging, bo);
      disp_mu.unlock();  // the next batch may launch while this one's nodes are made
      if (s == DSP_OK) {
        finish_batch(leaves, bo);
      } else {
        status[tid] = s;
        stop = true;
      }
      {
        std::unique_lock<std::mutex> lock(tree_mu_, std::defer_lock);
        if (locked) lock.lock();
        for (auto& x : take) {
          backup(x);
          wr(x.leaf->claimed, false);
        }
      }
      in_flight_.fetch_sub((int)take.size());  // after the publishes and the backups
      if (gap_reached()) stop = true;
    }
  };
  auto worker = [&](int tid) {
    cudaSetDevice(m_->device);
    Streams stream;
    if (stream.make(models_) != cudaSuccess) {
      status[tid] = fail(DSP_E_CUDA, "dsp_plan: stream");
      stop = true;
      return;
    }
    Pinned staging;
    while (!stop.load()) {
      if (batched) {
        size_t np;
        {
          std::lock_guard<std::mutex> lock(pend_mu);
          np = pending.size();
        }
        if (np >= (size_t)p_.batch) {  // a full batch waits: expand it rather than select further ahead
          dispatch(stream, staging, tid);
          std::this_thread::yield();
          continue;
        }
      }
      Trial t;
      {
        std::unique_lock<std::mutex> lock(tree_mu_, std::defer_lock);
        if (locked) lock.lock();
        if (stop.load()) break;
        if (started_.load() >= budget) {  // every budgeted expansion is taken
          stop = true;
          break;
        }
        t = select();
        if (t.leaf && started_.fetch_add(1) >= budget) {  // another thread took the last one
          backup(t);
          wr(t.leaf->claimed, false);
          in_flight_.fetch_sub(1);
          stop = true;
          break;
        }
      }
      if (t.leaf && batched) {
        {
          std::lock_guard<std::mutex> lock(pend_mu);
          pending.push_back(std::move(t));
        }
        dispatch(stream, staging, tid);
      } else if (t.leaf) {
        dsp_status s = expand_batch({t.leaf}, stream, staging);
        std::unique_lock<std::mutex> lock(tree_mu_, std::defer_lock);
        if (locked) lock.lock();
        if (s != DSP_OK) {
          status[tid] = s;
          stop = true;
        }
        backup(t);
        wr(t.leaf->claimed, false);
        in_flight_.fetch_sub(1);  // after the publish and the backup
        if (gap_reached()) stop = true;
      } else {
        if (batched) dispatch(stream, staging, tid);
        std::unique_lock<std::mutex> lock(tree_mu_, std::defer_lock);
        if (locked) lock.lock();
        backup(t);
        // nothing left worth expanding: no expansion in flight, none
        // published since this trial looked (else the tree changed: retry),
        // and no leaf reachable without the other threads' virtual loss
        if (in_flight_.load() == 0 && t.epoch == published_.load() && (p_.threads == 1 || !leaf_left()))
          stop = true;
        if (gap_reached()) stop = true;
      }
      if (p_.time_limit_s > 0) {
        double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el >= p_.time_limit_s) stop = true;
      }
      if (!t.leaf && !stop.load()) std::this_thread::yield();
    }
    if (batched) dispatch(stream, staging, tid);  // what is still pending
  };
  std::vector<std::thread> th;
  for (int i = 0; i < p_.threads; ++i) th.emplace_back(worker, i);
  for (auto& x : th) x.join();
  if (!locked) settle();
  for (auto s : status)
    if (s != DSP_OK) return s;
  return DSP_OK;
}

dsp_status Search::run(const uint32_t* root_host, int n, const int8_t* hist, dsp_search_result* out,
                       int32_t* visits) {
  auto t0 = std::chrono::steady_clock::now();
  root_ = new_node();
  root_->n = n;
  root_->W = (double)n / K_;
  if (hist) std::memcpy(root_->hist, hist, 32);
  void* p = nullptr;
  cudaError_t e = arenas_[0]->alloc((size_t)words_ * n * 4, &p);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: root states");
  root_->d_states = (uint32_t*)p;
  root_->dev = 0;
  e = cudaMemcpy(root_->d_states, root_host, (size_t)words_ * n * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: root upload");
  std::vector<uint16_t> ident(n);
  for (int i = 0; i < n; ++i) ident[i] = (uint16_t)i;
  for (size_t g = 0; g < models_.size(); ++g) {
    e = arenas_[g]->alloc((size_t)n * 2, &p);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: identity");
    ident_[g] = (uint16_t*)p;
    e = cudaMemcpy(ident_[g], ident.data(), (size_t)n * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: identity upload");
  }
  e = cudaSetDevice(m_->device);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_plan: device");
  uint64_t steps0 = 0, steps1 = 0;
  uint32_t status = 0;
  dsp_status s = DSP_OK;
  for (dsp_model* m : models_) {
    uint64_t x = 0;
    uint32_t st = 0;
    s = dsp_read_counters(m, &x, &st);
    if (s != DSP_OK) return s;
    steps0 += x;
  }
  if (!p_.deterministic && p_.use_queue && models_.size() == 1) {
    // the model keeps its queue (and the persistent kernel's graph) across
    // planning steps; every job carries the plan step it was submitted under
    const int want = std::max(64, 4 * p_.threads);
    if (m_->queue != nullptr && m_->queue_cap < want) {
      dsp_queue_destroy(m_->queue);
      m_->queue = nullptr;
    }
    if (m_->queue == nullptr) {
      s = dsp_queue_create(m_, want, 0, &m_->queue);
      if (s != DSP_OK) return s;
      m_->queue_cap = want;
    }
    queue_ = m_->queue;
  }
  s = p_.deterministic ? run_rounds() : run_threads();
  queue_ = nullptr;
  cudaSetDevice(m_->device);
  if (s != DSP_OK) return s;
  for (dsp_model* m : models_) {
    uint64_t x = 0;
    uint32_t st = 0;
    s = dsp_read_counters(m, &x, &st);
    if (s != DSP_OK) return s;
    steps1 += x;
    status |= st;
  }
  if (status != 0) return fail(DSP_E_DEVICE, "dsp_plan: device status word %u", status);
  out->root_u = ld(root_->U);
  out->root_l = ld(root_->L);
  out->nodes = (int32_t)n_nodes_;
  out->expansions = expansions_.load();
  out->rounds = rounds_;
  out->scenario_steps = steps1 - steps0;
  int best = -1;
  double bl = -std::numeric_limits<double>::infinity();
  for (int a = 0; a < root_->nq; ++a)
    if (ld(root_->q[a].L) > bl) {
      bl = ld(root_->q[a].L);
      best = a;
    }
  out->action = best;
  uint64_t sig = 0x12345678ull;
  for_each_node([&](const Node* v) {
    uint64_t ub, lb;
    const double vu = ld(v->U), vlo = ld(v->L);
    std::memcpy(&ub, &vu, 8);
    std::memcpy(&lb, &vlo, 8);
    sig = mix64(sig ^ (uint64_t)v->depth) ^ v->key;
    sig = mix64(sig ^ ub) ^ lb;
    sig = mix64(sig ^ (uint64_t)v->n ^ ((uint64_t)ld(v->N) << 32));
  });
  out->signature = sig;
  if (visits)
    for (int a = 0; a < root_->nq; ++a) visits[a] = (int32_t)ld(root_->Na[a]);
  out->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return DSP_OK;
}

// Expanded, non-terminal nodes with at least min_scen scenarios, in creation
// order: the tree's lower-bound action at each and its first scenario's state.
dsp_status Search::export_nodes(int min_scen, int cap, dsp_plan_node* nodes, uint32_t* states, int32_t* count) {
  int k = 0;
  std::vector<uint32_t> one(words_);
  for (size_t bi = 0; bi < blocks_.size() && k < cap; ++bi) {
    for (int bk = 0; bk < blocks_[bi].n && k < cap; ++bk) {
      const Node* v = blocks_[bi].p.get() + bk;
      if (!v->expanded.load() || v->term || v->n < min_scen || v->d_states == nullptr) continue;
      dsp_plan_node& o = nodes[k];
      o.depth = v->depth;
      o.n = v->n;
      o.visits = (int32_t)ld(v->N);
      o.U = ld(v->U);
      o.L = ld(v->L);
      std::memcpy(o.hist, v->hist, 32);
      int best = 0;
      for (int a = 1; a < v->nq; ++a)
        if (ld(v->q[a].L) > ld(v->q[best].L)) best = a;
      o.action = best;
      if (states) {
        cudaError_t e =
            cudaMemcpy2D(one.data(), 4, v->d_states, (size_t)v->n * 4, 4, words_, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "dsp_plan_nodes: node state");
        for (int w = 0; w < words_; ++w) states[(size_t)w * cap + k] = one[w];
      }
      ++k;
    }
  }
  *count = k;
  return DSP_OK;
}

// Root scenarios a plan may take: one-robot Rock Sample expands leaves of up
// to kMaxScenLarge scenarios (every leaf here has its leaf-state block),
// except through the device queue, which takes at most kMaxScen.
int max_root_scenarios(const dsp_model* m, const dsp_search_params* p) {
  const bool queue = p->use_queue && !p->deterministic;
  return m->host->kind == DSP_MODEL_GRID && !queue ? kMaxScenLarge : kMaxScen;
}

}  // namespace
}  // namespace dsp

extern "C" dsp_status dsp_plan(dsp_model* m, const uint32_t* root_states, int32_t n, const int8_t* hist,
                               const dsp_search_params* p, dsp_search_result* out, int32_t* root_visits) {
  using namespace dsp;
  if (!m || !root_states || !p || !out) return fail(DSP_E_INVALID, "dsp_plan: NULL argument");
  if (n < 1 || n > max_root_scenarios(m, p) || n > m->host->K)
    return fail(DSP_E_INVALID, "dsp_plan: %d root scenarios", n);
  if (p->threads < 1 || p->threads > 256) return fail(DSP_E_INVALID, "dsp_plan: threads %d", p->threads);
  if (p->rounds < 1) return fail(DSP_E_INVALID, "dsp_plan: rounds %d", p->rounds);
  std::memset(out, 0, sizeof(*out));
  Search s({m}, *p);
  return s.run(root_states, n, hist, out, root_visits);
}

extern "C" dsp_status dsp_route_leaves(int32_t n_leaves, int64_t first_expansion, int32_t n_models,
                                       const int32_t* parent_model, int32_t* target, int32_t* copy) {
  using namespace dsp;
  if (n_leaves < 0 || n_models < 1 || first_expansion < 0 || (n_leaves > 0 && (!parent_model || !target || !copy)))
    return fail(DSP_E_INVALID, "dsp_route_leaves: bad argument");
  for (int32_t k = 0; k < n_leaves; ++k) {
    if (parent_model[k] < 0 || parent_model[k] >= n_models)
      return fail(DSP_E_INVALID, "dsp_route_leaves: leaf %d: parent model %d of %d", k, parent_model[k], n_models);
    target[k] = (int32_t)((first_expansion + k) % n_models);
    copy[k] = target[k] != parent_model[k] ? 1 : 0;
  }
  return DSP_OK;
}

extern "C" dsp_status dsp_plan_multi(dsp_model* const* models, int32_t n_models, const uint32_t* root_states,
                                     int32_t n, const int8_t* hist, const dsp_search_params* p,
                                     dsp_search_result* out, int32_t* root_visits) {
  using namespace dsp;
  if (!models || n_models < 1 || n_models > 64) return fail(DSP_E_INVALID, "dsp_plan_multi: %d models", n_models);
  for (int32_t g = 0; g < n_models; ++g)
    if (!models[g]) return fail(DSP_E_INVALID, "dsp_plan_multi: model %d is NULL", g);
  if (!root_states || !p || !out) return fail(DSP_E_INVALID, "dsp_plan_multi: NULL argument");
  for (int32_t g = 1; g < n_models; ++g)
    if (std::memcmp(models[g]->host, models[0]->host, sizeof(DevModel)) != 0 ||
        models[g]->plan_step != models[0]->plan_step || models[g]->policy_on != models[0]->policy_on)
      return fail(DSP_E_INVALID, "dsp_plan_multi: model %d differs from model 0 (description, plan step or policy)",
                  g);
  if (n_models > 1 && p->use_queue && !p->deterministic)
    return fail(DSP_E_UNSUPPORTED, "dsp_plan_multi: the device queue serves one model");
  if (n < 1 || n > max_root_scenarios(models[0], p) || n > models[0]->host->K)
    return fail(DSP_E_INVALID, "dsp_plan_multi: %d root scenarios", n);
  if (p->threads < 1 || p->threads > 256) return fail(DSP_E_INVALID, "dsp_plan_multi: threads %d", p->threads);
  if (p->rounds < 1) return fail(DSP_E_INVALID, "dsp_plan_multi: rounds %d", p->rounds);
  std::memset(out, 0, sizeof(*out));
  cudaError_t e = cudaSetDevice(models[0]->device);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_plan_multi: device");
  Search s(std::vector<dsp_model*>(models, models + n_models), *p);
  return s.run(root_states, n, hist, out, root_visits);
}

extern "C" dsp_status dsp_plan_nodes(dsp_model* m, const uint32_t* root_states, int32_t n, const int8_t* hist,
                                     const dsp_search_params* p, dsp_search_result* out, int32_t* root_visits,
                                     int32_t min_scen, int32_t cap, dsp_plan_node* nodes, uint32_t* states,
                                     int32_t* count) {
  using namespace dsp;
  if (!nodes || !count || cap < 0) return fail(DSP_E_INVALID, "dsp_plan_nodes: NULL node buffer");
  *count = 0;
  if (!m || !root_states || !p || !out) return fail(DSP_E_INVALID, "dsp_plan_nodes: NULL argument");
  if (n < 1 || n > max_root_scenarios(m, p) || n > m->host->K)
    return fail(DSP_E_INVALID, "dsp_plan_nodes: %d root scenarios", n);
  if (p->threads < 1 || p->threads > 256) return fail(DSP_E_INVALID, "dsp_plan_nodes: threads %d", p->threads);
  if (p->rounds < 1) return fail(DSP_E_INVALID, "dsp_plan_nodes: rounds %d", p->rounds);
  std::memset(out, 0, sizeof(*out));
  Search s({m}, *p);
  dsp_status st = s.run(root_states, n, hist, out, root_visits);
  if (st != DSP_OK) return st;
  return s.export_nodes(min_scen, cap, nodes, states, count);
}
