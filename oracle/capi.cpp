// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// C entry points of the oracle for the test suite (loaded with ctypes). State
// blocks use the same word format as the product library's boundary (each
// model's pack/unpack documents it); everything else is the oracle's own.
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "despot.hpp"
#include "mlp.hpp"
#include "pomcp.hpp"

using namespace orc;

extern "C" {

typedef struct {
  int32_t kind;  // 0 grid (1 robot), 1 multigrid (2 robots), 2 car, 3 navigation
  int32_t n, m, P;
  float gamma;
  int32_t K, D;
  uint64_t seed;
  uint32_t plan_step;
  const int32_t* rock_cells;  // m entries, x | y << 8
  float path_len, dt, ped_speed, sigma;
  double fail_p;  // car: accelerate/decelerate failure; navigation: move failure
  int32_t fp64;   // 1: FP64 oracle, 0: FP32 oracle
  double sense_p;  // navigation: probability that one adjacent-cell reading is wrong
} orc_model;

typedef struct {
  int32_t threads, rounds;
  double c_a, c_o, xi, target_gap;
} orc_search_params;

typedef struct {
  double root_u, root_l;
  int32_t action, nodes, expansions, rounds;
  uint64_t steps, signature;
} orc_search_result;

void orc_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, int32_t rounds, uint32_t* out) {
  Block4 b = philox4x32(ctr, k0, k1, rounds);
  for (int i = 0; i < 4; ++i) out[i] = b.w[i];
}

void orc_scenario_random(uint64_t seed, uint32_t scen, uint32_t depth, uint32_t purpose, uint32_t element,
                         uint32_t plan_step, uint32_t* out) {
  Block4 b = scenario_random(seed, scen, depth, purpose, element, plan_step);
  for (int i = 0; i < 4; ++i) out[i] = b.w[i];
}

void orc_sensor_thresholds(int32_t max_d2, uint64_t* out) {
  std::vector<uint64_t> t = sensor_thresholds(max_d2);
  std::memcpy(out, t.data(), t.size() * 8);
}

void orc_gamma_powers(float gamma, int32_t n, float* out32, double* out64) {
  std::vector<float> g32 = gamma_powers<float>(gamma, n);
  std::vector<double> g64 = gamma_powers<double>(gamma, n);
  for (int i = 0; i < n; ++i) {
    out32[i] = g32[i];
    out64[i] = g64[i];
  }
}

}  // extern "C"

namespace {

const std::vector<double>& cached_gauss() {
  static std::once_flag once;
  static std::vector<double> t;
  std::call_once(once, [] { t = gauss_table_f64(); });
  return t;
}

template <class Real>
RockSample<Real> make_rs(const orc_model* d) {
  RockSample<Real> m;
  m.n = d->n;
  m.m = d->m;
  m.robots = d->kind == 1 ? 2 : 1;
  m.gamma = d->gamma;
  m.K = d->K;
  m.D = d->D;
  m.seed = d->seed;
  m.plan_step = d->plan_step;
  for (int i = 0; i < d->m; ++i) {
    m.rock_x[i] = d->rock_cells[i] & 0xFF;
    m.rock_y[i] = (d->rock_cells[i] >> 8) & 0xFF;
  }
  m.init();
  return m;
}

template <class Real>
Car<Real> make_car(const orc_model* d) {
  Car<Real> m;
  m.P = d->P;
  m.gamma = d->gamma;
  m.K = d->K;
  m.D = d->D;
  m.seed = d->seed;
  m.plan_step = d->plan_step;
  m.path_len = d->path_len;
  m.dt = d->dt;
  m.ped_speed = d->ped_speed;
  m.sigma = d->sigma;
  m.fail_p = d->fail_p;
  m.G = gamma_powers<Real>(m.gamma, 256);
  const std::vector<double>& g = cached_gauss();
  m.gauss.resize(4096);
  for (int i = 0; i < 4096; ++i) m.gauss[i] = (Real)g[i];
  m.fail_thresh = (uint64_t)std::floor(m.fail_p * 4294967296.0);
  return m;
}

template <class Real>
Nav<Real> make_nav(const orc_model* d) {
  Nav<Real> m;
  m.n = d->n;
  m.gamma = d->gamma;
  m.K = d->K;
  m.D = d->D;
  m.seed = d->seed;
  m.plan_step = d->plan_step;
  m.fail_p = d->fail_p;
  m.sense_p = d->sense_p;
  m.init();
  return m;
}

Hist hist_from(const int8_t* h) {
  Hist x{};
  if (h)
    for (int i = 0; i < 32; ++i) x.c[i] = h[i];
  return x;
}

// Runs `f(model)` with the model the descriptor names.
template <class F>
int with_model(const orc_model* d, F f) {
  if (d->kind == 0 || d->kind == 1) {
    if (d->fp64)
      f(make_rs<double>(d));
    else
      f(make_rs<float>(d));
    return 0;
  }
  if (d->kind == 2) {
    if (d->fp64)
      f(make_car<double>(d));
    else
      f(make_car<float>(d));
    return 0;
  }
  if (d->kind == 3) {
    if (d->fp64)
      f(make_nav<double>(d));
    else
      f(make_nav<float>(d));
    return 0;
  }
  return 1;
}

template <class M>
auto unpack_all(const M& m, const uint32_t* block, int cap, int count) {
  using S = decltype(m.unpack(block, cap, 0));
  std::vector<S> v(count);
  for (int i = 0; i < count; ++i) v[i] = m.unpack(block, cap, i);
  return v;
}

}  // namespace

extern "C" {

uint64_t orc_ops_read(void) { return op_counter(); }
void orc_ops_reset(void) { op_counter() = 0; }

void orc_gauss_table(double* out64, float* out32) {
  const std::vector<double>& g = cached_gauss();
  for (int i = 0; i < 4096; ++i) {
    out64[i] = g[i];
    out32[i] = (float)g[i];
  }
}

int32_t orc_state_words(const orc_model* d) {
  if (d->kind == 2) return 4 + 2 * d->P + (d->P + 3) / 4;
  if (d->kind == 3) return 2 + (d->n * d->n + 31) / 32;
  return 5;
}

// g for each scenario i of a block: (s', z, r) = g(s_i, actions[i], phi_depth).
int32_t orc_step(const orc_model* d, const uint32_t* in_block, int32_t cap, int32_t count,
                 const int32_t* actions, int32_t depth, uint32_t* out_block, int32_t out_cap, uint64_t* keys,
                 double* rewards) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, in_block, cap, count);
    for (int i = 0; i < count; ++i) {
      auto next = st[i];
      uint64_t key;
      auto r = m.step(st[i], actions[i], depth, next, &key);
      m.pack(next, out_block, out_cap, i);
      keys[i] = key;
      rewards[i] = (double)r;
    }
  });
}

// Default-policy value (Eq. lb for one scenario) from each state at start_depth;
// hist holds 32 counters per scenario.
int32_t orc_rollout(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count, const int8_t* hist,
                    int32_t start_depth, double* values, uint64_t* steps) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, block, cap, count);
    uint64_t total = 0;
    for (int i = 0; i < count; ++i) {
      uint64_t s = 0;
      values[i] = (double)rollout(m, st[i], hist_from(hist ? hist + 32 * i : nullptr), start_depth, &s);
      total += s;
    }
    *steps = total;
  });
}

// Heuristic u of each state and the horizon tail l.
int32_t orc_bounds(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count, double* upper,
                   double* tail) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, block, cap, count);
    for (int i = 0; i < count; ++i) {
      upper[i] = (double)m.upper(st[i]);
      tail[i] = (double)m.tail(st[i]);
    }
  });
}

int32_t orc_policy(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count, const int8_t* hist,
                   int32_t* actions) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, block, cap, count);
    for (int i = 0; i < count; ++i) actions[i] = m.policy(st[i], hist_from(hist ? hist + 32 * i : nullptr));
  });
}

// Leaf initialisation of one leaf (see despot.hpp). Output arrays are sized
// na, na*(cap+1), na*cap and na*n; leaf_block gets the leaf's n states.
int32_t orc_expand(const orc_model* d, const uint32_t* parent_block, int32_t parent_cap, int32_t parent_count,
                   const uint16_t* idx, int32_t n, int32_t last_action, int32_t depth, const int8_t* hist,
                   int32_t a0, int32_t na, int32_t cap, uint32_t* leaf_block, int32_t* child_count,
                   int32_t* child_off, uint64_t* key, int64_t* rew, int64_t* u, int64_t* l, uint16_t* perm,
                   uint64_t* steps) {
  return with_model(d, [&](const auto& m) {
    auto parent = unpack_all(m, parent_block, parent_cap, parent_count);
    using S = typename decltype(parent)::value_type;
    ExpandOut<S> e;
    expand_leaf(m, parent, idx, n, last_action, depth, hist_from(hist), a0, na, cap, e);
    if (leaf_block)
      for (int i = 0; i < n; ++i) m.pack(e.leaf[i], leaf_block, n, i);
    std::memcpy(child_count, e.child_count.data(), na * 4);
    std::memcpy(child_off, e.child_off.data(), e.child_off.size() * 4);
    std::memcpy(key, e.key.data(), e.key.size() * 8);
    std::memcpy(rew, e.rew.data(), e.rew.size() * 8);
    std::memcpy(u, e.u.data(), e.u.size() * 8);
    std::memcpy(l, e.l.data(), e.l.size() * 8);
    std::memcpy(perm, e.perm.data(), e.perm.size() * 2);
    *steps = e.steps;
  });
}

// One planning step of the tree search from the given root scenarios.
int32_t orc_plan(const orc_model* d, const uint32_t* root_block, int32_t n, const int8_t* hist,
                 const orc_search_params* p, orc_search_result* out, int32_t* root_na) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, root_block, n, n);
    using S = typename decltype(st)::value_type;
    SearchParams prm;
    prm.threads = p->threads;
    prm.rounds = p->rounds;
    prm.c_a = p->c_a;
    prm.c_o = p->c_o;
    prm.xi = p->xi;
    prm.target_gap = p->target_gap;
    Despot<std::decay_t<decltype(m)>, S> ds(m, prm);
    SearchResult r = ds.plan(st, hist_from(hist));
    out->root_u = r.root_u;
    out->root_l = r.root_l;
    out->action = r.action;
    out->nodes = r.nodes;
    out->expansions = r.expansions;
    out->rounds = r.rounds;
    out->steps = r.steps;
    out->signature = r.signature;
    if (root_na)
      for (size_t a = 0; a < r.root_na.size(); ++a) root_na[a] = r.root_na[a];
  });
}

typedef struct {
  int32_t action;
  double value;
  int32_t nodes, simulations, rollouts;
  uint64_t steps, signature;
} orc_pomcp_result;

// POMCP-style planning (pomcp.hpp) from the given root scenarios.
int32_t orc_pomcp(const orc_model* d, const uint32_t* root_block, int32_t n, const int8_t* hist, int32_t rounds,
                  int32_t batch, double c, orc_pomcp_result* out, double* root_q, int32_t* root_na) {
  return with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, root_block, n, n);
    using S = typename decltype(st)::value_type;
    PomcpParams prm;
    prm.rounds = rounds;
    prm.batch = batch;
    prm.c = c;
    Pomcp<std::decay_t<decltype(m)>, S> pc(m, prm);
    PomcpResult r = pc.plan(st, hist_from(hist));
    out->action = r.action;
    out->value = r.value;
    out->nodes = r.nodes;
    out->simulations = r.simulations;
    out->rollouts = r.rollouts;
    out->steps = r.steps;
    out->signature = r.signature;
    for (size_t a = 0; a < r.root_q.size(); ++a) {
      if (root_q) root_q[a] = r.root_q[a];
      if (root_na) root_na[a] = r.root_na[a];
    }
  });
}

// Optimal D-horizon value of the scenario tree below the given states.
double orc_exhaustive(const orc_model* d, const uint32_t* block, int32_t n, const int8_t* hist, int32_t depth) {
  double v = 0;
  with_model(d, [&](const auto& m) {
    auto st = unpack_all(m, block, n, n);
    v = exhaustive_value(m, st, hist_from(hist), depth);
  });
  return v;
}

}  // extern "C"

// ----------------------------------------------------------- learned pi0 ---

extern "C" {

int32_t orc_mlp_forward(const double* W1, const double* b1, const double* W2, const double* b2, const double* W3,
                        const double* b3, const double* X, int32_t B, int32_t bf16, double* logits) {
  return mlp_forward(W1, b1, W2, b2, W3, b3, X, B, bf16, logits);
}

int32_t orc_mlp_loss_grad(const double* W1, const double* b1, const double* W2, const double* b2, const double* W3,
                          const double* b3, const double* X, const int32_t* y, int32_t B, int32_t n_actions,
                          double* loss, double* gW1, double* gb1, double* gW2, double* gb2, double* gW3,
                          double* gb3, int32_t bf16_forward) {
  return mlp_loss_grad(W1, b1, W2, b2, W3, b3, X, y, B, n_actions, loss, gW1, gb1, gW2, gb2, gW3, gb3,
                       bf16_forward);
}

// Policy features of a car state (not in the paper; the learned default
// policy's input): s / path length, v / 3, then for the 8 pedestrians nearest
// to the car (squared distance from the car's position, lower index first on
// ties, nearest first): dx / 10, dy / 10 (pedestrian minus car) and 1 when the
// pedestrian is in the danger zone of the heuristic policy (0 < dx <= 4,
// -1 <= dy <= 1), else 0; zero beyond. All FP32 in this order.
static void car_features(const Car<float>& m, const CarState<float>& s, float* f) {
  for (int k = 0; k < kMlpIn; ++k) f[k] = 0.0f;
  const float inv_len = 1.0f / m.path_len;
  const float third = 1.0f / 3.0f;
  f[0] = s.s * inv_len;
  f[1] = (float)s.v * third;
  const float cx = m.car_x(s), cy = m.car_y();
  int idx[8];
  float dd[8];
  int k = 0;
  for (int i = 0; i < m.P; ++i) {
    const float ex = s.px[i] - cx, ey = s.py[i] - cy;
    const float d2 = ex * ex + ey * ey;
    // insertion into the sorted list of the nearest (strictly nearer goes first)
    int at = k;
    while (at > 0 && dd[at - 1] > d2) --at;
    if (at >= 8) continue;
    for (int q = (k < 8 ? k : 7); q > at; --q) {
      dd[q] = dd[q - 1];
      idx[q] = idx[q - 1];
    }
    dd[at] = d2;
    idx[at] = i;
    if (k < 8) ++k;
  }
  for (int q = 0; q < k; ++q) {
    const float ex = s.px[idx[q]] - cx, ey = s.py[idx[q]] - cy;
    f[2 + 3 * q] = ex * 0.1f;
    f[3 + 3 * q] = ey * 0.1f;
    f[4 + 3 * q] = (ex > 0.0f && ex <= 4.0f && ey >= -1.0f && ey <= 1.0f) ? 1.0f : 0.0f;
  }
}

int32_t orc_features_car(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count, float* out) {
  if (d->kind != 2) return 1;
  Car<float> m = make_car<float>(d);
  for (int i = 0; i < count; ++i) car_features(m, m.unpack(block, cap, i), out + (size_t)i * kMlpIn);
  return 0;
}

int32_t orc_features_rs(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count, const int8_t* hist,
                        float* out) {
  return features_rs(d->n, d->m, d->rock_cells, block, cap, count, hist, out);
}

// Default-policy rollout (Eq. lb) of the car with the learned policy: the
// argmax of logits 0..3 (every action is allowed; logit 3 "defer" takes the
// heuristic policy's action), lowest index on ties; with `logged` the logged
// actions are replayed as for Rock Sample.
static int32_t rollout_learned_car(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count,
                                   int32_t start_depth, const double* W1, const double* b1, const double* W2,
                                   const double* b2, const double* W3, const double* b3, const int32_t* logged,
                                   double tol, double* values, int32_t* disagree, uint64_t* steps,
                                   double* logits_out) {
  Car<float> m = make_car<float>(d);
  Net w{W1, b1, W2, b2, W3, b3};
  const int na = m.num_actions();
  uint64_t total = 0;
  for (int i = 0; i < count; ++i) {
    CarState<float> s = m.unpack(block, cap, i);
    Hist h = hist_from(nullptr);
    float v = 0.0f;
    int t = start_depth, k = 0, bad = 0;
    while (t < m.D && !m.terminal(s)) {
      float fx[kMlpIn];
      car_features(m, s, fx);
      double x64[kMlpIn], lg[kMlpOut];
      for (int q = 0; q < kMlpIn; ++q) x64[q] = (double)fx[q];
      forward_bf16(w, x64, lg);
      if (logits_out)
        for (int q = 0; q < kMlpOut; ++q) logits_out[((size_t)i * m.D + k) * kMlpOut + q] = lg[q];
      int best = 0;
      for (int a = 1; a <= na; ++a)
        if (lg[a] > lg[best]) best = a;
      const int heur = m.policy(s, h);
      const int chosen = best == na ? heur : best;
      int a = chosen;
      if (logged) {
        a = logged[(size_t)i * m.D + k];
        bool ok = a == chosen;
        if (!ok && a >= 0 && a < na && lg[best] - lg[a] <= tol) ok = true;
        if (!ok && a == heur && lg[best] - lg[na] <= tol) ok = true;
        if (!ok) bad += 1;
        if (a < 0 || a >= na) a = chosen;
      }
      CarState<float> next;
      uint64_t key;
      float r = m.step(s, a, t, next, &key);
      v = v + m.G[t - start_depth] * r;
      s = next;
      t += 1;
      k += 1;
    }
    if (!m.terminal(s)) v = v + m.G[m.D - start_depth] * m.tail(s);
    values[i] = (double)v;
    if (disagree) disagree[i] = bad;
    total += (uint64_t)k;
  }
  *steps = total;
  return 0;
}

// Actions the learned policy may take in a one-robot Rock Sample state with
// counters h (a function of the observable history only): no move off the N,
// S or W border and no Sample off an unsampled rock (both cost -100 and leave
// the state as it was, so a deterministic policy would repeat them to depth
// D), and no Sense of a sampled rock or of one whose counter already reads
// +-3 (the features clamp there, so a repeated Sense could never change the
// policy's input). East is always allowed.
static bool learned_allowed(const RockSample<float>& m, const RSState& s, const Hist& h, int a) {
  const int x = s.x[0], y = s.y[0];
  if (a == 0) return y < m.n - 1;
  if (a == 1) return true;
  if (a == 2) return y > 0;
  if (a == 3) return x > 0;
  if (a == 4) {
    int i = m.rock_at(x, y);
    return i >= 0 && !((s.sampled >> i) & 1u);
  }
  int i = a - 5;
  return !((s.sampled >> i) & 1u) && h.c[i] < 3 && h.c[i] > -3;
}

// The learned policy's allowed actions per state of one-robot Rock Sample
// (learned_allowed), as bits, with bit |A| (defer) always set.
int32_t orc_learned_allowed(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count,
                            const int8_t* hist, uint32_t* bits) {
  if (d->kind != 0) return 1;
  RockSample<float> m = make_rs<float>(d);
  const int na = m.num_actions();
  for (int i = 0; i < count; ++i) {
    RSState s = m.unpack(block, cap, i);
    Hist h = hist_from(hist ? hist + 32 * (size_t)i : nullptr);
    uint32_t b = 1u << na;
    for (int a = 0; a < na; ++a)
      if (learned_allowed(m, s, h, a)) b |= 1u << a;
    bits[i] = b;
  }
  return 0;
}

// Default-policy rollout (Eq. lb) of one-robot Rock Sample with the learned
// policy: at every step the features of (state, counters) go through the
// network in its BF16/FP32 form; the argmax of logits 0..|A| over the allowed
// actions (learned_allowed) and logit |A| ("defer", always allowed), lowest
// index on ties, picks the action, defer meaning the heuristic policy's
// action. With `logged` (count x D actions) the rollout follows the logged
// actions instead and counts, per scenario, the steps whose logged action is
// neither this choice nor reachable by a column (an allowed action, or defer
// for the heuristic's action) within `tol` of the best logit. `logits_out`
// (count x D x 32, may be null) gets the network's logits of every step.
int32_t orc_rollout_learned(const orc_model* d, const uint32_t* block, int32_t cap, int32_t count,
                            const int8_t* hist, int32_t start_depth, const double* W1, const double* b1,
                            const double* W2, const double* b2, const double* W3, const double* b3,
                            const int32_t* logged, double tol, double* values, int32_t* disagree,
                            uint64_t* steps, double* logits_out) {
  if (d->kind == 2) return rollout_learned_car(d, block, cap, count, start_depth, W1, b1, W2, b2, W3, b3, logged, tol,
                                              values, disagree, steps, logits_out);
  if (d->kind != 0) return 1;
  RockSample<float> m = make_rs<float>(d);
  Net w{W1, b1, W2, b2, W3, b3};
  const int na = m.num_actions();
  uint64_t total = 0;
  for (int i = 0; i < count; ++i) {
    RSState s = m.unpack(block, cap, i);
    Hist h = hist_from(hist ? hist + 32 * (size_t)i : nullptr);
    float v = 0.0f;
    int t = start_depth, k = 0, bad = 0;
    while (t < m.D && !m.terminal(s)) {
      // features of this state and history (the same map as features_rs)
      uint32_t one[5];
      for (int f = 0; f < 5; ++f) one[f] = 0;
      m.pack(s, one, 1, 0);
      int8_t hh[32];
      for (int r = 0; r < 32; ++r) hh[r] = h.c[r];
      float fx[kMlpIn];
      features_rs(d->n, d->m, d->rock_cells, one, 1, 1, hh, fx);
      double x64[kMlpIn], lg[kMlpOut];
      for (int q = 0; q < kMlpIn; ++q) x64[q] = (double)fx[q];
      forward_bf16(w, x64, lg);
      if (logits_out)
        for (int q = 0; q < kMlpOut; ++q) logits_out[((size_t)i * m.D + k) * kMlpOut + q] = lg[q];
      int best = -1;
      for (int a = 0; a <= na; ++a)
        if ((a == na || learned_allowed(m, s, h, a)) && (best < 0 || lg[a] > lg[best])) best = a;
      const int heur = m.policy(s, h);
      const int chosen = best == na ? heur : best;
      int a = chosen;
      if (logged) {
        a = logged[(size_t)i * m.D + k];
        bool ok = a == chosen;
        if (!ok && a >= 0 && a < na && learned_allowed(m, s, h, a) && lg[best] - lg[a] <= tol) ok = true;
        if (!ok && a == heur && lg[best] - lg[na] <= tol) ok = true;
        if (!ok) bad += 1;
        if (a < 0 || a >= na) a = chosen;
      }
      RSState next;
      uint64_t key;
      float r = m.step(s, a, t, next, &key);
      m.observe(h, a, key);
      v = v + m.G[t - start_depth] * r;
      s = next;
      t += 1;
      k += 1;
    }
    if (!m.terminal(s)) v = v + m.G[m.D - start_depth] * m.tail(s);
    values[i] = (double)v;
    if (disagree) disagree[i] = bad;
    total += (uint64_t)k;
  }
  *steps = total;
  return 0;
}

}  // extern "C"
