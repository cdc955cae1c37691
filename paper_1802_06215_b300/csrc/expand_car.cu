// Leaf expansion for the car among pedestrians, one persistent kernel: each
// unit is (job, one action); TPS lanes share a scenario (element-level
// parallelism, Sec. III-D) through gather, update, the expansion step with its
// observation key, u0 and the default-policy rollout; then the CTA groups the
// action's scenarios by key (Eq. newnodes), checks every member's full
// observation (speed and all pedestrian cells, kept in a per-CTA scratch slot
// in global memory) against its child's first member, and sums rewards and
// bounds per child in int64 fixed point.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "car_model.cuh"
#include "group.cuh"
#include "model.hpp"
#include "queue_ring.cuh"

namespace dsp {
namespace {

constexpr int kCarObsWords = kMaxPeds + 1;  // speed | terminal, then one word per pedestrian

// The children's int64 sums reuse the grouping's hash table (keys and first
// positions, 12 KB), which is dead once group_by_key has returned: 51 KB per
// CTA, so that four CTAs share an SM.
struct CarUnitSmem {
  CarShared c;
  uint64_t key[kMaxScen];
  float rew[kMaxScen], uval[kMaxScen], lval[kMaxScen];
  GroupSmem grp;
  int unit;
  dsp_leaf_job job;
};
static_assert(sizeof(GroupSmem::tkey) >= 2 * kMaxScen * sizeof(unsigned long long) &&
                  sizeof(GroupSmem::tfirst) >= kMaxScen * sizeof(unsigned long long),
              "the sums alias the hash table");

// One (job, action) unit of the car expansion by the whole CTA, the job's
// descriptor in S.job: gather + update into the leaf, the expansion step
// with its observation key, u0, and the rollout (or, with a learned policy,
// the stepped state into the item list at item_base), then the grouping by
// key with the full-observation check, the per-child sums and the results
// of action offset `ao`. obs: the CTA's observation scratch. Ends with a
// barrier.
template <int TPS, int KP>
__device__ __forceinline__ void car_unit(CarUnitSmem& S, const CarModel<TPS, KP>& M, int ao, long long item_base,
                                         int job_index, uint32_t* obs, const CarItems& items, DevWork* work,
                                         unsigned long long& steps) {
  const int P = M.P;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int groups = nthr / TPS, g = tid / TPS;
  const dsp_leaf_job& job = S.job;
  const int n = job.n_scen, depth = job.depth;
  const int a = job.first_action + ao;
  const bool first_unit = ao == 0;
  for (int base = 0; base < n; base += groups) {
    const int p = base + g;
    const bool valid = p < n;
    CarLane<TPS, KP> L;
    if (valid) {
      M.load(L, job.parent, job.parent_cap, job.idx[p]);
    } else {
      L.s = 0.0f;
      L.v = 0;
      L.term = true;
      L.scen = 0;
      L.goals = 0;
#pragma unroll
      for (int k = 0; k < 2 * CarLane<TPS, KP>::kPairs; ++k) L.px[k] = L.py[k] = 0.0f;
    }
    bool danger = false;
    uint64_t key = 0;
    if (job.last_action >= 0) {  // update by the action into this leaf
      bool live = valid && !L.term;
      if (live && M.gl == 0 && first_unit) steps += 1;
      uint32_t uf = M.fail_word(L.scen, depth - 1);
      M.template step<false>(L, live, job.last_action, depth - 1, uf, danger, key);
    }
    if (first_unit && job.leaf_states != nullptr) M.store(L, job.leaf_states, n, p, valid);
    // Eq. expand with the observation key
    bool live = valid && !L.term;
    if (live && M.gl == 0) steps += 1;
    uint32_t uf = M.fail_word(L.scen, depth);
    float r = M.template step<true>(L, live, a, depth, uf, danger, key);
    if (valid) {
      uint32_t* ob = obs + (size_t)p * kCarObsWords;
      if (M.gl == 0) ob[0] = (uint32_t)L.v | ((uint32_t)L.term << 8);
#pragma unroll
      for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          int j = 2 * (M.gl + k * TPS) + e;
          if (j < P) {
            int qx = (int)floorf(__fmul_rn(2.0f, L.px[2 * k + e]));
            int qy = (int)floorf(__fmul_rn(2.0f, L.py[2 * k + e]));
            ob[1 + j] = (uint32_t)(uint16_t)(int16_t)qx | ((uint32_t)(uint16_t)(int16_t)qy << 16);
          }
        }
    }
    // Eq. ub (the tail heuristic is zero at depth D) and Eq. lb; with a
    // learned policy the stepped state goes to the item list instead and the
    // learned-rollout kernel adds the rollout values afterwards
    float uv = (depth + 1 >= M.D) ? 0.0f : M.upper(L);
    float lv = 0.0f;
    if (items.base != nullptr)
      M.store(L, items.base, (int)items.total, item_base + p, valid);
    else
      lv = M.rollout(L, valid, danger, depth + 1, steps);
    if (valid && M.gl == 0) {
      S.key[p] = key;
      S.rew[p] = r;
      S.uval[p] = uv;
      S.lval[p] = lv;
    }
  }
  __syncthreads();
  group_by_key(S.grp, S.key, n);
  const int nchild = S.grp.nchild;
  unsigned long long* sr = reinterpret_cast<unsigned long long*>(S.grp.tkey);
  unsigned long long* su = sr + kMaxScen;
  unsigned long long* sl = reinterpret_cast<unsigned long long*>(S.grp.tfirst);
  for (int c = tid; c < nchild; c += nthr) {
    sr[c] = 0;
    su[c] = 0;
    sl[c] = 0;
  }
  __syncthreads();
  // full-observation check of every member against its child's first member
  for (int q = tid; q < n; q += nthr) {
    int c = S.grp.gcid[q];
    int f = S.grp.cfirst[c];
    if (f != q) {
      const uint32_t* a0 = obs + (size_t)f * kCarObsWords;
      const uint32_t* a1 = obs + (size_t)q * kCarObsWords;
      bool same = a0[0] == a1[0];
      for (int w = 1; w <= P; ++w) same = same && (a0[w] == a1[w]);
      if (!same) report(work, kStatusKeyClash);
    }
    atomicAdd(&sr[c], (unsigned long long)to_fixed(S.rew[q]));
    atomicAdd(&su[c], (unsigned long long)to_fixed(S.uval[q]));
    atomicAdd(&sl[c], (unsigned long long)to_fixed(S.lval[q]));
  }
  __syncthreads();
  const int cap = job.child_cap;
  if (tid == 0) {
    job.child_count[ao] = nchild;
    if (nchild > cap) report(work, kStatusOverflow);
  }
  const int ncw = min(nchild, cap);
  for (int c = tid; c <= ncw; c += nthr) job.child_off[(size_t)ao * (cap + 1) + c] = c < nchild ? S.grp.coff[c] : n;
  for (int c = tid; c < ncw; c += nthr) {
    size_t o = (size_t)ao * cap + c;
    job.child_key[o] = S.key[S.grp.cfirst[c]];
    job.rew_sum[o] = (long long)sr[c];
    job.u_sum[o] = (long long)su[c];
    job.l_sum[o] = (long long)sl[c];
  }
  for (int q = tid; q < n; q += nthr) {
    int c = S.grp.gcid[q];
    job.perm[(size_t)ao * n + S.grp.coff[c] + S.grp.rank[q]] = (uint16_t)q;
    if (items.base != nullptr) {
      items.meta()[item_base + q] = ((uint32_t)depth << 24) | (uint32_t)(ao * cap + min(c, cap - 1));
      items.job()[item_base + q] = (uint32_t)job_index;
    }
  }
  __syncthreads();
}

// CTAs per SM the register budget is sized for: the pairs a lane holds set
// the registers it needs
template <int TPS, int KP>
constexpr int kCarMinBlocks = (TPS >= 16 || KP == 1) ? 4 : (KP == 2 ? 3 : (KP <= 4 ? 2 : 1));

template <int TPS, int KP = kDefaultPairs<TPS>>
__global__ void __launch_bounds__(256, (kCarMinBlocks<TPS, KP>)) car_expand_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                         const dsp_leaf_job* __restrict__ jobs,
                                                         const int4* __restrict__ units, int n_units,
                                                         unsigned int* head, uint32_t plan_step,
                                                         uint32_t* scratch, CarItems items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CarUnitSmem& S = *reinterpret_cast<CarUnitSmem*>(smem_raw);
  load_car_consts(S.c, gm);
  CarModel<TPS, KP> M = make_car_model<TPS, KP>(gm, &S.c, plan_step);
  const int tid = threadIdx.x;
  uint32_t* obs = scratch + (size_t)blockIdx.x * kMaxScen * kCarObsWords;
  unsigned long long steps = 0;
  __syncthreads();
  while (true) {
    if (tid == 0) S.unit = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int u = S.unit;
    __syncthreads();
    if (u >= n_units) break;
    const int4 un = units[u];
    if (tid == 0) S.job = jobs[un.x];
    __syncthreads();
    car_unit<TPS, KP>(S, M, un.y, un.z, un.x, obs, items, work, steps);
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_step for the car (TPS = 8 lanes per scenario).
__global__ void __launch_bounds__(256) car_step_kernel(const DevModel* __restrict__ gm, const uint32_t* in,
                                                       int in_cap, int count, const int32_t* actions, int depth,
                                                       uint32_t* out, int out_cap, uint64_t* keys, float* rewards,
                                                       uint32_t plan_step) {
  constexpr int TPS = 8;
  __shared__ CarShared c;
  load_car_consts(c, gm);
  __syncthreads();
  CarModel<TPS> M = make_car_model<TPS>(gm, &c, plan_step);
  const int groups = blockDim.x / TPS;
  for (int base = blockIdx.x * groups; base < count; base += gridDim.x * groups) {
    int i = base + (int)threadIdx.x / TPS;
    bool valid = i < count;
    CarLane<TPS> L;
    M.load(L, in, in_cap, valid ? i : 0);
    bool live = valid && !L.term;
    int a = valid ? actions[i] : 0;
    uint32_t uf = M.fail_word(L.scen, depth);
    bool danger;
    uint64_t key;
    float r = M.template step<true>(L, live, a, depth, uf, danger, key);
    M.store(L, out, out_cap, i, valid);
    if (valid && M.gl == 0) {
      keys[i] = key;
      rewards[i] = r;
    }
  }
}

// dsp_rollout for the car (TPS = 8).
__global__ void __launch_bounds__(256) car_rollout_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                          const uint32_t* block, int cap, int count,
                                                          int start_depth, float* value, uint32_t plan_step) {
  constexpr int TPS = 8;
  __shared__ CarShared c;
  load_car_consts(c, gm);
  __syncthreads();
  CarModel<TPS> M = make_car_model<TPS>(gm, &c, plan_step);
  const int groups = blockDim.x / TPS;
  unsigned long long steps = 0;
  for (int base = blockIdx.x * groups; base < count; base += gridDim.x * groups) {
    int i = base + (int)threadIdx.x / TPS;
    bool valid = i < count;
    CarLane<TPS> L;
    M.load(L, block, cap, valid ? i : 0);
    if (!valid) L.term = true;
    bool danger = M.danger_now(L);
    float v = M.rollout(L, valid, danger, start_depth, steps);
    if (valid && M.gl == 0) value[i] = v;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// Persistent queue kernel of the car: a CTA claims a published job, runs its
// actions as units (car_unit, heuristic rollouts) with its own observation
// scratch, then publishes the job done. Idle CTAs back off and exit after
// idle_ns without a job; the host relaunches the kernel when jobs come.
template <int TPS, int KP = kDefaultPairs<TPS>>
__global__ void __launch_bounds__(256, (kCarMinBlocks<TPS, KP>))
    car_queue_kernel(const DevModel* __restrict__ gm, DevWork* work, QueueRing ring, unsigned long long* head,
                     uint32_t* scratch, dsp_leaf_job* jcopy, unsigned long long idle_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CarUnitSmem& S = *reinterpret_cast<CarUnitSmem*>(smem_raw);
  __shared__ long long s_ticket;
  __shared__ unsigned int s_plan_step;
  __shared__ int s_exit;
  load_car_consts(S.c, gm);
  CarModel<TPS, KP> M = make_car_model<TPS, KP>(gm, &S.c, 0u);
  const int tid = threadIdx.x;
  uint32_t* obs = scratch + (size_t)blockIdx.x * kMaxScen * kCarObsWords;
  const CarItems none{nullptr, 0, 0};
  unsigned long long steps = 0, last_work = qring::now_ns();
  unsigned int backoff = 256;
  __syncthreads();
  while (true) {
    if (tid < 32) {
      const long long t = qring::take_job(ring, head, &S.job, jcopy, &s_plan_step);
      if (tid == 0) s_ticket = t;
    }
    __syncthreads();
    const long long ticket = s_ticket;
    if (ticket >= 0) {
      M.plan_step = s_plan_step;
      for (int ao = 0; ao < S.job.n_actions; ++ao) car_unit<TPS, KP>(S, M, ao, 0, 0, obs, none, work, steps);
      __threadfence();  // every thread's results, before the job is published done
      __syncthreads();
      if (tid == 0) qring::finish_job(ring, (unsigned long long)ticket);
    }
    if (tid == 0) s_exit = qring::idle_exit(ring, ticket >= 0, last_work, backoff, idle_ns);
    __syncthreads();
    if (s_exit) break;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

template <int TPS, int KP>
cudaError_t queue_tps(dsp_model* m, QueueRing ring, unsigned long long* head, uint32_t* scratch, dsp_leaf_job* jcopy,
                      unsigned long long idle_ns, int grid, cudaStream_t st) {
  car_queue_kernel<TPS, KP><<<grid, 256, sizeof(CarUnitSmem), st>>>(m->dmodel, m->dwork, ring, head, scratch, jcopy,
                                                                     idle_ns);
  return cudaGetLastError();
}

template <int TPS, int KP>
cudaError_t queue_tps_setup(int* per_sm) {
  const size_t smem = sizeof(CarUnitSmem);
  cudaError_t e =
      cudaFuncSetAttribute(car_queue_kernel<TPS, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, car_queue_kernel<TPS, KP>, 256, smem);
  return e;
}

template <int TPS, int KP = kDefaultPairs<TPS>>
cudaError_t launch_tps(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units, unsigned int* head,
                       CarItems items, cudaStream_t st) {
  size_t smem = sizeof(CarUnitSmem);
  cudaError_t e =
      cudaFuncSetAttribute(car_expand_kernel<TPS, KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, car_expand_kernel<TPS, KP>, 256, smem);
  if (m->tune_ctas_car > 0) per_sm = std::min(per_sm, m->tune_ctas_car);
  per_sm = std::max(1, per_sm);
  int grid = std::max(1, std::min(n_units, per_sm * m->num_sms));
  // observation slots, one per CTA, stream-ordered so that launches on other
  // streams (other search threads) never share them
  size_t need = (size_t)grid * kMaxScen * kCarObsWords * sizeof(uint32_t);
  uint32_t* scratch = nullptr;
  e = cudaMallocFromPoolAsync((void**)&scratch, need, m->pool, st);
  if (e != cudaSuccess) return e;
  car_expand_kernel<TPS, KP><<<grid, 256, smem, st>>>(m->dmodel, m->dwork, djobs, dunits, n_units, head,
                                                       m->plan_step, scratch, items);
  e = cudaGetLastError();
  cudaError_t e2 = cudaFreeAsync(scratch, st);
  return e != cudaSuccess ? e : e2;
}

// Pairs per lane fitted to the crowd: KP = ceil(pairs / TPS) up to four
// pairs a lane, else the kernel sized for kMaxPeds; f is called with the
// chosen KP as a std::integral_constant.
template <int TPS, class F>
cudaError_t with_fitted_pairs(int pairs, F&& f) {
  const int kp = (pairs + TPS - 1) / TPS;
  if (kp <= 1) return f(std::integral_constant<int, 1>{});
  if constexpr (kDefaultPairs<TPS> > 2)
    if (kp == 2) return f(std::integral_constant<int, 2>{});
  if constexpr (kDefaultPairs<TPS> > 3)
    if (kp == 3) return f(std::integral_constant<int, 3>{});
  if constexpr (kDefaultPairs<TPS> > 4)
    if (kp == 4) return f(std::integral_constant<int, 4>{});
  return f(std::integral_constant<int, kDefaultPairs<TPS>>{});
}

// f called with the lanes per scenario tps as a std::integral_constant
template <class F>
cudaError_t with_tps(int tps, F&& f) {
  switch (tps) {
    case 4: return f(std::integral_constant<int, 4>{});
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    default: return f(std::integral_constant<int, 32>{});
  }
}

}  // namespace

// The untuned lanes per scenario: the one whose pair slots (TPS lanes x
// fitted pairs per lane) the crowd fills best; on a tie the most lanes
// (fewer registers per lane).
int car_default_tps(int P) {
  const int pairs = (P + 1) / 2;
  int best = 32;
  double best_fill = -1.0;
  for (int tps : {32, 16, 8, 4}) {
    int kp = (pairs + tps - 1) / tps;
    if (kp > 4) kp = (kMaxPeds / 2 + tps - 1) / tps;
    const double fill = (double)pairs / (double)(tps * std::max(1, kp));
    if (fill > best_fill + 1e-9) {
      best_fill = fill;
      best = tps;
    }
  }
  return best;
}

cudaError_t launch_car_expand(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units,
                              unsigned int* head, CarItems items, cudaStream_t st) {
  const int pairs = (m->host->P + 1) / 2;
  return with_tps(m->tune_tps > 0 ? m->tune_tps : car_default_tps(m->host->P), [&](auto t) {
    constexpr int TPS = decltype(t)::value;
    return with_fitted_pairs<TPS>(pairs, [&](auto k) {
      return launch_tps<TPS, decltype(k)::value>(m, djobs, dunits, n_units, head, items, st);
    });
  });
}

// The persistent queue kernel's lanes per scenario: the expansion's untuned
// default for the crowd, with the fitted pairs per lane. Sets the kernel's
// shared-memory limit (before any capture) and returns the CTAs that fit per
// SM.
cudaError_t car_queue_setup(const dsp_model* m, int* per_sm) {
  const int pairs = (m->host->P + 1) / 2;
  return with_tps(car_default_tps(m->host->P), [&](auto t) {
    constexpr int TPS = decltype(t)::value;
    return with_fitted_pairs<TPS>(pairs, [&](auto k) { return queue_tps_setup<TPS, decltype(k)::value>(per_sm); });
  });
}

size_t car_queue_scratch_words(int grid) { return (size_t)grid * kMaxScen * kCarObsWords; }

cudaError_t launch_car_queue(dsp_model* m, QueueRing ring, unsigned long long* head, uint32_t* scratch,
                             dsp_leaf_job* jcopy, unsigned long long idle_ns, int grid, cudaStream_t st) {
  const int pairs = (m->host->P + 1) / 2;
  return with_tps(car_default_tps(m->host->P), [&](auto t) {
    constexpr int TPS = decltype(t)::value;
    return with_fitted_pairs<TPS>(pairs, [&](auto k) {
      return queue_tps<TPS, decltype(k)::value>(m, ring, head, scratch, jcopy, idle_ns, grid, st);
    });
  });
}

cudaError_t launch_car_step(const DevModel* gm, int P, const uint32_t* in, int in_cap, int count,
                            const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                            float* rewards, uint32_t plan_step, cudaStream_t st) {
  (void)P;
  int groups = 256 / 8;
  int grid = std::min(4096, (count + groups - 1) / groups);
  car_step_kernel<<<grid, 256, 0, st>>>(gm, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                                        plan_step);
  return cudaGetLastError();
}

cudaError_t launch_car_rollout(const DevModel* gm, int P, DevWork* work, const uint32_t* block, int cap, int count,
                               int start_depth, float* value, uint32_t plan_step, cudaStream_t st) {
  (void)P;
  int groups = 256 / 8;
  int grid = std::min(4096, (count + groups - 1) / groups);
  car_rollout_kernel<<<grid, 256, 0, st>>>(gm, work, block, cap, count, start_depth, value, plan_step);
  return cudaGetLastError();
}

}  // namespace dsp
