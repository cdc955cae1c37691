// Default-policy rollouts (Eq. lb) of the car among pedestrians with the
// learned policy pi0, on the fifth-generation tensor cores. A CTA keeps 128
// live scenarios: two adjacent lanes share one scenario (each moves every
// other pedestrian pair, as the car expansion's lanes do) and the scenario is
// row `lane pair` of the network's 128-row tile. Per step every pair writes
// its scenario's features into the layer-1 A tile, the three layers run as
// tcgen05.mma (tc_mlp.cuh), the thread that owns the row in tensor memory takes
// the argmax of its logits over the three actions and "defer" (the heuristic
// policy's action) and hands it back through shared memory, and the pair steps
// g exactly as the heuristic rollout does. A finished scenario adds its value
// to its child (or to its output slot) and the pair takes the next item.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "car_model.cuh"
#include "kernels.cuh"
#include "mlp.cuh"
#include "model.hpp"
#include "tc_mlp.cuh"

namespace dsp {

// Feature values of the car policy (26 used of 64): s / path length, v / 3,
// then for the 8 pedestrians nearest to the car (squared distance, lower
// index first on ties, nearest first) dx / 10, dy / 10 and 1 if the
// pedestrian is in the heuristic policy's danger zone (0 < dx <= 4,
// -1 <= dy <= 1). Both lanes of the pair call it; both end with the values.
constexpr int kCarFeat = 26;

struct Near8 {
  float d[8], ex[8], ey[8];
  int i[8];
};

__device__ __forceinline__ void near_insert(Near8& N, float d, int idx, float ex, float ey) {
  // the new entry sinks through the sorted list; at each slot the smaller
  // (distance, index) stays
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool before = d < N.d[q] || (d == N.d[q] && idx < N.i[q]);
    const float td = N.d[q], tx = N.ex[q], ty = N.ey[q];
    const int ti = N.i[q];
    if (before) {
      N.d[q] = d;
      N.ex[q] = ex;
      N.ey[q] = ey;
      N.i[q] = idx;
      d = td;
      ex = tx;
      ey = ty;
      idx = ti;
    }
  }
}

template <int TPS>
__device__ __forceinline__ void car_features_group(const CarModel<TPS>& M, const CarLane<TPS>& L,
                                                   float (&F)[kCarFeat]) {
  static_assert(TPS == 2, "the pair merge assumes two lanes per scenario");
  const float cx = __fadd_rn(-10.0f, L.s), cy = 20.0f;
  Near8 N;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    N.d[q] = 3.0e38f;
    N.ex[q] = N.ey[q] = 0.0f;
    N.i[q] = 0x7FFFFFFF;
  }
#pragma unroll
  for (int k = 0; k < CarLane<TPS>::kPairs; ++k)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int j = 2 * (M.gl + k * TPS) + e;
      if (j < M.P) {
        const float ex = __fsub_rn(L.px[2 * k + e], cx), ey = __fsub_rn(L.py[2 * k + e], cy);
        near_insert(N, __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), j, ex, ey);
      }
    }
  // merge the partner lane's list
  float od[8], ox[8], oy[8];
  int oi[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    od[q] = __shfl_xor_sync(0xFFFFFFFFu, N.d[q], 1);
    ox[q] = __shfl_xor_sync(0xFFFFFFFFu, N.ex[q], 1);
    oy[q] = __shfl_xor_sync(0xFFFFFFFFu, N.ey[q], 1);
    oi[q] = __shfl_xor_sync(0xFFFFFFFFu, N.i[q], 1);
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) near_insert(N, od[q], oi[q], ox[q], oy[q]);
  F[0] = __fmul_rn(L.s, __fdiv_rn(1.0f, M.path_len));
  F[1] = __fmul_rn((float)L.v, __fdiv_rn(1.0f, 3.0f));
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const bool have = N.i[q] != 0x7FFFFFFF;
    const float ex = N.ex[q], ey = N.ey[q];
    F[2 + 3 * q] = have ? __fmul_rn(ex, 0.1f) : 0.0f;
    F[3 + 3 * q] = have ? __fmul_rn(ey, 0.1f) : 0.0f;
    F[4 + 3 * q] = (have && ex > 0.0f && ex <= 4.0f && ey >= -1.0f && ey <= 1.0f) ? 1.0f : 0.0f;
  }
}

namespace {

using namespace tc;

constexpr int kTPS = 2;  // lanes per car scenario

struct CarTcSmem {
  Weights W;
  uint8_t x[kRows * kMlpIn * 2];  // A of layer 1: the 128 scenarios' features
  CarShared c;
  int act[kRows];                 // the chosen action of each row
  int heur[kRows];                // the heuristic policy's action of each row (defer)
  long long lrow[kRows];          // logged rollouts: the row's logits slot (item * D + step), or -1
  unsigned long long mbar;
  uint32_t tmem_base;
};

struct CarItemSource {
  const dsp_leaf_job* jobs;  // expansion: the items of the car expansion
  CarItems items;
  const uint32_t* block;     // single rollouts: a state block
  int cap, count, start_depth;
  float* value;
  int32_t* log;              // [count][D] actions, or null
  float* logits;             // [count][D][32] logits of every step (bias added), or null
  unsigned int* next;
};

template <bool kExpand>
__global__ void __launch_bounds__(kThreads, 1) car_rollout_tc_kernel(const DevModel* __restrict__ gm,
                                                                     DevWork* work,
                                                                     const uint8_t* __restrict__ policy,
                                                                     CarItemSource src, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CarTcSmem& S = *reinterpret_cast<CarTcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, half = tid >> 7;
  const int row = tid / kTPS;  // the pair's scenario and network row
  load_car_consts(S.c, gm);
  load_weights(S.W, policy);
  const uint32_t mbar = smem_u32(&S.mbar);
  setup(mbar, smem_u32(&S.tmem_base));
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = S.tmem_base;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const uint32_t sx = smem_u32(S.x);
  const CarModel<kTPS> M = make_car_model<kTPS>(gm, &S.c, plan_step);
  constexpr int na = 3;
  const long long total = kExpand ? src.items.total : (long long)src.count;

  CarLane<kTPS> L;
  L.s = 0.0f;
  L.v = 0;
  L.term = true;
  L.scen = 0;
  L.goals = 0;
#pragma unroll
  for (int k = 0; k < 2 * CarLane<kTPS>::kPairs; ++k) L.px[k] = L.py[k] = 0.0f;
  float v = 0.0f;
  int t = 0, t0 = 0;
  long long item = -1;
  bool alive = false, exhausted = false, failed = false;
  const dsp_leaf_job* J = nullptr;
  uint32_t slot = 0, phase = 0;
  unsigned long long steps = 0;
  while (true) {
    // refill the pair's scenario (both lanes take the same item)
    while (!alive && !exhausted) {
      unsigned long long it = 0;
      if (M.gl == 0) it = atomicAdd(src.next, 1u);
      it = __shfl_sync(M.gmask, it, M.gbase);
      if ((long long)it >= total) {
        exhausted = true;
        break;
      }
      item = (long long)it;
      v = 0.0f;
      if (kExpand) {
        M.load(L, src.items.base, (int)src.items.total, (int)it);
        const uint32_t meta = src.items.meta()[it];
        J = src.jobs + src.items.job()[it];
        slot = meta & 0xFFFFFFu;
        t0 = (int)(meta >> 24) + 1;
      } else {
        M.load(L, src.block, src.cap, (int)it);
        t0 = src.start_depth;
      }
      t = t0;
      if (t < M.D && !L.term) {
        alive = true;
      } else if (M.gl == 0) {  // nothing to roll out (the car's tail value is zero)
        if (kExpand)
          sum_add(J->l_sum + slot, to_fixed(v));
        else
          src.value[it] = v;
      }
    }
    // features into the A tile, the heuristic's action for defer
    {
      float F[kCarFeat];
      car_features_group(M, L, F);
      const bool danger = M.danger_now(L);
      if (M.gl == 0) {
        uint32_t pr[kMlpIn / 2];
#pragma unroll
        for (int p = 0; p < kMlpIn / 2; ++p)
          pr[p] = (alive && 2 * p + 1 < kCarFeat) ? pack_bf16(F[2 * p], F[2 * p + 1]) : 0u;
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; ++c)
          *reinterpret_cast<uint4*>(S.x + kmajor_off(row, 8 * c, kMlpIn)) =
              make_uint4(pr[4 * c], pr[4 * c + 1], pr[4 * c + 2], pr[4 * c + 3]);
        S.heur[row] = M.policy(L, danger);
        S.lrow[row] = alive ? item * M.D + (t - t0) : -1LL;
      }
    }
    fence_async_smem();
    if (!__syncthreads_or(alive ? 1 : 0)) break;
    if (!run_layers(S.W, sx, tmem, trow, mbar, phase, half, []() {})) {
      failed = true;
      break;
    }
    float lg[32];
    if (half == 0) tmem_ld32(trow + kColL, lg);
    fence_before_sync();
    if (tid < kRows) {
      const int best = masked_argmax(lg, S.W.b3, 0xFu, na);
      S.act[tid] = best == na ? S.heur[tid] : best;
      if (!kExpand && src.logits && S.lrow[tid] >= 0) {
        float4* o = reinterpret_cast<float4*>(src.logits + (size_t)S.lrow[tid] * kMlpOut);
#pragma unroll
        for (int q = 0; q < kMlpOut / 4; ++q)
          o[q] = make_float4(__fadd_rn(lg[4 * q], S.W.b3[4 * q]), __fadd_rn(lg[4 * q + 1], S.W.b3[4 * q + 1]),
                             __fadd_rn(lg[4 * q + 2], S.W.b3[4 * q + 2]), __fadd_rn(lg[4 * q + 3], S.W.b3[4 * q + 3]));
      }
    }
    __syncthreads();
    // step the pair's scenario (every lane calls: the step takes group ballots)
    const int a = S.act[row];
    const uint32_t ufail = M.fail_word(L.scen, t);
    bool danger_next;
    uint64_t key;
    const float r = M.template step<false>(L, alive, a, t, ufail, danger_next, key);
    if (alive) {
      if (!kExpand && src.log && M.gl == 0) src.log[(size_t)item * M.D + (t - t0)] = a;
      v = __fadd_rn(v, __fmul_rn(S.c.G[t - t0], r));
      t += 1;
      if (M.gl == 0) steps += 1;
      if (L.term || t >= M.D) {
        if (M.gl == 0) {
          if (kExpand)
            sum_add(J->l_sum + slot, to_fixed(v));
          else
            src.value[item] = v;
        }
        alive = false;
      }
    }
  }
  teardown(tmem, mbar, phase, failed, work);
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_features for the car: one lane pair per scenario, FP32 values.
__global__ void car_features_kernel(const DevModel* __restrict__ gm, const uint32_t* __restrict__ block, int cap,
                                    int count, float* __restrict__ out) {
  __shared__ CarShared c;
  load_car_consts(c, gm);
  __syncthreads();
  const CarModel<kTPS> M = make_car_model<kTPS>(gm, &c, 0u);
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) / kTPS;
  CarLane<kTPS> L;
  M.load(L, block, cap, i < count ? i : 0);
  float F[kCarFeat];
  car_features_group(M, L, F);
  if (i < count && M.gl == 0) {
    float4* o = reinterpret_cast<float4*>(out + (size_t)i * kMlpIn);
#pragma unroll
    for (int k = 0; k < kMlpIn / 4; ++k) {
      float q[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) q[e] = 4 * k + e < kCarFeat ? F[4 * k + e] : 0.0f;
      o[k] = make_float4(q[0], q[1], q[2], q[3]);
    }
  }
}

// The car's hand-written default policy per state (kTPS lanes per state).
__global__ void car_policy_kernel(const DevModel* __restrict__ gm, const uint32_t* __restrict__ block, int cap,
                                  int count, int32_t* __restrict__ actions) {
  __shared__ CarShared c;
  load_car_consts(c, gm);
  __syncthreads();
  const CarModel<kTPS> M = make_car_model<kTPS>(gm, &c, 0u);
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) / kTPS;
  CarLane<kTPS> L;
  M.load(L, block, cap, i < count ? i : 0);
  const int a = M.policy(L, M.danger_now(L));
  if (i < count && M.gl == 0) actions[i] = a;
}

template <bool kExpand>
cudaError_t launch_car_mlp(const dsp_model* m, const CarItemSource& src, long long total, cudaStream_t st) {
  size_t smem = sizeof(CarTcSmem);
  cudaError_t e = cudaFuncSetAttribute(car_rollout_tc_kernel<kExpand>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (int)std::max(1LL, std::min<long long>((total + kRows - 1) / kRows, (long long)m->num_sms));
  car_rollout_tc_kernel<kExpand><<<grid, kThreads, smem, st>>>(m->dmodel, m->dwork, (const uint8_t*)m->policy, src,
                                                               m->plan_step);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_car_rollout_mlp_items(dsp_model* m, const dsp_leaf_job* jobs, CarItems items, unsigned int* counter,
                                         cudaStream_t st) {
  CarItemSource src{};
  src.jobs = jobs;
  src.items = items;
  src.next = counter;
  return launch_car_mlp<true>(m, src, items.total, st);
}

cudaError_t launch_car_rollout_logged(const dsp_model* m, const uint32_t* block, int cap, int count, int start_depth,
                                      float* value, int32_t* actions, float* logits, unsigned int* counter,
                                      cudaStream_t st) {
  CarItemSource src{};
  src.block = block;
  src.cap = cap;
  src.count = count;
  src.start_depth = start_depth;
  src.value = value;
  src.log = actions;
  src.logits = logits;
  src.next = counter;
  return launch_car_mlp<false>(m, src, count, st);
}

cudaError_t launch_car_features(const dsp_model* m, const uint32_t* block, int cap, int count, float* out,
                                cudaStream_t st) {
  const int threads = 256, per = threads / kTPS;
  car_features_kernel<<<(count + per - 1) / per, threads, 0, st>>>(m->dmodel, block, cap, count, out);
  return cudaGetLastError();
}

cudaError_t launch_car_policy(const dsp_model* m, const uint32_t* block, int cap, int count, int32_t* actions,
                              cudaStream_t st) {
  const int threads = 256, per = threads / kTPS;
  car_policy_kernel<<<(count + per - 1) / per, threads, 0, st>>>(m->dmodel, block, cap, count, actions);
  return cudaGetLastError();
}

}  // namespace dsp
