// Default-policy rollouts (Eq. lb) with the learned policy pi0, one-robot Rock
// Sample. A CTA keeps 64 live scenarios (rows) and advances them one step at a
// time: each row writes its features (BF16) into a shared tile, the network
// runs as tensor-core tiles over the 64 rows (mma.sync m16n8k16, BF16 inputs,
// FP32 accumulation; weights resident in shared memory), each row takes the
// argmax of its first |A| logits (lowest index on ties) and steps g exactly as
// the heuristic rollout does. A row whose scenario ends (terminal or depth D)
// adds its value to its child and takes the next item at once, so the tile
// stays full until the item list runs out.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"
#include "mlp.cuh"
#include "model.hpp"
#include "rs_common.cuh"

struct dsp_mlp;  // training object (mlp_train.cu); its FP32 master is read here
extern "C" dsp_status dsp_mlp_get_weights(const dsp_mlp* mlp, float* host_params);

namespace dsp {
namespace {

constexpr int kRows = 64;        // scenarios per CTA
constexpr int kThreads = 128;    // 4 warps x 16 rows for the tensor-core layers
// device policy buffer: transposed BF16 weights [n][k], FP32 biases
constexpr size_t kPolW1 = 0;
constexpr size_t kPolW2 = kPolW1 + (size_t)kMlpHid * kMlpIn * 2;
constexpr size_t kPolW3 = kPolW2 + (size_t)kMlpHid * kMlpHid * 2;
constexpr size_t kPolB1 = kPolW3 + (size_t)kMlpOut * kMlpHid * 2;
constexpr size_t kPolB2 = kPolB1 + kMlpHid * 4;
constexpr size_t kPolB3 = kPolB2 + kMlpHid * 4;
constexpr size_t kPolBytes = kPolB3 + kMlpOut * 4;

// shared memory in 32-bit words (BF16 pairs); rows of 32 or 128 words with
// the word index XOR-swizzled by (row & 7) << 2, so the eight rows a fragment
// load touches fall in distinct banks
struct MlpSmem {
  uint32_t w1[kMlpHid * (kMlpIn / 2)];
  uint32_t w2[kMlpHid * (kMlpHid / 2)];
  uint32_t w3[kMlpOut * (kMlpHid / 2)];
  uint32_t x[kRows * (kMlpIn / 2)];
  uint32_t h[kRows * (kMlpHid / 2)];
  float b1[kMlpHid], b2[kMlpHid], b3[kMlpOut];
  RSShared c;
  int act[kRows];
  uint32_t allow[kRows];  // bit a: action a allowed for the row (learned_allow); bit |A|: defer
  int heur[kRows];        // the heuristic policy's action for the row (taken on defer)
};

__device__ __forceinline__ int swz(int row, int word) { return word ^ ((row & 7) << 2); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Actions the learned policy may take (a function of the observable history):
// no move off the N, S or W border and no Sample off an unsampled rock (both
// cost -100 and leave the state unchanged, so a deterministic policy would
// repeat them to depth D), no Sense of a sampled rock or of one whose counter
// reads +-3 (the features clamp there). East is always allowed.
__device__ __forceinline__ uint32_t learned_allow(const RSShared& c, int n, int m, uint32_t pos, uint32_t sampled,
                                                  const int8_t* cnt) {
  const int x = (int)(pos & 0xFFu), y = (int)((pos >> 8) & 0xFFu);
  uint32_t a = 0x2u;
  if (y < n - 1) a |= 0x1u;
  if (y > 0) a |= 0x4u;
  if (x > 0) a |= 0x8u;
  const int i = c.cell_rock[y * n + x];
  if (i != 0xFF && !((sampled >> i) & 1u)) a |= 0x10u;
  for (int r = 0; r < m; ++r)
    if (!((sampled >> r) & 1u) && cnt[r] < 3 && cnt[r] > -3) a |= 0x20u << r;
  return a;
}

// The network on the 64 rows of S.x; writes S.act: the argmax of the logits
// over the allowed actions of S.allow and column na ("defer"), lowest index on
// ties, with defer replaced by the heuristic's action S.heur. All 128
// threads; warp w owns rows 16w .. 16w + 15.
__device__ __forceinline__ void policy_tile(MlpSmem& S, int na) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = 16 * warp + g, r1 = r0 + 8;
  // layer 1: h = relu(x W1 + b1), 64 columns at a time
  for (int nc = 0; nc < kMlpHid; nc += 64) {
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll
    for (int kw = 0; kw < kMlpIn / 2; kw += 8) {
      uint32_t a0 = S.x[r0 * 32 + swz(r0, kw + t)], a1 = S.x[r1 * 32 + swz(r1, kw + t)];
      uint32_t a2 = S.x[r0 * 32 + swz(r0, kw + t + 4)], a3 = S.x[r1 * 32 + swz(r1, kw + t + 4)];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int n = nc + 8 * j + g;
        mma16816(acc[j], a0, a1, a2, a3, S.w1[n * 32 + swz(n, kw + t)], S.w1[n * 32 + swz(n, kw + t + 4)]);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int col = nc + 8 * j + 2 * t;
      float bl = S.b1[col], bh = S.b1[col + 1];
      S.h[r0 * 128 + swz(r0, col / 2)] = pack_bf16(fmaxf(acc[j][0] + bl, 0.0f), fmaxf(acc[j][1] + bh, 0.0f));
      S.h[r1 * 128 + swz(r1, col / 2)] = pack_bf16(fmaxf(acc[j][2] + bl, 0.0f), fmaxf(acc[j][3] + bh, 0.0f));
    }
  }
  __syncwarp();
  // layer 2: h = relu(h W2 + b2), all 256 columns kept in registers, then
  // written over the warp's own rows
  {
    float acc[32][4];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll 2
    for (int kw = 0; kw < kMlpHid / 2; kw += 8) {
      uint32_t a0 = S.h[r0 * 128 + swz(r0, kw + t)], a1 = S.h[r1 * 128 + swz(r1, kw + t)];
      uint32_t a2 = S.h[r0 * 128 + swz(r0, kw + t + 4)], a3 = S.h[r1 * 128 + swz(r1, kw + t + 4)];
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        int n = 8 * j + g;
        mma16816(acc[j], a0, a1, a2, a3, S.w2[n * 128 + swz(n, kw + t)], S.w2[n * 128 + swz(n, kw + t + 4)]);
      }
    }
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      int col = 8 * j + 2 * t;
      float bl = S.b2[col], bh = S.b2[col + 1];
      S.h[r0 * 128 + swz(r0, col / 2)] = pack_bf16(fmaxf(acc[j][0] + bl, 0.0f), fmaxf(acc[j][1] + bh, 0.0f));
      S.h[r1 * 128 + swz(r1, col / 2)] = pack_bf16(fmaxf(acc[j][2] + bl, 0.0f), fmaxf(acc[j][3] + bh, 0.0f));
    }
  }
  __syncwarp();
  // layer 3: logits = h W3 + b3, then the argmax of each row
  float acc[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.0f;
#pragma unroll 4
  for (int kw = 0; kw < kMlpHid / 2; kw += 8) {
    uint32_t a0 = S.h[r0 * 128 + swz(r0, kw + t)], a1 = S.h[r1 * 128 + swz(r1, kw + t)];
    uint32_t a2 = S.h[r0 * 128 + swz(r0, kw + t + 4)], a3 = S.h[r1 * 128 + swz(r1, kw + t + 4)];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int n = 8 * j + g;
      mma16816(acc[j], a0, a1, a2, a3, S.w3[n * 128 + swz(n, kw + t)], S.w3[n * 128 + swz(n, kw + t + 4)]);
    }
  }
  float best0 = -3.0e38f, best1 = -3.0e38f;
  int arg0 = 0x7FFF, arg1 = 0x7FFF;
  const uint32_t al0 = S.allow[r0], al1 = S.allow[r1];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int col = 8 * j + 2 * t + e;
      if (col <= na) {
        float v0 = acc[j][e] + S.b3[col], v1 = acc[j][2 + e] + S.b3[col];
        if (((al0 >> col) & 1u) && (arg0 == 0x7FFF || v0 > best0)) {
          best0 = v0;
          arg0 = col;
        }
        if (((al1 >> col) & 1u) && (arg1 == 0x7FFF || v1 > best1)) {
          best1 = v1;
          arg1 = col;
        }
      }
    }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    float ov0 = __shfl_xor_sync(0xFFFFFFFFu, best0, o), ov1 = __shfl_xor_sync(0xFFFFFFFFu, best1, o);
    int oa0 = __shfl_xor_sync(0xFFFFFFFFu, arg0, o), oa1 = __shfl_xor_sync(0xFFFFFFFFu, arg1, o);
    if (oa0 != 0x7FFF && (arg0 == 0x7FFF || ov0 > best0 || (ov0 == best0 && oa0 < arg0))) {
      best0 = ov0;
      arg0 = oa0;
    }
    if (oa1 != 0x7FFF && (arg1 == 0x7FFF || ov1 > best1 || (ov1 == best1 && oa1 < arg1))) {
      best1 = ov1;
      arg1 = oa1;
    }
  }
  if (t == 0) {
    S.act[r0] = arg0 == na ? S.heur[r0] : arg0;
    S.act[r1] = arg1 == na ? S.heur[r1] : arg1;
  }
}

// Where the rows' scenarios come from and where their values go.
struct ItemSource {
  // expansion: the grouping phase's item list
  const dsp_leaf_job* jobs;
  Items<1> items;
  // single rollouts (dsp_rollout): a state block, per-scenario counters
  const uint32_t* block;
  int cap, count, start_depth;
  const int8_t* hist;
  float* value;
  int32_t* log;  // [count][D] actions, or null
  unsigned int* next;  // item counter
};

template <bool kExpand>
__global__ void __launch_bounds__(kThreads, 1) rs_rollout_mlp_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                     const uint8_t* __restrict__ policy,
                                                                     ItemSource src, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MlpSmem& S = *reinterpret_cast<MlpSmem*>(smem_raw);
  const int tid = threadIdx.x;
  load_rs_consts(S.c, gm);
  {
    const uint32_t* w1 = reinterpret_cast<const uint32_t*>(policy + kPolW1);
    const uint32_t* w2 = reinterpret_cast<const uint32_t*>(policy + kPolW2);
    const uint32_t* w3 = reinterpret_cast<const uint32_t*>(policy + kPolW3);
    for (int i = tid; i < kMlpHid * 32; i += kThreads) S.w1[(i / 32) * 32 + swz(i / 32, i % 32)] = w1[i];
    for (int i = tid; i < kMlpHid * 128; i += kThreads) S.w2[(i / 128) * 128 + swz(i / 128, i % 128)] = w2[i];
    for (int i = tid; i < kMlpOut * 128; i += kThreads) S.w3[(i / 128) * 128 + swz(i / 128, i % 128)] = w3[i];
    const float* b1 = reinterpret_cast<const float*>(policy + kPolB1);
    const float* b2 = reinterpret_cast<const float*>(policy + kPolB2);
    const float* b3 = reinterpret_cast<const float*>(policy + kPolB3);
    for (int i = tid; i < kMlpHid; i += kThreads) {
      S.b1[i] = b1[i];
      S.b2[i] = b2[i];
    }
    for (int i = tid; i < kMlpOut; i += kThreads) S.b3[i] = b3[i];
  }
  __syncthreads();
  const RSModel<1> M = make_rs<1>(gm, &S.c, plan_step);
  const int na = gm->num_actions;
  const long long total = kExpand ? src.items.total : (long long)src.count;
  // per-row state (threads 0..63)
  RSS s;
  uint32_t h[8];
  uint32_t pm = 0;
  int t = 0, t0 = 0;
  float v = 0.0f, u = 0.0f;
  long long item = -1;
  bool alive = false, exhausted = false;
  const dsp_leaf_job* J = nullptr;
  uint32_t slot = 0;
  unsigned long long steps = 0;
  while (true) {
    if (tid < kRows) {
      // refill: take items until one needs rolling out (or none is left)
      while (!alive && !exhausted) {
        long long it = (long long)atomicAdd(src.next, 1u);
        if (it >= total) {
          exhausted = true;
          break;
        }
        item = it;
        v = 0.0f;
        if (kExpand) {
          s.pos[0] = src.items.f(0)[it];
          s.pos[1] = 0u;
          s.good = src.items.f(1)[it];
          s.sampled = src.items.f(2)[it];
          s.scen = src.items.f(3)[it];
          const uint32_t meta = src.items.f(5)[it];
          J = src.jobs + src.items.f(6)[it];
          slot = meta & 0xFFFFFFu;
          t0 = (int)(meta >> 24) + 1;
          const uint32_t* hw = reinterpret_cast<const uint32_t*>(J->hist);
#pragma unroll
          for (int k = 0; k < 8; ++k) h[k] = hw[k];
          pm = positive_mask(h, M.m);
          const int cap = J->child_cap;
          M.observe(h, pm, J->first_action + (int)(slot / (uint32_t)cap), J->child_key[slot]);
          u = M.terminal(s) ? 0.0f : ((t0 >= M.D) ? M.tail(s) : M.upper(s));
        } else {
          s = M.load(src.block, src.cap, (int)it);
#pragma unroll
          for (int k = 0; k < 8; ++k)
            h[k] = src.hist ? *reinterpret_cast<const uint32_t*>(src.hist + 32 * (size_t)it + 4 * k) : 0u;
          pm = positive_mask(h, M.m);
          t0 = src.start_depth;
        }
        t = t0;
        if (t < M.D && !M.terminal(s)) {
          alive = true;
        } else {
          if (!M.terminal(s)) v = __fadd_rn(v, __fmul_rn(S.c.G[M.D - t0], M.tail(s)));
          if (kExpand) {
            atomicAdd((unsigned long long*)(J->u_sum + slot), (unsigned long long)to_fixed(u));
            atomicAdd((unsigned long long*)(J->l_sum + slot), (unsigned long long)to_fixed(v));
          } else {
            src.value[it] = v;
          }
        }
      }
      // features of the row's state and counters, BF16 into the tile
      float f[kMlpIn];
      if (alive) {
        int8_t cnt[kMaxRocks];
#pragma unroll
        for (int r = 0; r < kMaxRocks; ++r) cnt[r] = (int8_t)((h[r >> 2] >> (8 * (r & 3))) & 0xFFu);
        rs_features(M.n, M.m, S.c.rock_xy, s.pos[0], s.sampled, cnt, f);
        S.allow[tid] = learned_allow(S.c, M.n, M.m, s.pos[0], s.sampled, cnt) | (1u << na);
        S.heur[tid] = M.policy(s, pm);
      } else {
        S.allow[tid] = 0x2u;
        S.heur[tid] = 1;
#pragma unroll
        for (int k = 0; k < kMlpIn; ++k) f[k] = 0.0f;
      }
#pragma unroll
      for (int w = 0; w < kMlpIn / 2; ++w) S.x[tid * 32 + swz(tid, w)] = pack_bf16(f[2 * w], f[2 * w + 1]);
    }
    if (!__syncthreads_or(alive ? 1 : 0)) break;
    policy_tile(S, na);
    __syncthreads();
    if (tid < kRows && alive) {
      const int a = S.act[tid];
      if (!kExpand && src.log) src.log[(size_t)item * M.D + (t - t0)] = a;
      uint64_t key;
      float r = M.step(s, a, t, key);
      M.observe(h, pm, a, key);
      if (r != 0.0f) v = __fadd_rn(v, __fmul_rn(S.c.G[t - t0], r));
      t += 1;
      steps += 1;
      if (M.terminal(s) || t >= M.D) {
        if (!M.terminal(s)) v = __fadd_rn(v, __fmul_rn(S.c.G[M.D - t0], M.tail(s)));
        if (kExpand) {
          atomicAdd((unsigned long long*)(J->u_sum + slot), (unsigned long long)to_fixed(u));
          atomicAdd((unsigned long long*)(J->l_sum + slot), (unsigned long long)to_fixed(v));
        } else {
          src.value[item] = v;
        }
        alive = false;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

__global__ void pack_policy(const float* master, uint8_t* pol) {
  __nv_bfloat16* w1 = reinterpret_cast<__nv_bfloat16*>(pol + kPolW1);
  __nv_bfloat16* w2 = reinterpret_cast<__nv_bfloat16*>(pol + kPolW2);
  __nv_bfloat16* w3 = reinterpret_cast<__nv_bfloat16*>(pol + kPolW3);
  float* b1 = reinterpret_cast<float*>(pol + kPolB1);
  float* b2 = reinterpret_cast<float*>(pol + kPolB2);
  float* b3 = reinterpret_cast<float*>(pol + kPolB3);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpHid * kMlpHid; i += gridDim.x * blockDim.x) {
    int n = i / kMlpHid, k = i % kMlpHid;
    w2[i] = __float2bfloat16_rn(master[kOffW2 + k * kMlpHid + n]);
    if (i < kMlpHid * kMlpIn) {
      int n1 = i / kMlpIn, k1 = i % kMlpIn;
      w1[i] = __float2bfloat16_rn(master[kOffW1 + k1 * kMlpHid + n1]);
    }
    if (i < kMlpOut * kMlpHid) {
      int n3 = i / kMlpHid, k3 = i % kMlpHid;
      w3[i] = __float2bfloat16_rn(master[kOffW3 + k3 * kMlpOut + n3]);
    }
    if (i < kMlpHid) {
      b1[i] = master[kOffB1 + i];
      b2[i] = master[kOffB2 + i];
    }
    if (i < kMlpOut) b3[i] = master[kOffB3 + i];
  }
}

template <bool kExpand>
cudaError_t launch_mlp(const DevModel* gm, DevWork* work, const uint8_t* policy, const ItemSource& src,
                       uint32_t plan_step, int num_sms, long long total, cudaStream_t st) {
  size_t smem = sizeof(MlpSmem);
  cudaError_t e = cudaFuncSetAttribute(rs_rollout_mlp_kernel<kExpand>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (int)std::max(1LL, std::min<long long>((total + kRows - 1) / kRows, (long long)num_sms));
  rs_rollout_mlp_kernel<kExpand><<<grid, kThreads, smem, st>>>(gm, work, policy, src, plan_step);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rs_rollout_mlp_items(const DevModel* gm, DevWork* work, const dsp_leaf_job* jobs,
                                        uint32_t* item_buf, long long total_items, unsigned int* counter,
                                        const void* policy, uint32_t plan_step, int num_sms, cudaStream_t st) {
  ItemSource src{};
  src.jobs = jobs;
  src.items = Items<1>{item_buf, total_items};
  src.next = counter;
  return launch_mlp<true>(gm, work, (const uint8_t*)policy, src, plan_step, num_sms, total_items, st);
}

__global__ void features_kernel(const DevModel* __restrict__ gm, const uint32_t* __restrict__ block, int cap,
                                int count, const int8_t* __restrict__ hist, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float f[kMlpIn];
  rs_features(gm->n, gm->m, gm->rock_xy, block[i], block[3 * (size_t)cap + i], hist + (size_t)i * 32, f);
  float4* o = reinterpret_cast<float4*>(out + (size_t)i * kMlpIn);
  for (int k = 0; k < kMlpIn / 4; ++k) o[k] = make_float4(f[4 * k], f[4 * k + 1], f[4 * k + 2], f[4 * k + 3]);
}

}  // namespace dsp

using namespace dsp;

extern "C" {

dsp_status dsp_features(const dsp_model* m, const uint32_t* block, int32_t cap, int32_t count, const int8_t* hist,
                        float* out, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_features: model is NULL");
  if (m->host->kind != DSP_MODEL_GRID) return fail(DSP_E_UNSUPPORTED, "dsp_features: one-robot Rock Sample only");
  if (count < 0 || cap < count || (count > 0 && (!block || !hist || !out)))
    return fail(DSP_E_INVALID, "dsp_features: bad buffers");
  if (((uintptr_t)out & 15) != 0) return fail(DSP_E_INVALID, "dsp_features: out must be 16-byte aligned");
  if (count == 0) return DSP_OK;
  features_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->dmodel, block, cap, count, hist, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_features");
}

dsp_status dsp_set_policy(dsp_model* m, const dsp_mlp* mlp) {
  if (!m) return fail(DSP_E_INVALID, "dsp_set_policy: model is NULL");
  if (mlp == nullptr) {
    m->policy_on = false;
    return DSP_OK;
  }
  if (m->host->kind != DSP_MODEL_GRID)
    return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: the learned policy serves one-robot Rock Sample");
  if (m->host->num_actions + 1 > kMlpOut)
    return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: more than 31 actions (the network's last used logit defers)");
  if (m->host->m > 15) return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: features hold 15 rocks");
  cudaError_t e = cudaSuccess;
  if (m->policy == nullptr) e = cudaMalloc(&m->policy, kPolBytes);
  float* master = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&master, kMlpParams * sizeof(float));
  std::vector<float> host(kMlpParams);
  dsp_status s = dsp_mlp_get_weights(mlp, host.data());
  if (s != DSP_OK) {
    if (master) cudaFree(master);
    return s;
  }
  if (e == cudaSuccess) e = cudaMemcpy(master, host.data(), kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    pack_policy<<<256, 256>>>(master, (uint8_t*)m->policy);
    e = cudaDeviceSynchronize();
  }
  if (master) cudaFree(master);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_set_policy");
  m->policy_on = true;
  return DSP_OK;
}

dsp_status dsp_rollout_logged(const dsp_model* m, const uint32_t* block, int32_t cap, int32_t count,
                              const int8_t* hist, int32_t start_depth, float* value, int32_t* actions,
                              void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_rollout_logged: model is NULL");
  if (!m->policy_on) return fail(DSP_E_UNSUPPORTED, "dsp_rollout_logged: no learned policy set");
  if (count < 0 || cap < count || !block || !value) return fail(DSP_E_INVALID, "dsp_rollout_logged: bad buffers");
  if (start_depth < 0 || start_depth > m->host->D) return fail(DSP_E_INVALID, "dsp_rollout_logged: start depth");
  if (count == 0) return DSP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned int* counter = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&counter, sizeof(unsigned int), m->pool, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned int), st);
  if (e == cudaSuccess) {
    ItemSource src{};
    src.block = block;
    src.cap = cap;
    src.count = count;
    src.start_depth = start_depth;
    src.hist = hist;
    src.value = value;
    src.log = actions;
    src.next = counter;
    e = launch_mlp<false>(m->dmodel, m->dwork, (const uint8_t*)m->policy, src, m->plan_step, m->num_sms, count, st);
  }
  if (counter) cudaFreeAsync(counter, st);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_rollout_logged");
}

}  // extern "C"
