// Default-policy rollouts (Eq. lb) with the learned policy pi0, one-robot Rock
// Sample, on the fifth-generation tensor cores. A CTA keeps 128 live
// scenarios (rows) and advances them one step at a time: the network runs as
// tcgen05.mma over the 128 rows (BF16 inputs, FP32 accumulators in tensor
// memory, weights resident in shared memory), each row takes the argmax of its
// logits over the allowed actions and "defer" (the heuristic's action) and
// steps g exactly as the heuristic rollout does. A row whose scenario ends
// (terminal or depth D) adds its value to its child and takes the next item at
// once, so the tile stays full until the item list runs out.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>

#include "kernels.cuh"
#include "mlp.cuh"
#include "model.hpp"
#include "rs_common.cuh"
#include "tc_mlp.cuh"

struct dsp_mlp;  // training object (mlp_train.cu); its FP32 master is read here
extern "C" dsp_status dsp_mlp_get_weights(const dsp_mlp* mlp, float* host_params);

namespace dsp {
namespace {

using namespace tc;


// Per-CTA tables of the feature pairs that depend on one rock. The offset
// pair ((float)dx / n, (float)dy / n) for dx, dy in -(n-1) .. n-1 is one BF16
// pair per entry, (2n-1)^2 entries of 4 bytes; where that table does not fit
// in shared memory (n = 32) the pair is computed from a 2n-1 entry table of
// single BF16 values. The counter/sampled pair is fcs[(c + 3) * 2 + sampled].
struct FeatTables {
  const uint32_t* pair;   // (2n-1)^2 pairs, or null
  const uint16_t* one;    // 2n-1 single values (dx + n - 1)
  const uint32_t* fcs;
  int n;
};

// The row's features (the feature map of rs_features, same arithmetic) as
// BF16 pairs straight into the layer-1 A tile: pair 0 = (x/n, y/n), pairs
// 1 + 2r = ((rock x - x)/n, (rock y - y)/n), 2 + 2r = (clamp(c_r)/3, sampled_r),
// zero beyond 1 + 2m. Fully unrolled, so nothing goes through local memory.
__device__ __forceinline__ void write_features(uint8_t* xs, int row, int m, const int* rock_xy, uint32_t pos,
                                               uint32_t sampled, const uint32_t (&h)[8], const FeatTables& T) {
  const int n = T.n, w = 2 * n - 1;
  const float inv_n = 1.0f / (float)n;
  const int x = (int)(pos & 0xFFu), y = (int)((pos >> 8) & 0xFFu);
  uint32_t pr[kMlpIn / 2];
  pr[0] = pack_bf16((float)x * inv_n, (float)y * inv_n);
#pragma unroll
  for (int r = 0; r < 15; ++r) {
    if (r < m) {
      const int rxy = rock_xy[r];
      int c = (int)(int8_t)((h[r >> 2] >> (8 * (r & 3))) & 0xFFu);
      c = c > 3 ? 3 : (c < -3 ? -3 : c);
      const int dx = (rxy & 0xFF) - x + n - 1, dy = (rxy >> 8) - y + n - 1;
      pr[1 + 2 * r] = T.pair != nullptr ? T.pair[dx * w + dy]
                                        : ((uint32_t)T.one[dx] | ((uint32_t)T.one[dy] << 16));
      pr[2 + 2 * r] = T.fcs[(c + 3) * 2 + (int)((sampled >> r) & 1u)];
    } else {
      pr[1 + 2 * r] = 0u;
      pr[2 + 2 * r] = 0u;
    }
  }
  pr[31] = 0u;
#pragma unroll
  for (int c = 0; c < kMlpIn / 8; ++c)
    *reinterpret_cast<uint4*>(xs + kmajor_off(row, 8 * c, kMlpIn)) =
        make_uint4(pr[4 * c], pr[4 * c + 1], pr[4 * c + 2], pr[4 * c + 3]);
}

// Actions the learned policy may take (a function of the observable history):
// no move off the N, S or W border and no Sample off an unsampled rock (both
// cost -100 and leave the state unchanged, so a deterministic policy would
// repeat them to depth D), no Sense of a sampled rock or of one whose counter
// reads +-3 (the features clamp there). East is always allowed.
__device__ __forceinline__ uint32_t learned_allow(const RSShared& c, int n, int m, uint32_t pos, uint32_t sampled,
                                                  const uint32_t (&h)[8]) {
  const int x = (int)(pos & 0xFFu), y = (int)((pos >> 8) & 0xFFu);
  uint32_t a = 0x2u;
  if (y < n - 1) a |= 0x1u;
  if (y > 0) a |= 0x4u;
  if (x > 0) a |= 0x8u;
  const int i = c.cell_rock[y * n + x];
  if (i != 0xFF && !((sampled >> i) & 1u)) a |= 0x10u;
#pragma unroll
  for (int r = 0; r < 15; ++r) {
    const int cr = (int)(int8_t)((h[r >> 2] >> (8 * (r & 3))) & 0xFFu);
    if (r < m && !((sampled >> r) & 1u) && cr < 3 && cr > -3) a |= 0x20u << r;
  }
  return a;
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
  float* logits;  // [count][D][32] logits of every step (bias added), or null
  unsigned int* next;  // item counter
};

// Shared memory of the learned rollout: the policy (B operands), one layer-1
// A tile per row tile, the model's constants and the feature tables (the
// pair table last, sized (2n-1)^2 at launch when it fits).
struct TcSmem {
  Weights W;
  uint8_t x[2][kRows * kMlpIn * 2];   // A of layer 1 per tile: M = 128, K = 64 (features)
  RSShared c;
  uint32_t fcs[14];                   // BF16 pair (clamp(c) / 3, sampled), c in -3..3
  uint16_t one[2 * kMaxSide];         // BF16 of (float)d / n, d in -(n-1)..n-1
  unsigned long long mbar[2];         // completion of each tile's MMAs
  uint32_t tmem_base;
  uint32_t pair[1];                   // (2n-1)^2 offset pairs when they fit (dynamic)
};
constexpr size_t kTcSmemMax = 227 * 1024;

__host__ __device__ constexpr size_t tc_pair_bytes(int n) { return (size_t)(2 * n - 1) * (2 * n - 1) * 4; }
__host__ __device__ constexpr bool tc_pair_fits(int n) { return offsetof(TcSmem, pair) + tc_pair_bytes(n) <= kTcSmemMax; }

// The learned policy's rollouts, one-robot Rock Sample. A CTA holds two
// tiles of 128 live scenarios (rows), one per warpgroup, each thread owning
// one row. Per step, each tile independently: its rows write their features
// (BF16) into the tile's layer-1 A operand in shared memory; the tile's
// first thread issues layer 1, both halves of layer 2 and layer 3 as
// tcgen05.mma (M = 128, BF16 in, FP32 accumulators in the tile's 256
// tensor-memory columns, weights resident in shared memory as the B
// operands, hidden activations fed back through tensor memory as the A
// operand), each committed to the tile's mbarrier; after each completion
// every thread reads its own row: bias + ReLU + BF16 for the hidden layers,
// then the masked argmax of its logits and g. While one tile is in its
// epilogues or its scalar step, the tensor pipe runs the other tile's
// layers. A row whose scenario ends adds its value to its child and takes
// the next item at once, so the tiles stay full until the item list runs out.
template <bool kExpand>
__global__ void __launch_bounds__(kThreads, 1) rs_rollout_tc_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                    const uint8_t* __restrict__ policy,
                                                                    ItemSource src, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tile = tid >> 7, row = tid & 127, bar = 1 + tile;
  load_rs_consts(S.c, gm);
  load_weights(S.W, policy);
  const int n = gm->n;
  const bool pairs = tc_pair_fits(n);
  {
    const float inv_n = 1.0f / (float)n;
    const float third = 1.0f / 3.0f;
    const int w = 2 * n - 1;
    if (pairs)
      for (int i = tid; i < w * w; i += blockDim.x) {
        const int dx = i / w - (n - 1), dy = i % w - (n - 1);
        S.pair[i] = pack_bf16((float)dx * inv_n, (float)dy * inv_n);
      }
    for (int i = tid; i < w; i += blockDim.x) {
      const __nv_bfloat16 b = __float2bfloat16_rn((float)(i - (n - 1)) * inv_n);
      S.one[i] = *reinterpret_cast<const uint16_t*>(&b);
    }
    for (int i = tid; i < 14; i += blockDim.x) S.fcs[i] = pack_bf16((float)(i / 2 - 3) * third, (i & 1) ? 1.0f : 0.0f);
  }
  if (tid == 0) {
    for (int g = 0; g < 2; ++g)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&S.mbar[g])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const FeatTables T{pairs ? S.pair : nullptr, S.one, S.fcs, n};
  const uint32_t tbase = S.tmem_base + (uint32_t)tile * kTileCols;          // the tile's columns
  const uint32_t trow = tbase + ((uint32_t)(32 * (warp & 3)) << 16);       // this warp's lanes
  const uint32_t sx = smem_u32(S.x[tile]);
  const uint32_t mbar = smem_u32(&S.mbar[tile]);
  const bool issuer = row == 0;

  const RSModel<1> M = make_rs<1>(gm, &S.c, plan_step);
  const int na = gm->num_actions;
  const long long total = kExpand ? src.items.total : (long long)src.count;
  RSS s;
  uint32_t h[8];
  uint32_t pm = 0, allow = 0;
  int t = 0, t0 = 0, heur = 1;
  float v = 0.0f, u = 0.0f;
  long long item = -1;
  bool alive = false;
  const dsp_leaf_job* J = nullptr;
  uint32_t slot = 0, phase = 0;
  unsigned long long steps = 0;
  bool failed = false;
  // The row's next item, fetched one dependent stage per step so that no
  // load latency stalls the tile when a rollout ends: 0 nothing fetched,
  // 1 index claimed, 2 fields loaded, 3 ready (job data loaded), 4 no items left.
  int pst = 0;
  long long pit = -1;
  uint32_t pf[7], ph[8], pcap = 1, pfa = 0;
  uint64_t pkey = 0;
  auto advance = [&]() {
    if (pst == 0) {
      pit = (long long)atomicAdd(src.next, 1u);
      pst = pit < total ? 1 : 4;
    } else if (pst == 1) {
      if (kExpand) {
#pragma unroll
        for (int k = 0; k < 7; ++k) pf[k] = src.items.f(k)[pit];
        pst = 2;
      } else {
#pragma unroll
        for (int k = 0; k < 5; ++k) pf[k] = src.block[(size_t)k * src.cap + pit];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          ph[k] = src.hist ? *reinterpret_cast<const uint32_t*>(src.hist + 32 * (size_t)pit + 4 * k) : 0u;
        pst = 3;
      }
    } else if (pst == 2) {
      const dsp_leaf_job* PJ = src.jobs + pf[6];
      const uint32_t* hw = reinterpret_cast<const uint32_t*>(PJ->hist);
#pragma unroll
      for (int k = 0; k < 8; ++k) ph[k] = hw[k];
      pcap = (uint32_t)PJ->child_cap;
      pfa = (uint32_t)PJ->first_action;
      pkey = PJ->child_key[pf[5] & 0xFFFFFFu];
      pst = 3;
    }
  };
  advance();
  advance();
  advance();
  // one step of the network: waits (bounded) for the tile's MMAs, agreed by
  // the tile's threads
  auto wait_layer = [&]() -> bool {
    const bool ok = tile_and(bar, mbar_wait(mbar, phase));
    phase ^= 1u;
    fence_after_sync();
    return ok;
  };
  while (true) {
    // a row whose scenario ended takes the fetched item (an item that needs
    // no rollout is settled at once and the row waits for the next fetch)
    while (!alive && pst == 3) {
      const long long it = pit;
      pst = 0;
      item = it;
      v = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] = ph[k];
      pm = positive_mask(h, M.m);
      if (kExpand) {
        s.pos[0] = pf[0];
        s.pos[1] = 0u;
        s.good = pf[1];
        s.sampled = pf[2];
        s.scen = pf[3];
        const uint32_t meta = pf[5];
        J = src.jobs + pf[6];
        slot = meta & 0xFFFFFFu;
        t0 = (int)(meta >> 24) + 1;
        M.observe(h, pm, (int)pfa + (int)(slot / pcap), pkey);
        u = M.terminal(s) ? 0.0f : ((t0 >= M.D) ? M.tail(s) : M.upper(s));
      } else {
        s.pos[0] = pf[0];
        s.pos[1] = 0u;  // one robot (as RSModel<1>::load)
        s.good = pf[2];
        s.sampled = pf[3];
        s.scen = pf[4];
        t0 = src.start_depth;
      }
      t = t0;
      if (t < M.D && !M.terminal(s)) {
        alive = true;
      } else {
        if (!M.terminal(s)) v = __fadd_rn(v, __fmul_rn(S.c.G[M.D - t0], M.tail(s)));
        if (kExpand) {
          sum_add(J->u_sum + slot, to_fixed(u));
          sum_add(J->l_sum + slot, to_fixed(v));
        } else {
          src.value[it] = v;
        }
      }
    }
    // features of the row's state and counters, BF16 into the tile's A operand
    if (alive) {
      write_features(S.x[tile], row, M.m, S.c.rock_xy, s.pos[0], s.sampled, h, T);
    } else {
#pragma unroll
      for (int c = 0; c < kMlpIn / 8; ++c)
        *reinterpret_cast<uint4*>(S.x[tile] + kmajor_off(row, 8 * c, kMlpIn)) = make_uint4(0u, 0u, 0u, 0u);
    }
    fence_async_smem();
    if (!tile_or(bar, alive || pst != 4)) break;
    // layer 1; meanwhile the row's allowed actions, the heuristic's action
    // and the next fetch stage
    if (issuer) issue_layer1(S.W, sx, tbase, mbar);
    if (alive) {
      allow = learned_allow(S.c, M.n, M.m, s.pos[0], s.sampled, h) | (1u << na);
      heur = M.policy(s, pm);
    }
    advance();
    if (!wait_layer()) {
      failed = true;
      break;
    }
    epilogue1_inplace(trow, S.W.b1);
    fence_before_sync();
    tile_sync(bar);
    // layer 2, first half; its BF16 outputs wait in registers
    if (issuer) issue_layer2_half(S.W, tbase, tbase + 128, 0, mbar);
    if (!wait_layer()) {
      failed = true;
      break;
    }
    uint32_t h2a[64];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      float acc[64];
      tmem_ld64(trow + 128 + 64 * c, acc);
      relu_pack32(*reinterpret_cast<const float(*)[32]>(acc), S.W.b2 + 64 * c, h2a + 32 * c);
      relu_pack32(*reinterpret_cast<const float(*)[32]>(acc + 32), S.W.b2 + 64 * c + 32, h2a + 32 * c + 16);
    }
    fence_before_sync();
    tile_sync(bar);
    // layer 2, second half; then H2 replaces H1 in columns 0..127
    if (issuer) issue_layer2_half(S.W, tbase, tbase + 128, 1, mbar);
    if (!wait_layer()) {
      failed = true;
      break;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) tmem_st16p(trow + 16 * c, h2a + 16 * c);
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      float acc[64];
      uint32_t packed[32];
      tmem_ld64(trow + 128 + 64 * c, acc);
      relu_pack32(*reinterpret_cast<const float(*)[32]>(acc), S.W.b2 + 128 + 64 * c, packed);
      relu_pack32(*reinterpret_cast<const float(*)[32]>(acc + 32), S.W.b2 + 128 + 64 * c + 32, packed + 16);
      tmem_st16p(trow + 64 + 32 * c, packed);
      tmem_st16p(trow + 64 + 32 * c + 16, packed + 16);
    }
    tmem_wait_st();
    fence_before_sync();
    tile_sync(bar);
    // layer 3: the logits
    if (issuer) issue_layer3(S.W, tbase, tbase + 128, mbar);
    if (!wait_layer()) {
      failed = true;
      break;
    }
    float lg[32];
    tmem_ld32(trow + 128, lg);
    fence_before_sync();
    if (alive) {
      // argmax over the allowed actions and defer (column na), lowest index on ties
      const int best = masked_argmax(lg, S.W.b3, allow, na);
      const int a = best == na ? heur : best;
      if (!kExpand && src.log) src.log[(size_t)item * M.D + (t - t0)] = a;
      if (!kExpand && src.logits) {
        float4* o = reinterpret_cast<float4*>(src.logits + ((size_t)item * M.D + (t - t0)) * kMlpOut);
#pragma unroll
        for (int q = 0; q < kMlpOut / 4; ++q)
          o[q] = make_float4(__fadd_rn(lg[4 * q], S.W.b3[4 * q]), __fadd_rn(lg[4 * q + 1], S.W.b3[4 * q + 1]),
                             __fadd_rn(lg[4 * q + 2], S.W.b3[4 * q + 2]), __fadd_rn(lg[4 * q + 3], S.W.b3[4 * q + 3]));
      }
      uint64_t key;
      float r = M.step(s, a, t, key);
      M.observe(h, pm, a, key);
      if (r != 0.0f) v = __fadd_rn(v, __fmul_rn(S.c.G[t - t0], r));
      t += 1;
      steps += 1;
      if (M.terminal(s) || t >= M.D) {
        if (!M.terminal(s)) v = __fadd_rn(v, __fmul_rn(S.c.G[M.D - t0], M.tail(s)));
        if (kExpand) {
          sum_add(J->u_sum + slot, to_fixed(u));
          sum_add(J->l_sum + slot, to_fixed(v));
        } else {
          src.value[item] = v;
        }
        alive = false;
      }
    }
  }
  // a tile whose layer timed out reports it and waits (bounded) for its MMAs
  // in flight before the tensor memory is freed
  if (failed && issuer) {
    report(work, kStatusTimeout);
    mbar_wait(mbar, phase ^ 1u);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base), "r"(kTmemCols)
                 : "memory");
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
  // the whole opt-in shared memory: the pair table's size depends on the map
  // side, which the kernel reads from the model (one CTA per SM either way)
  const size_t smem = kTcSmemMax;
  cudaError_t e = cudaFuncSetAttribute(rs_rollout_tc_kernel<kExpand>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (int)std::max(1LL, std::min<long long>((total + 2 * kRows - 1) / (2 * kRows), (long long)num_sms));
  rs_rollout_tc_kernel<kExpand><<<grid, kThreads, smem, st>>>(gm, work, policy, src, plan_step);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rs_rollout_mlp_items(const DevModel* gm, DevWork* work, const dsp_leaf_job* jobs,
                                        uint32_t* item_buf, long long total_items, unsigned int* counter,
                                        const void* policy, uint32_t plan_step, int num_sms, cudaStream_t st) {
  ItemSource src{};
  src.jobs = jobs;
  src.items = Items<1>{item_buf, total_items, true};
  src.next = counter;
  return launch_mlp<true>(gm, work, (const uint8_t*)policy, src, plan_step, num_sms, total_items, st);
}

// The hand-written default policy of Rock Sample per state (the joint
// action for two robots) and, for one robot, the learned policy's allowed
// actions with the defer column.
template <int R>
__global__ void rs_policy_kernel(const DevModel* __restrict__ gm, const uint32_t* __restrict__ block, int cap,
                                 int count, const int8_t* __restrict__ hist, int32_t* __restrict__ actions,
                                 uint32_t* __restrict__ allowed) {
  __shared__ RSShared c;
  load_rs_consts(c, gm);
  __syncthreads();
  const RSModel<R> M = make_rs<R>(gm, &c, 0u);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const RSS s = M.load(block, cap, i);
  uint32_t h[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) h[k] = hist ? *reinterpret_cast<const uint32_t*>(hist + 32 * (size_t)i + 4 * k) : 0u;
  actions[i] = M.policy(s, positive_mask(h, M.m));
  if (R == 1 && allowed)
    allowed[i] = learned_allow(c, M.n, M.m, s.pos[0], s.sampled, h) | (1u << gm->num_actions);
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
  if (m->host->kind == DSP_MODEL_MULTIGRID)
    return fail(DSP_E_UNSUPPORTED, "dsp_features: one-robot Rock Sample or the car");
  const bool car = m->host->kind == DSP_MODEL_CAR;
  if (count < 0 || cap < count || (count > 0 && (!block || (!car && !hist) || !out)))
    return fail(DSP_E_INVALID, "dsp_features: bad buffers");
  if (((uintptr_t)out & 15) != 0) return fail(DSP_E_INVALID, "dsp_features: out must be 16-byte aligned");
  if (count == 0) return DSP_OK;
  if (car) {
    cudaError_t e = launch_car_features(m, block, cap, count, out, (cudaStream_t)stream);
    return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_features");
  }
  features_kernel<<<(count + 255) / 256, 256, 0, (cudaStream_t)stream>>>(m->dmodel, block, cap, count, hist, out);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_features");
}

dsp_status dsp_default_policy(const dsp_model* m, const uint32_t* block, int32_t cap, int32_t count,
                              const int8_t* hist, int32_t* actions, uint32_t* allowed, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_default_policy: model is NULL");
  const int kind = m->host->kind;
  if (count < 0 || cap < count || (count > 0 && (!actions || (kind != DSP_MODEL_NAV && !block) ||
                                                 (kind == DSP_MODEL_NAV && !hist))))
    return fail(DSP_E_INVALID, "dsp_default_policy: bad buffers");
  if (allowed && kind != DSP_MODEL_GRID)
    return fail(DSP_E_UNSUPPORTED, "dsp_default_policy: allowed actions are one-robot Rock Sample's");
  if (count == 0) return DSP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (kind == DSP_MODEL_CAR) {
    e = launch_car_policy(m, block, cap, count, actions, st);
  } else if (kind == DSP_MODEL_NAV) {
    e = launch_nav_policy(m->dmodel, hist, count, actions, st);
  } else if (kind == DSP_MODEL_GRID) {
    rs_policy_kernel<1><<<(count + 255) / 256, 256, 0, st>>>(m->dmodel, block, cap, count, hist, actions, allowed);
    e = cudaGetLastError();
  } else {
    rs_policy_kernel<2><<<(count + 255) / 256, 256, 0, st>>>(m->dmodel, block, cap, count, hist, actions, nullptr);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_default_policy");
}

dsp_status dsp_set_policy(dsp_model* m, const dsp_mlp* mlp) {
  if (!m) return fail(DSP_E_INVALID, "dsp_set_policy: model is NULL");
  if (mlp == nullptr) {
    m->policy_on = false;
    return DSP_OK;
  }
  if (m->host->kind == DSP_MODEL_MULTIGRID || m->host->kind == DSP_MODEL_NAV)
    return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: the learned policy serves one-robot Rock Sample and the car");
  if (m->host->num_actions + 1 > kMlpOut)
    return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: more than 31 actions (the network's last used logit defers)");
  if (m->host->kind == DSP_MODEL_GRID && m->host->m > 15)
    return fail(DSP_E_UNSUPPORTED, "dsp_set_policy: features hold 15 rocks");
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
                              float* logits, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_rollout_logged: model is NULL");
  if (!m->policy_on) return fail(DSP_E_UNSUPPORTED, "dsp_rollout_logged: no learned policy set");
  if (count < 0 || cap < count || !block || !value) return fail(DSP_E_INVALID, "dsp_rollout_logged: bad buffers");
  if (((uintptr_t)logits & 15) != 0) return fail(DSP_E_INVALID, "dsp_rollout_logged: logits must be 16-byte aligned");
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
    src.logits = logits;
    src.next = counter;
    if (m->host->kind == DSP_MODEL_CAR)
      e = launch_car_rollout_logged(m, block, cap, count, start_depth, value, actions, logits, counter, st);
    else
      e = launch_mlp<false>(m->dmodel, m->dwork, (const uint8_t*)m->policy, src, m->plan_step, m->num_sms, count,
                            st);
  }
  if (counter) cudaFreeAsync(counter, st);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_rollout_logged");
}

}  // extern "C"
