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

#include "kernels.cuh"
#include "mlp.cuh"
#include "model.hpp"
#include "rs_common.cuh"

struct dsp_mlp;  // training object (mlp_train.cu); its FP32 master is read here
extern "C" dsp_status dsp_mlp_get_weights(const dsp_mlp* mlp, float* host_params);

namespace dsp {
namespace {

constexpr int kRows = 128;       // scenarios per CTA: the MMA's M
constexpr int kThreads = 256;    // two threads per row: warps w and w + 4 reach TMEM lanes 32w .. 32w + 31
                                 // and split the hidden epilogues' columns; the first owns the scenario
// device policy buffer: transposed BF16 weights [n][k], FP32 biases
constexpr size_t kPolW1 = 0;
constexpr size_t kPolW2 = kPolW1 + (size_t)kMlpHid * kMlpIn * 2;
constexpr size_t kPolW3 = kPolW2 + (size_t)kMlpHid * kMlpHid * 2;
constexpr size_t kPolB1 = kPolW3 + (size_t)kMlpOut * kMlpHid * 2;
constexpr size_t kPolB2 = kPolB1 + kMlpHid * 4;
constexpr size_t kPolB3 = kPolB2 + kMlpHid * 4;
constexpr size_t kPolBytes = kPolB3 + kMlpOut * 4;

// Tensor memory of a CTA (all 512 columns; the kernel's shared memory keeps
// one CTA per SM): layer-1 and layer-2 accumulators share columns 0..255
// (FP32, row r in lane r), the hidden activations of the next layer's A
// operand take 256..383 (BF16 pairs along K), the logits 384..415.
constexpr int kDxy = 63;          // rock offsets -31..31 (map side <= 32)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD = 0;
constexpr uint32_t kColH = 256;
constexpr uint32_t kColL = 384;

// Shared memory. Matrices are stored in the canonical K-major layout without
// swizzle that tcgen05 descriptors address: 8 rows x 16 bytes form a core
// matrix (128 contiguous bytes), core matrices along K lie 128 bytes apart
// (leading byte offset) and 8-row groups lie K/8 * 128 bytes apart (stride
// byte offset).
struct TcSmem {
  uint8_t w1[kMlpHid * kMlpIn * 2];   // B of layer 1: N = 256, K = 64
  uint8_t w2[kMlpHid * kMlpHid * 2];  // B of layer 2: N = 256, K = 256
  uint8_t w3[kMlpOut * kMlpHid * 2];  // B of layer 3: N = 32, K = 256
  uint8_t x[kRows * kMlpIn * 2];      // A of layer 1: M = 128, K = 64 (features)
  float b1[kMlpHid], b2[kMlpHid], b3[kMlpOut];
  uint32_t fdxy[kDxy * kDxy];          // BF16 pair ((float)dx / n, (float)dy / n), dx, dy in -31..31
  uint32_t fcs[14];                    // BF16 pair (clamp(c) / 3, sampled), c in -3..3
  RSShared c;
  unsigned long long mbar;            // completion of each layer's MMAs
  uint32_t tmem_base;
};

__device__ __forceinline__ uint32_t kmajor_off(int row, int k, int K) {
  return (uint32_t)((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all in 16-byte units), descriptor version 1, base offset 0, no
// swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ uint64_t global_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with this parity to complete, for at most 2 s.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  if (mbar_try(mbar, parity)) return true;
  const uint64_t t0 = global_timer();
  while (!mbar_try(mbar, parity))
    if (global_timer() - t0 > 2000000000ull) return false;
  return true;
}

// 32 FP32 columns of the warp's 32 lanes (one row per thread), waited for.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 FP32 columns of the warp's 32 lanes, waited for.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 columns of 32-bit words into the warp's 32 lanes.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::
          "r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Hidden layer epilogue of one row, columns [128 half, 128 half + 128):
// ReLU(accumulator + bias), rounded to BF16, written back as the next layer's
// A operand.
__device__ __forceinline__ void hidden_epilogue(uint32_t trow, const float* bias, int half) {
#pragma unroll 1
  for (int c = 2 * half; c < 2 * half + 2; ++c) {
    float acc[64];
    tmem_ld64(trow + kColD + 64 * c, acc);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      uint32_t packed[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int col = 64 * c + 32 * q + 2 * j;
        float lo = fmaxf(__fadd_rn(acc[32 * q + 2 * j], bias[col]), 0.0f);
        float hi = fmaxf(__fadd_rn(acc[32 * q + 2 * j + 1], bias[col + 1]), 0.0f);
        packed[j] = pack_bf16(lo, hi);
      }
      tmem_st16(trow + kColH + 32 * c + 16 * q, packed);
    }
  }
  tmem_wait_st();
}

// The row's features (the feature map of rs_features, same arithmetic) as
// BF16 pairs straight into the layer-1 A tile: pair 0 = (x/n, y/n), pairs
// 1 + 2r = ((rock x - x)/n, (rock y - y)/n), 2 + 2r = (clamp(c_r)/3, sampled_r),
// zero beyond 1 + 2m. Fully unrolled, so nothing goes through local memory.
// The BF16 feature pairs that depend on one rock, tabulated per CTA with the
// arithmetic of rs_features: fdxy[(dx + 31) * 63 + dy + 31] for the offset
// pair and fcs[(c + 3) * 2 + sampled] for the counter/sampled pair.
__device__ __forceinline__ void build_feature_tables(uint32_t* fdxy, uint32_t* fcs, int n) {
  const float inv_n = 1.0f / (float)n;
  const float third = 1.0f / 3.0f;
  for (int i = threadIdx.x; i < kDxy * kDxy; i += blockDim.x) {
    const int dx = i / kDxy - 31, dy = i % kDxy - 31;
    fdxy[i] = pack_bf16((float)dx * inv_n, (float)dy * inv_n);
  }
  for (int i = threadIdx.x; i < 14; i += blockDim.x) fcs[i] = pack_bf16((float)(i / 2 - 3) * third, (i & 1) ? 1.0f : 0.0f);
}

__device__ __forceinline__ void write_features(uint8_t* xs, int row, int n, int m, const int* rock_xy, uint32_t pos,
                                               uint32_t sampled, const uint32_t (&h)[8], const uint32_t* fdxy,
                                               const uint32_t* fcs) {
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
      pr[1 + 2 * r] = fdxy[((rxy & 0xFF) - x + 31) * kDxy + ((rxy >> 8) - y + 31)];
      pr[2 + 2 * r] = fcs[(c + 3) * 2 + (int)((sampled >> r) & 1u)];
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
  unsigned int* next;  // item counter
};

// A CTA keeps 128 live scenarios (rows, one per thread) and advances them one
// step at a time: each row writes its features (BF16) into the layer-1 A tile
// in shared memory, one elected thread issues the three layers as tcgen05.mma
// (M = 128, BF16 in, FP32 accumulators in tensor memory, weights resident in
// shared memory as the B operands, the hidden activations fed back through
// tensor memory as the A operand), and after each layer's completion every
// thread reads its own row from tensor memory: bias + ReLU + BF16 for the
// hidden layers, then the masked argmax of its logits. A row whose scenario
// ends adds its value to its child and takes the next item at once.
template <bool kExpand>
__global__ void __launch_bounds__(kThreads, 1) rs_rollout_tc_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                    const uint8_t* __restrict__ policy,
                                                                    ItemSource src, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TcSmem& S = *reinterpret_cast<TcSmem*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, half = tid >> 7;
  const bool owner = half == 0;  // the thread that holds the row's scenario
  load_rs_consts(S.c, gm);
  {
    const uint4* w1 = reinterpret_cast<const uint4*>(policy + kPolW1);
    const uint4* w2 = reinterpret_cast<const uint4*>(policy + kPolW2);
    const uint4* w3 = reinterpret_cast<const uint4*>(policy + kPolW3);
    for (int i = tid; i < kMlpHid * kMlpIn / 8; i += kThreads) {
      const int n = i / (kMlpIn / 8), c = i % (kMlpIn / 8);
      *reinterpret_cast<uint4*>(S.w1 + kmajor_off(n, 8 * c, kMlpIn)) = w1[i];
    }
    for (int i = tid; i < kMlpHid * kMlpHid / 8; i += kThreads) {
      const int n = i / (kMlpHid / 8), c = i % (kMlpHid / 8);
      *reinterpret_cast<uint4*>(S.w2 + kmajor_off(n, 8 * c, kMlpHid)) = w2[i];
    }
    for (int i = tid; i < kMlpOut * kMlpHid / 8; i += kThreads) {
      const int n = i / (kMlpHid / 8), c = i % (kMlpHid / 8);
      *reinterpret_cast<uint4*>(S.w3 + kmajor_off(n, 8 * c, kMlpHid)) = w3[i];
    }
    const float* b1 = reinterpret_cast<const float*>(policy + kPolB1);
    const float* b2 = reinterpret_cast<const float*>(policy + kPolB2);
    const float* b3 = reinterpret_cast<const float*>(policy + kPolB3);
    for (int i = tid; i < kMlpHid; i += kThreads) {
      S.b1[i] = b1[i];
      S.b2[i] = b2[i];
    }
    for (int i = tid; i < kMlpOut; i += kThreads) S.b3[i] = b3[i];
  }
  build_feature_tables(S.fdxy, S.fcs, gm->n);
  const uint32_t mbar = smem_u32(&S.mbar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
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
  const uint32_t tmem = S.tmem_base;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lanes
  const uint32_t sx = smem_u32(S.x), sw1 = smem_u32(S.w1), sw2 = smem_u32(S.w2), sw3 = smem_u32(S.w3);
  constexpr uint32_t kId1 = idesc_bf16(kRows, kMlpHid), kId3 = idesc_bf16(kRows, kMlpOut);

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
  if (owner) {
    advance();
    advance();
    advance();
  }
  while (true) {
    // rows whose scenario ended take the fetched item (an item that needs no
    // rollout is settled at once and the row waits for the next fetch)
    while (owner && !alive && pst == 3) {
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
          atomicAdd((unsigned long long*)(J->u_sum + slot), (unsigned long long)to_fixed(u));
          atomicAdd((unsigned long long*)(J->l_sum + slot), (unsigned long long)to_fixed(v));
        } else {
          src.value[it] = v;
        }
      }
    }
    // features of the row's state and counters, BF16 into the A tile
    if (owner) {
      if (alive) {
        write_features(S.x, tid, M.n, M.m, S.c.rock_xy, s.pos[0], s.sampled, h, S.fdxy, S.fcs);
      } else {
#pragma unroll
        for (int c = 0; c < kMlpIn / 8; ++c)
          *reinterpret_cast<uint4*>(S.x + kmajor_off(tid, 8 * c, kMlpIn)) = make_uint4(0u, 0u, 0u, 0u);
      }
    }
    fence_async_smem();
    if (!__syncthreads_or((alive || (owner && pst != 4)) ? 1 : 0)) break;
    // layer 1: D = X W1^T, four K = 16 steps
    if (tid == 0) {
      fence_after_sync();
#pragma unroll
      for (int k = 0; k < kMlpIn / 16; ++k)
        mma_ss(tmem + kColD, smem_desc(sx + 256 * k, 128, (kMlpIn / 8) * 128),
               smem_desc(sw1 + 256 * k, 128, (kMlpIn / 8) * 128), kId1, k > 0);
      mma_commit(mbar);
    }
    // while layer 1 runs: the row's allowed actions, the heuristic's action
    // and the next fetch stage
    if (owner) {
      if (alive) {
        allow = learned_allow(S.c, M.n, M.m, s.pos[0], s.sampled, h) | (1u << na);
        heur = M.policy(s, pm);
      }
      advance();
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) {
      failed = true;
      break;
    }
    phase ^= 1u;
    fence_after_sync();
    hidden_epilogue(trow, S.b1, half);
    fence_before_sync();
    __syncthreads();
    // layer 2: D = H1 W2^T, A from tensor memory, sixteen K = 16 steps
    if (tid == 0) {
      fence_after_sync();
#pragma unroll 4
      for (int k = 0; k < kMlpHid / 16; ++k)
        mma_ts(tmem + kColD, tmem + kColH + 8 * k, smem_desc(sw2 + 256 * k, 128, (kMlpHid / 8) * 128), kId1, k > 0);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) {
      failed = true;
      break;
    }
    phase ^= 1u;
    fence_after_sync();
    hidden_epilogue(trow, S.b2, half);
    fence_before_sync();
    __syncthreads();
    // layer 3: logits = H2 W3^T
    if (tid == 0) {
      fence_after_sync();
#pragma unroll 4
      for (int k = 0; k < kMlpHid / 16; ++k)
        mma_ts(tmem + kColL, tmem + kColH + 8 * k, smem_desc(sw3 + 256 * k, 128, (kMlpHid / 8) * 128), kId3, k > 0);
      mma_commit(mbar);
    }
    if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) {
      failed = true;
      break;
    }
    phase ^= 1u;
    fence_after_sync();
    float lg[32];
    if (owner) tmem_ld32(trow + kColL, lg);
    fence_before_sync();
    if (alive) {
      // argmax over the allowed actions and defer (column na), lowest index on ties
      float xv[32];
      int xi[32];
#pragma unroll
      for (int col = 0; col < 32; ++col) {
        const bool ok = col <= na && ((allow >> col) & 1u);
        xv[col] = ok ? __fadd_rn(lg[col], S.b3[col]) : 0.0f;
        xi[col] = ok ? col : 0x7FFF;
      }
      // pairwise tournament; the right entry wins only if strictly larger,
      // so the lowest index wins ties
#pragma unroll
      for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
        for (int k = 0; k < w; ++k) {
          const bool take = xi[k + w] != 0x7FFF && (xi[k] == 0x7FFF || xv[k + w] > xv[k]);
          xv[k] = take ? xv[k + w] : xv[k];
          xi[k] = take ? xi[k + w] : xi[k];
        }
      const int best = xi[0];
      const int a = best == na ? heur : best;
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
  if (failed) {
    // a layer did not complete in time: report, give the MMAs in flight one
    // more bounded wait, then free the tensor memory
    if (tid == 0) report(work, kStatusTimeout);
    mbar_wait(mbar, phase);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
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
  size_t smem = sizeof(TcSmem);
  cudaError_t e = cudaFuncSetAttribute(rs_rollout_tc_kernel<kExpand>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  int grid = (int)std::max(1LL, std::min<long long>((total + kRows - 1) / kRows, (long long)num_sms));
  rs_rollout_tc_kernel<kExpand><<<grid, kThreads, smem, st>>>(gm, work, policy, src, plan_step);
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
