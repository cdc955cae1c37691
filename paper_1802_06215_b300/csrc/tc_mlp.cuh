// Building blocks of the learned default policy on the fifth-generation
// tensor cores, shared by the Rock Sample and car rollout kernels: the
// policy's weights in shared memory as tcgen05 B operands, the three layers
// of the network over a 128-row tile (M = 128, BF16 inputs, FP32
// accumulators in tensor memory, the hidden activations fed back through
// tensor memory as the next A operand) and the primitives they use.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"
#include "mlp.cuh"

namespace dsp {
namespace tc {

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
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColD = 0;
constexpr uint32_t kColH = 256;
constexpr uint32_t kColL = 384;

// The policy in shared memory. Matrices are stored in the canonical K-major
// layout without swizzle that tcgen05 descriptors address: 8 rows x 16 bytes
// form a core matrix (128 contiguous bytes), core matrices along K lie 128
// bytes apart (leading byte offset) and 8-row groups lie K/8 * 128 bytes
// apart (stride byte offset).
struct Weights {
  uint8_t w1[kMlpHid * kMlpIn * 2];   // B of layer 1: N = 256, K = 64
  uint8_t w2[kMlpHid * kMlpHid * 2];  // B of layer 2: N = 256, K = 256
  uint8_t w3[kMlpOut * kMlpHid * 2];  // B of layer 3: N = 32, K = 256
  float b1[kMlpHid], b2[kMlpHid], b3[kMlpOut];
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


// Copies the device policy buffer into shared memory in the descriptor layout
// (all threads of the CTA).
__device__ __forceinline__ void load_weights(Weights& W, const uint8_t* __restrict__ policy) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const uint4* w1 = reinterpret_cast<const uint4*>(policy + kPolW1);
  const uint4* w2 = reinterpret_cast<const uint4*>(policy + kPolW2);
  const uint4* w3 = reinterpret_cast<const uint4*>(policy + kPolW3);
  for (int i = tid; i < kMlpHid * kMlpIn / 8; i += nt) {
    const int n = i / (kMlpIn / 8), c = i % (kMlpIn / 8);
    *reinterpret_cast<uint4*>(W.w1 + kmajor_off(n, 8 * c, kMlpIn)) = w1[i];
  }
  for (int i = tid; i < kMlpHid * kMlpHid / 8; i += nt) {
    const int n = i / (kMlpHid / 8), c = i % (kMlpHid / 8);
    *reinterpret_cast<uint4*>(W.w2 + kmajor_off(n, 8 * c, kMlpHid)) = w2[i];
  }
  for (int i = tid; i < kMlpOut * kMlpHid / 8; i += nt) {
    const int n = i / (kMlpHid / 8), c = i % (kMlpHid / 8);
    *reinterpret_cast<uint4*>(W.w3 + kmajor_off(n, 8 * c, kMlpHid)) = w3[i];
  }
  const float* b1 = reinterpret_cast<const float*>(policy + kPolB1);
  const float* b2 = reinterpret_cast<const float*>(policy + kPolB2);
  const float* b3 = reinterpret_cast<const float*>(policy + kPolB3);
  for (int i = tid; i < kMlpHid; i += nt) {
    W.b1[i] = b1[i];
    W.b2[i] = b2[i];
  }
  for (int i = tid; i < kMlpOut; i += nt) W.b3[i] = b3[i];
}

// The mbarrier (thread 0) and the CTA's 512 tensor-memory columns (warp 0);
// the caller synchronises afterwards and reads the column base.
__device__ __forceinline__ void setup(uint32_t mbar, uint32_t tmem_slot) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tmem_slot), "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
}

// Frees the tensor memory after a last bounded wait if a layer timed out.
__device__ __forceinline__ void teardown(uint32_t tmem, uint32_t mbar, uint32_t phase, bool failed, DevWork* work) {
  if (failed) {
    if (threadIdx.x == 0) report(work, kStatusTimeout);
    mbar_wait(mbar, phase);
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// The three layers over the 128-row A tile at sx (written, fenced and
// synchronised by the caller). Thread 0 issues each layer and commits to the
// mbarrier; every thread waits (bounded), and the two threads of a row (half
// 0 and 1) split the hidden epilogues. during_l1() runs while layer 1 is in
// flight. Returns false if a layer did not complete in time; on success the
// logits are in columns kColL.. of tensor memory (not yet read).
template <class F>
__device__ __forceinline__ bool run_layers(const Weights& W, uint32_t sx, uint32_t tmem, uint32_t trow, uint32_t mbar,
                                           uint32_t& phase, int half, F&& during_l1) {
  const int tid = threadIdx.x;
  const uint32_t sw1 = smem_u32(W.w1), sw2 = smem_u32(W.w2), sw3 = smem_u32(W.w3);
  constexpr uint32_t kId1 = idesc_bf16(kRows, kMlpHid), kId3 = idesc_bf16(kRows, kMlpOut);
  // layer 1: D = X W1^T, four K = 16 steps
  if (tid == 0) {
    fence_after_sync();
#pragma unroll
    for (int k = 0; k < kMlpIn / 16; ++k)
      mma_ss(tmem + kColD, smem_desc(sx + 256 * k, 128, (kMlpIn / 8) * 128),
             smem_desc(sw1 + 256 * k, 128, (kMlpIn / 8) * 128), kId1, k > 0);
    mma_commit(mbar);
  }
  during_l1();
  if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) return false;
  phase ^= 1u;
  fence_after_sync();
  hidden_epilogue(trow, W.b1, half);
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
  if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) return false;
  phase ^= 1u;
  fence_after_sync();
  hidden_epilogue(trow, W.b2, half);
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
  if (!__syncthreads_and(mbar_wait(mbar, phase) ? 1 : 0)) return false;
  phase ^= 1u;
  fence_after_sync();
  return true;
}

// Argmax over the columns whose bit is set in `allow` (column na is "defer"),
// lowest index on ties, by a pairwise tournament: the right entry wins only
// if strictly larger. Returns the column.
__device__ __forceinline__ int masked_argmax(const float (&lg)[32], const float* b3, uint32_t allow, int na) {
  float xv[32];
  int xi[32];
#pragma unroll
  for (int col = 0; col < 32; ++col) {
    const bool ok = col <= na && ((allow >> col) & 1u);
    xv[col] = ok ? __fadd_rn(lg[col], b3[col]) : 0.0f;
    xi[col] = ok ? col : 0x7FFF;
  }
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1)
#pragma unroll
    for (int k = 0; k < w; ++k) {
      const bool take = xi[k + w] != 0x7FFF && (xi[k] == 0x7FFF || xv[k + w] > xv[k]);
      xv[k] = take ? xv[k + w] : xv[k];
      xi[k] = take ? xi[k + w] : xi[k];
    }
  return xi[0];
}

// ---------------------------------------------------------------------------
// Two tiles per CTA. A CTA of 256 threads holds two 128-row tiles, one per
// warpgroup (warps 0-3 tile 0, warps 4-7 tile 1; every thread owns one row
// of its tile and reaches that row's TMEM lane), each with 256 of the 512
// tensor-memory columns. While one tile runs its epilogues and its scalar
// step (argmax, g, features), the tensor pipe works on the other's layers.
// A tile's 256 columns (relative to its base):
//  - layer 1: the FP32 accumulator in 0..255; its epilogue packs the BF16
//    activations H1 in place into 0..127 (chunk c of 32 columns goes to
//    16c.., columns already read);
//  - layer 2 in two N = 128 halves, each accumulating in 128..255 with H1 in
//    0..127 as the A operand; the first half's BF16 outputs wait in
//    registers while the second half runs, then H2 fills 0..127 (H1 is dead);
//  - layer 3: the logits in 128..159 with H2 as the A operand.
constexpr uint32_t kTileCols = 256;

// Named barrier of one tile's 128 threads (ids 1 and 2; 0 is __syncthreads).
// The threads of a warp may reach it apart (after a bounded spin on an
// mbarrier, or a branch taken by one thread), so the barriers are the
// non-aligned forms, with the warp reconverged before and after (the
// tensor-memory loads and stores that follow need the whole warp).
__device__ __forceinline__ void tile_sync(int id) {
  __syncwarp();
  asm volatile("barrier.cta.sync %0, 128;" ::"r"(id) : "memory");
  __syncwarp();
}
__device__ __forceinline__ bool tile_and(int id, bool p) {
  uint32_t r;
  __syncwarp();
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbarrier.cta.red.and.pred q, %2, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id)
      : "memory");
  __syncwarp();
  return r != 0;
}
__device__ __forceinline__ bool tile_or(int id, bool p) {
  uint32_t r;
  __syncwarp();
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbarrier.cta.red.or.pred q, %2, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p), "r"(id)
      : "memory");
  __syncwarp();
  return r != 0;
}

// 16 columns of 32-bit words from r[0..15] into the warp's 32 lanes.
__device__ __forceinline__ void tmem_st16p(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::
          "r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

// Two FP32 values rounded to a BF16 pair (lo in the low half) with negative
// results clamped to zero, in one conversion: the same values as rounding
// max(x, 0), up to the sign of a zero.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// ReLU(accumulator + bias) of 32 FP32 columns, rounded to 16 BF16 pairs.
// (Reading the bias four floats at a time was 4 % slower in the learned
// rollout on B300.)
__device__ __forceinline__ void relu_pack32(const float (&acc)[32], const float* bias, uint32_t* out) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    out[j] = pack_bf16_relu(__fadd_rn(acc[2 * j], bias[2 * j]), __fadd_rn(acc[2 * j + 1], bias[2 * j + 1]));
}

// Layer 1 of a tile (issuing thread): D (256 FP32 columns at d) = X W1^T,
// X the tile's features in shared memory at sx; commits to mbar.
__device__ __forceinline__ void issue_layer1(const Weights& W, uint32_t sx, uint32_t d, uint32_t mbar) {
  constexpr uint32_t kId = idesc_bf16(kRows, kMlpHid);
  const uint32_t sw1 = smem_u32(W.w1);
  fence_after_sync();
#pragma unroll
  for (int k = 0; k < kMlpIn / 16; ++k)
    mma_ss(d, smem_desc(sx + 256 * k, 128, (kMlpIn / 8) * 128), smem_desc(sw1 + 256 * k, 128, (kMlpIn / 8) * 128),
           kId, k > 0);
  mma_commit(mbar);
}

// Half h of layer 2 (issuing thread): D (128 FP32 columns at d) = H1 (BF16
// pairs in tensor memory at a) times rows 128h .. 128h + 127 of W2, transposed.
__device__ __forceinline__ void issue_layer2_half(const Weights& W, uint32_t a, uint32_t d, int h, uint32_t mbar) {
  constexpr uint32_t kId = idesc_bf16(kRows, 128);
  const uint32_t sw2 = smem_u32(W.w2) + (uint32_t)h * (128 / 8) * (kMlpHid / 8) * 128;
  fence_after_sync();
#pragma unroll 4
  for (int k = 0; k < kMlpHid / 16; ++k)
    mma_ts(d, a + 8 * k, smem_desc(sw2 + 256 * k, 128, (kMlpHid / 8) * 128), kId, k > 0);
  mma_commit(mbar);
}

// Layer 3 (issuing thread): logits (32 FP32 columns at d) = H2 (at a) W3^T.
__device__ __forceinline__ void issue_layer3(const Weights& W, uint32_t a, uint32_t d, uint32_t mbar) {
  constexpr uint32_t kId = idesc_bf16(kRows, kMlpOut);
  const uint32_t sw3 = smem_u32(W.w3);
  fence_after_sync();
#pragma unroll 4
  for (int k = 0; k < kMlpHid / 16; ++k)
    mma_ts(d, a + 8 * k, smem_desc(sw3 + 256 * k, 128, (kMlpHid / 8) * 128), kId, k > 0);
  mma_commit(mbar);
}

// Layer 1's epilogue for the thread's row (trow = the tile's base column on
// the row's lane): H1 = BF16(ReLU(D + b1)) packed in place into columns
// 0..127 (chunk c of 64 accumulator columns to 32c..32c+31, columns the
// thread has already read). 64 columns per load: one wait per 64.
__device__ __forceinline__ void epilogue1_inplace(uint32_t trow, const float* b1) {
#pragma unroll 1
  for (int c = 0; c < kMlpHid / 64; ++c) {
    float acc[64];
    uint32_t packed[32];
    tmem_ld64(trow + 64 * c, acc);
    relu_pack32(*reinterpret_cast<const float(*)[32]>(acc), b1 + 64 * c, packed);
    relu_pack32(*reinterpret_cast<const float(*)[32]>(acc + 32), b1 + 64 * c + 32, packed + 16);
    tmem_st16p(trow + 32 * c, packed);
    tmem_st16p(trow + 32 * c + 16, packed + 16);
  }
  tmem_wait_st();
}

}  // namespace tc
}  // namespace dsp
