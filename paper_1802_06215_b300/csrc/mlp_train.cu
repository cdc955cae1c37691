// Training of the learned default policy pi0: softmax cross-entropy on
// (state features, action label) pairs with this library's own kernels: BF16
// GEMMs on the fifth-generation tensor cores (tcgen05.mma, FP32 accumulators
// in tensor memory) with fused epilogues, softmax cross-entropy, column sums
// for the bias gradients, and
// Adam on FP32 master weights with BF16 copies for the next step. The labels
// are the caller's: the shipped Rock Sample weights were trained first on
// the plain planner's chosen actions (imitation, "defer" where it chose the
// heuristic's action), then on approximate policy-iteration labels (the best
// allowed action by a leaf expansion's Q estimate, else "defer").
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "mlp.cuh"
#include "tc_mlp.cuh"
#include "model.hpp"

struct dsp_mlp {
  int max_batch = 0;
  int ldt = 0;                 // row length of the transposed activations: max_batch rounded up to 128
  long long step = 0;
  float* master = nullptr;     // device FP32 parameters (packed)
  float* adam_m = nullptr;     // device Adam first moments
  float* adam_v = nullptr;     // device Adam second moments
  float* grad = nullptr;       // device FP32 gradients (packed)
  __nv_bfloat16* wb = nullptr; // device BF16 W1, W2, W3 input-major ([in][out]): B operands of the backward pass
  __nv_bfloat16* wt = nullptr; // device BF16 W1, W2, W3 output-major ([out][in]): B operands of the forward pass
  // activations and their gradients, row-major [batch][features] and
  // transposed [features][ldt] (the K-major operands of the weight gradients)
  __nv_bfloat16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dl = nullptr, *dh1 = nullptr, *dh2 = nullptr;
  __nv_bfloat16 *xt = nullptr, *h1t = nullptr, *h2t = nullptr, *dlt = nullptr, *dh1t = nullptr, *dh2t = nullptr;
  float* logits = nullptr;
  float* loss = nullptr;       // device scalar
  float* ws = nullptr;          // split-K partial weight gradients: kMaxSplits x 256 x 256
  unsigned int* status = nullptr;  // device: nonzero once a tensor-core wait ran out
};

namespace dsp {
namespace {

// ------------------------------------------------------------------ GEMM ---
// C = A B^T on the fifth-generation tensor cores: A [M][K] and B [N][K], both
// BF16 with K contiguous (the canonical K-major operands), FP32 accumulators
// in tensor memory. A CTA of 128 threads owns a 128-row tile of C and all N
// (<= 256) columns; grid.y splits K into slices whose partial tiles add into
// C (weight gradients, K = batch). Two pipeline stages of 64 along K: all
// threads copy a stage's operands into shared memory with cp.async in the
// no-swizzle core-matrix layout (8 rows x 16 bytes per core matrix), thread 0
// issues its four K = 16 MMAs and commits them to the stage's mbarrier, and
// the next stage's copy overlaps them. Each thread then reads its row from
// tensor memory for the epilogue. Every wait is bounded; a wait that runs
// out sets *status.
constexpr int kTileM = 128;   // rows per CTA: the MMA's M
constexpr int kStageK = 64;   // K per pipeline stage
constexpr int kGemmThreads = 128;

// kBiasRelu: ReLU(acc + bias) as BF16 (hidden layers); kBiasF32: acc + bias
// (logits); kMaskRelu: acc where mask > 0, else 0, as BF16 (the gradient
// through a ReLU); kPartialF32: the K slice's partial tile, to slab
// blockIdx.y of a workspace that reduce_splits sums (weight gradients; the
// sum does not depend on timing, so the gradient is reproducible).
enum Epilogue { kBiasRelu = 0, kBiasF32 = 1, kMaskRelu = 2, kPartialF32 = 3 };
constexpr int kSplitCTAs = 148;  // split-K: about one CTA per SM over the grid
constexpr int kMaxSplits = (kSplitCTAs + 1) / 2;  // for the two 128-row tiles of a 256-row weight gradient

struct GemmArgs {
  const __nv_bfloat16* A;
  int lda;                      // [M][K] (rows of A beyond M read as 0)
  const __nv_bfloat16* B;
  int ldb;                      // [N][K]
  int M, N, K;                  // K: a multiple of 8 (beyond K: 0)
  int kslice;                   // K per CTA along grid.y, a multiple of kStageK
  const float* bias;            // [N]
  const __nv_bfloat16* mask;    // [M][ldc]
  __nv_bfloat16* Cb;            // BF16 result [M][ldc]
  int ldc;
  __nv_bfloat16* Ct;            // its transpose [N][ldt], rows of the tile beyond M written as 0; or null
  int ldt;
  float* Cf;                    // kBiasF32: [M][ldm] row-major; kPartialF32: workspace [splits][M][N]
  long long ldm;
  unsigned int* status;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

template <int EPI, int N>
__global__ void __launch_bounds__(kGemmThreads) gemm_tc(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t kBytesA = kTileM * kStageK * 2, kBytesB = N * kStageK * 2, kStage = kBytesA + kBytesB;
  constexpr uint32_t kCols = N;  // 32, 64 or 256 FP32 columns (a power of two, at least 32)
  constexpr uint32_t kIdesc = tc::idesc_bf16(kTileM, N);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * kStage);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTileM;
  const int kb = blockIdx.y * g.kslice, ke = min(g.K, kb + g.kslice);
  const int nk = ke > kb ? (ke - kb + kStageK - 1) / kStageK : 0;
  const uint32_t mb0 = tc::smem_u32(&mbar[0]), mb1 = tc::smem_u32(&mbar[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tslot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  // stage s <- K columns [kb + 64 c, kb + 64 c + 64) of the tile's A rows and all B rows
  auto load = [&](int c, int s) {
    const int k0 = kb + c * kStageK;
    const uint32_t sa = tc::smem_u32(smem + s * kStage), sb = sa + kBytesA;
    for (int i = tid; i < kTileM * (kStageK / 8); i += kGemmThreads) {
      const int r = i / (kStageK / 8), ch = i % (kStageK / 8), m = m0 + r, k = k0 + 8 * ch;
      const bool in = m < g.M && k < ke;
      cp_async16(sa + tc::kmajor_off(r, 8 * ch, kStageK), in ? (const void*)(g.A + (size_t)m * g.lda + k) : g.A,
                 in ? 16u : 0u);
    }
    for (int i = tid; i < N * (kStageK / 8); i += kGemmThreads) {
      const int r = i / (kStageK / 8), ch = i % (kStageK / 8), k = k0 + 8 * ch;
      const bool in = r < g.N && k < ke;
      cp_async16(sb + tc::kmajor_off(r, 8 * ch, kStageK), in ? (const void*)(g.B + (size_t)r * g.ldb + k) : g.B,
                 in ? 16u : 0u);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  bool ok = true;
  if (nk > 0) load(0, 0);
  for (int c = 0; c < nk; ++c) {
    const int s = c & 1;
    if (c + 1 < nk) {
      // stage s ^ 1 last held chunk c - 1: its MMAs must be done reading it
      if (c >= 1) ok = tc::mbar_wait(s ? mb0 : mb1, ((c - 1) >> 1) & 1) && ok;
      load(c + 1, s ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    tc::fence_async_smem();  // this thread's copies, visible to the tensor cores
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t sa = tc::smem_u32(smem + s * kStage), sb = sa + kBytesA;
      const int k16 = min(kStageK / 16, (ke - (kb + c * kStageK) + 15) / 16);
      for (int k = 0; k < k16; ++k)
        tc::mma_ss(tmem, tc::smem_desc(sa + 256 * k, 128, (kStageK / 8) * 128),
                   tc::smem_desc(sb + 256 * k, 128, (kStageK / 8) * 128), kIdesc, (c > 0 || k > 0) ? 1u : 0u);
      tc::mma_commit(s ? mb1 : mb0);
    }
  }
  if (nk > 0) ok = tc::mbar_wait(((nk - 1) & 1) ? mb1 : mb0, ((nk - 1) >> 1) & 1) && ok;
  tc::fence_after_sync();
  if (!ok && g.status != nullptr) atomicOr(g.status, 1u);

  // epilogue: thread (warp, lane) owns row m0 + 32 warp + lane (tensor-memory lane 32 warp + lane)
  const int m = m0 + 32 * warp + lane;
  const bool row = m < g.M;
  const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
  // the pipeline's stages are dead now: each warp's 32 x 32 transpose tile
  __nv_bfloat16(*tp)[34] = reinterpret_cast<__nv_bfloat16(*)[34]>(smem + warp * 32 * 34 * 2);
  if (nk > 0 && ok) {
#pragma unroll 1
    for (int c0 = 0; c0 < N; c0 += 32) {
      float v[32];
      tc::tmem_ld32(trow + c0, v);
      if (EPI == kPartialF32) {
        if (row) {
          float4* dst = reinterpret_cast<float4*>(g.Cf + ((size_t)blockIdx.y * g.M + m) * N + c0);
#pragma unroll
          for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
      } else if (EPI == kBiasF32) {
        if (row) {
          float4* dst = reinterpret_cast<float4*>(g.Cf + (size_t)m * g.ldm + c0);
#pragma unroll
          for (int q = 0; q < 8; ++q)
            dst[q] = make_float4(__fadd_rn(v[4 * q], g.bias[c0 + 4 * q]), __fadd_rn(v[4 * q + 1], g.bias[c0 + 4 * q + 1]),
                                 __fadd_rn(v[4 * q + 2], g.bias[c0 + 4 * q + 2]),
                                 __fadd_rn(v[4 * q + 3], g.bias[c0 + 4 * q + 3]));
        }
      } else {
        __nv_bfloat16 mk[32];
        if (EPI == kMaskRelu) {
          uint4* mv = reinterpret_cast<uint4*>(mk);
          const uint4* src = reinterpret_cast<const uint4*>(g.mask + (size_t)m * g.ldc + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) mv[q] = row ? src[q] : make_uint4(0u, 0u, 0u, 0u);
        }
        __nv_bfloat16 o[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          float x;
          if (EPI == kBiasRelu)
            x = fmaxf(__fadd_rn(v[j], g.bias[c0 + j]), 0.0f);
          else
            x = __bfloat162float(mk[j]) > 0.0f ? v[j] : 0.0f;
          o[j] = __float2bfloat16_rn(row ? x : 0.0f);
        }
        if (row) {
          uint4* dst = reinterpret_cast<uint4*>(g.Cb + (size_t)m * g.ldc + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
        }
        if (g.Ct != nullptr) {
          // through the warp's tile: lane r writes row r, then lane j reads
          // column j and stores its 32 rows as 64 contiguous bytes
#pragma unroll
          for (int j = 0; j < 32; ++j) tp[lane][j] = o[j];
          __syncwarp();
          __nv_bfloat16 col[32];
#pragma unroll
          for (int r = 0; r < 32; ++r) col[r] = tp[r][lane];
          uint4* dst = reinterpret_cast<uint4*>(g.Ct + (size_t)(c0 + lane) * g.ldt + m0 + 32 * warp);
#pragma unroll
          for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(col)[q];
          __syncwarp();
        }
      }
    }
  }
  // a wait that ran out: wait once more (bounded) for the last MMAs before
  // the tensor memory is freed
  if (nk > 0 && !ok) tc::mbar_wait(((nk - 1) & 1) ? mb1 : mb0, ((nk - 1) >> 1) & 1);
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

template <int EPI, int N>
cudaError_t gemm(GemmArgs g, cudaStream_t st, int* splits_out = nullptr) {
  constexpr size_t smem = 2 * (size_t)(kTileM * kStageK * 2 + N * kStageK * 2) + 64;
  static bool attr = false;  // set once per process (the attribute is per function)
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(gemm_tc<EPI, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  int splits = 1;
  const int tiles = (g.M + kTileM - 1) / kTileM;
  if (EPI == kPartialF32) {  // about one CTA per SM, at most kMaxSplits slabs
    const int chunks = (g.K + kStageK - 1) / kStageK;
    splits = std::max(1, std::min({chunks, (kSplitCTAs + tiles - 1) / tiles, kMaxSplits}));
    g.kslice = ((chunks + splits - 1) / splits) * kStageK;
    splits = (g.K + g.kslice - 1) / g.kslice;
  } else {
    g.kslice = ((g.K + kStageK - 1) / kStageK) * kStageK;
  }
  gemm_tc<EPI, N><<<dim3(tiles, splits), kGemmThreads, smem, st>>>(g);
  if (splits_out != nullptr) *splits_out = splits;
  return cudaGetLastError();
}

// out[m * ldm + n * ldn] = sum over the split-K slabs of ws[s][m][n].
__global__ void reduce_splits(const float* __restrict__ ws, int splits, int M, int N, float* out, int ldm,
                              int ldn) {
  const int total = M * N;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    float acc = 0.0f;
    for (int s = 0; s < splits; ++s) acc += ws[(size_t)s * total + i];
    out[(size_t)(i / N) * ldm + (size_t)(i % N) * ldn] = acc;
  }
}

// A weight gradient C[M][N] = A B^T over K = the padded batch, split over K,
// summed into out[m * ldm + n * ldn].
template <int N>
cudaError_t weight_grad(GemmArgs g, float* ws, float* out, int ldm, int ldn, cudaStream_t st) {
  g.Cf = ws;
  int splits = 1;
  cudaError_t e = gemm<kPartialF32, N>(g, st, &splits);
  if (e != cudaSuccess) return e;
  reduce_splits<<<(g.M * N + 255) / 256, 256, 0, st>>>(ws, splits, g.M, N, out, ldm, ldn);
  return cudaGetLastError();
}

// X (FP32 [B][64]) -> xb (BF16, row-major) and xt ([64][ldt], zero for rows
// B .. rounded up to the tile).
__global__ void to_bf16(const float* x, __nv_bfloat16* xb, __nv_bfloat16* xt, int B, int Bpad, int ldt) {
  const size_t n = (size_t)Bpad * kMlpIn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(i % kMlpIn), b = (int)(i / kMlpIn);
    const __nv_bfloat16 v = __float2bfloat16_rn(b < B ? x[i] : 0.0f);
    if (b < B) xb[i] = v;
    xt[(size_t)k * ldt + b] = v;
  }
}

// Per row: loss -log softmax(logits[:na])[y] (summed into *loss) and
// dlogits = (softmax - onehot) / B (zero past na), in BF16, row-major and
// transposed (rows B .. Bpad of the transpose are 0).
__global__ void softmax_ce(const float* logits, const int32_t* y, int B, int Bpad, int na, __nv_bfloat16* dl,
                           __nv_bfloat16* dlt, int ldt, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Bpad) return;
  const bool live = i < B;
  const float* l = logits + (size_t)(live ? i : 0) * kMlpOut;
  float mx = l[0];
  for (int a = 1; a < na; ++a) mx = fmaxf(mx, l[a]);
  float z = 0.0f;
  for (int a = 0; a < na; ++a) z += expf(l[a] - mx);
  const int yi = live ? y[i] : 0;
  float li = live ? -(l[yi] - mx - logf(z)) : 0.0f;
  for (int o = 16; o > 0; o >>= 1) li += __shfl_down_sync(0xFFFFFFFFu, li, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, li);  // one atomic per warp (Bpad is a multiple of 32)
  for (int a = 0; a < kMlpOut; ++a) {
    const float p = a < na ? expf(l[a] - mx) / z : 0.0f;
    const __nv_bfloat16 d = __float2bfloat16_rn(live ? (p - (a == yi ? 1.0f : 0.0f)) / (float)B : 0.0f);
    if (live) dl[(size_t)i * kMlpOut + a] = d;
    dlt[(size_t)a * ldt + i] = d;
  }
}

// out[n] += sum over rows of x[row][n]: CTA b sums rows [b * kColRows,
// (b + 1) * kColRows) for every column (one thread per column) and adds its
// partial sums into the zeroed out.
constexpr int kColRows = 32;
__global__ void col_sum(const __nv_bfloat16* x, int rows, int cols, float* out) {
  const int n = threadIdx.x;
  if (n >= cols) return;
  const int r0 = blockIdx.x * kColRows, r1 = min(rows, r0 + kColRows);
  float s = 0.0f;
  for (int r = r0; r < r1; ++r) s += __bfloat162float(x[(size_t)r * cols + n]);
  atomicAdd(out + n, s);
}

__global__ void adam(float* p, float* m, float* v, const float* g, int n, float lr, float b1, float b2, float eps,
                     float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// BF16 copies of the master weights, input-major ([in][out], wb) and
// output-major ([out][in], wt).
__global__ void pack_weights_bf16(const float* master, __nv_bfloat16* wb, __nv_bfloat16* wt) {
  const int n1 = kMlpIn * kMlpHid, n2 = kMlpHid * kMlpHid, n3 = kMlpHid * kMlpOut;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3; i += gridDim.x * blockDim.x) {
    int base, in_dim, out_dim, off;
    if (i < n1) {
      base = 0, in_dim = kMlpIn, out_dim = kMlpHid, off = kOffW1;
    } else if (i < n1 + n2) {
      base = n1, in_dim = kMlpHid, out_dim = kMlpHid, off = kOffW2;
    } else {
      base = n1 + n2, in_dim = kMlpHid, out_dim = kMlpOut, off = kOffW3;
    }
    const int r = i - base, in = r / out_dim, out = r % out_dim;
    const __nv_bfloat16 v = __float2bfloat16_rn(master[off + r]);
    wb[i] = v;
    wt[base + out * in_dim + in] = v;
  }
}

cudaError_t col_sums(const __nv_bfloat16* x, int rows, int cols, float* out, cudaStream_t st) {
  col_sum<<<(rows + kColRows - 1) / kColRows, cols, 0, st>>>(x, rows, cols, out);
  return cudaGetLastError();
}

int pad_rows(int B) { return (B + kTileM - 1) / kTileM * kTileM; }

GemmArgs gemm_args(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K,
                   unsigned int* status) {
  GemmArgs g{};
  g.A = A, g.lda = lda, g.B = B, g.ldb = ldb, g.M = M, g.N = N, g.K = K, g.status = status;
  return g;
}

// Forward pass on X (device, FP32, B x 64): xb, xt, h1, h1t, h2, h2t (BF16)
// and the logits (FP32).
cudaError_t forward(dsp_mlp* q, const float* X, int B, cudaStream_t st) {
  const int Bp = pad_rows(B);
  const __nv_bfloat16* W1t = q->wt;
  const __nv_bfloat16* W2t = q->wt + kMlpIn * kMlpHid;
  const __nv_bfloat16* W3t = W2t + kMlpHid * kMlpHid;
  to_bf16<<<256, 256, 0, st>>>(X, q->xb, q->xt, B, Bp, q->ldt);
  // H1 = ReLU(X W1 + b1): A = X [B][64], B operand W1^T [256][64]
  GemmArgs g = gemm_args(q->xb, kMlpIn, W1t, kMlpIn, B, kMlpHid, kMlpIn, q->status);
  g.bias = q->master + kOffB1, g.Cb = q->h1, g.ldc = kMlpHid, g.Ct = q->h1t, g.ldt = q->ldt;
  cudaError_t e = gemm<kBiasRelu, kMlpHid>(g, st);
  // H2 = ReLU(H1 W2 + b2)
  g = gemm_args(q->h1, kMlpHid, W2t, kMlpHid, B, kMlpHid, kMlpHid, q->status);
  g.bias = q->master + kOffB2, g.Cb = q->h2, g.ldc = kMlpHid, g.Ct = q->h2t, g.ldt = q->ldt;
  if (e == cudaSuccess) e = gemm<kBiasRelu, kMlpHid>(g, st);
  // logits = H2 W3 + b3
  g = gemm_args(q->h2, kMlpHid, W3t, kMlpHid, B, kMlpOut, kMlpHid, q->status);
  g.bias = q->master + kOffB3, g.Cf = q->logits, g.ldm = kMlpOut;
  if (e == cudaSuccess) e = gemm<kBiasF32, kMlpOut>(g, st);
  return e;
}

// Loss and packed FP32 gradient into q->grad (after a forward pass). The
// weight gradients reduce over the batch: K = the padded batch of the
// transposed activations (the padding is 0).
cudaError_t backward(dsp_mlp* q, const int32_t* y, int B, int na, cudaStream_t st) {
  const int Bp = pad_rows(B);
  const __nv_bfloat16* W2 = q->wb + kMlpIn * kMlpHid;
  const __nv_bfloat16* W3 = W2 + kMlpHid * kMlpHid;
  cudaMemsetAsync(q->loss, 0, sizeof(float), st);
  cudaMemsetAsync(q->grad, 0, kMlpParams * sizeof(float), st);  // the bias column sums add into it
  softmax_ce<<<Bp / 128, 128, 0, st>>>(q->logits, y, B, Bp, na, q->dl, q->dlt, q->ldt, q->loss);
  // dW3[in][out] = sum_b H2[b][in] dL[b][out]: C[M = in][N = out], A = H2^T, B operand dL^T
  GemmArgs g = gemm_args(q->h2t, q->ldt, q->dlt, q->ldt, kMlpHid, kMlpOut, Bp, q->status);
  cudaError_t e = weight_grad<kMlpOut>(g, q->ws, q->grad + kOffW3, kMlpOut, 1, st);
  if (e == cudaSuccess) e = col_sums(q->dl, B, kMlpOut, q->grad + kOffB3, st);
  // dH2 = (dL W3^T) where H2 > 0: A = dL [B][32], B operand W3 [256 in][32 out]
  g = gemm_args(q->dl, kMlpOut, W3, kMlpOut, B, kMlpHid, kMlpOut, q->status);
  g.mask = q->h2, g.Cb = q->dh2, g.ldc = kMlpHid, g.Ct = q->dh2t, g.ldt = q->ldt;
  if (e == cudaSuccess) e = gemm<kMaskRelu, kMlpHid>(g, st);
  // dW2[in][out] = sum_b H1[b][in] dH2[b][out]
  g = gemm_args(q->h1t, q->ldt, q->dh2t, q->ldt, kMlpHid, kMlpHid, Bp, q->status);
  if (e == cudaSuccess) e = weight_grad<kMlpHid>(g, q->ws, q->grad + kOffW2, kMlpHid, 1, st);
  if (e == cudaSuccess) e = col_sums(q->dh2, B, kMlpHid, q->grad + kOffB2, st);
  // dH1 = (dH2 W2^T) where H1 > 0: B operand W2 [256 in][256 out]
  g = gemm_args(q->dh2, kMlpHid, W2, kMlpHid, B, kMlpHid, kMlpHid, q->status);
  g.mask = q->h1, g.Cb = q->dh1, g.ldc = kMlpHid, g.Ct = q->dh1t, g.ldt = q->ldt;
  if (e == cudaSuccess) e = gemm<kMaskRelu, kMlpHid>(g, st);
  // dW1[in][out] = sum_b X[b][in] dH1[b][out], as C[M = out][N = in] (A = dH1^T,
  // B operand X^T), written transposed
  g = gemm_args(q->dh1t, q->ldt, q->xt, q->ldt, kMlpHid, kMlpIn, Bp, q->status);
  if (e == cudaSuccess) e = weight_grad<kMlpIn>(g, q->ws, q->grad + kOffW1, 1, kMlpHid, st);
  if (e == cudaSuccess) e = col_sums(q->dh1, B, kMlpHid, q->grad + kOffB1, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// The tensor-core status word: a wait that ran out makes the call fail.
cudaError_t check_status(dsp_mlp* q, cudaStream_t st, bool* timed_out) {
  unsigned int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, q->status, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *timed_out = h != 0;
  return e;
}

}  // namespace
}  // namespace dsp

using namespace dsp;

extern "C" {

dsp_status dsp_mlp_create(int32_t max_batch, uint64_t seed, dsp_mlp** out) {
  if (!out || max_batch < 1) return fail(DSP_E_INVALID, "dsp_mlp_create: bad argument");
  *out = nullptr;
  dsp_mlp* q = new dsp_mlp();
  q->max_batch = max_batch;
  q->ldt = pad_rows(max_batch);
  const size_t P = kMlpParams * sizeof(float);
  const size_t W = (size_t)(kMlpIn * kMlpHid + kMlpHid * kMlpHid + kMlpHid * kMlpOut) * sizeof(__nv_bfloat16);
  const size_t B = (size_t)max_batch, T = (size_t)q->ldt;
  cudaError_t e = cudaMalloc(&q->master, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->adam_m, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->adam_v, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->grad, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->wb, W);
  if (e == cudaSuccess) e = cudaMalloc(&q->wt, W);
  if (e == cudaSuccess) e = cudaMalloc(&q->xt, T * kMlpIn * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->h1t, T * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->h2t, T * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dh1t, T * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dh2t, T * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dlt, T * kMlpOut * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->ws, (size_t)kMaxSplits * kMlpHid * kMlpHid * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&q->status, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(q->status, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc(&q->xb, B * kMlpIn * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->h1, B * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->h2, B * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dh1, B * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dh2, B * kMlpHid * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->dl, B * kMlpOut * 2);
  if (e == cudaSuccess) e = cudaMalloc(&q->logits, B * kMlpOut * 4);
  if (e == cudaSuccess) e = cudaMalloc(&q->loss, 4);
  if (e == cudaSuccess) e = cudaMemset(q->adam_m, 0, P);
  if (e == cudaSuccess) e = cudaMemset(q->adam_v, 0, P);
  if (e != cudaSuccess) {
    dsp_status s = cuda_fail(e, "dsp_mlp_create");
    dsp_mlp_destroy(q);
    return s;
  }
  // He-normal weights, zero biases
  std::vector<float> h(kMlpParams, 0.0f);
  std::mt19937_64 rng(seed);
  auto fill = [&](int off, int fan_in, int count) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / fan_in));
    for (int i = 0; i < count; ++i) h[off + i] = (float)nd(rng);
  };
  fill(kOffW1, kMlpIn, kMlpIn * kMlpHid);
  fill(kOffW2, kMlpHid, kMlpHid * kMlpHid);
  fill(kOffW3, kMlpHid, kMlpHid * kMlpOut);
  dsp_status s = dsp_mlp_set_weights(q, h.data());
  if (s != DSP_OK) {
    dsp_mlp_destroy(q);
    return s;
  }
  *out = q;
  return DSP_OK;
}

void dsp_mlp_destroy(dsp_mlp* q) {
  if (!q) return;
  void* ptrs[] = {q->master, q->adam_m, q->adam_v, q->grad, q->wb,  q->wt,  q->xb,   q->h1,   q->h2,     q->dh1,
                  q->dh2,    q->dl,     q->xt,     q->h1t, q->h2t, q->dh1t, q->dh2t, q->dlt, q->logits, q->loss,
                  q->ws,     q->status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete q;
}

dsp_status dsp_mlp_set_weights(dsp_mlp* q, const float* host) {
  if (!q || !host) return fail(DSP_E_INVALID, "dsp_mlp_set_weights: NULL argument");
  cudaError_t e = cudaMemcpy(q->master, host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    pack_weights_bf16<<<128, 256>>>(q->master, q->wb, q->wt);
    e = cudaDeviceSynchronize();
  }
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_set_weights");
}

dsp_status dsp_mlp_get_weights(const dsp_mlp* q, float* host) {
  if (!q || !host) return fail(DSP_E_INVALID, "dsp_mlp_get_weights: NULL argument");
  cudaError_t e = cudaMemcpy(host, q->master, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_get_weights");
}

dsp_status dsp_mlp_forward(dsp_mlp* q, const float* X, int32_t B, float* logits, void* stream) {
  if (!q || !X || !logits || B < 1 || B > q->max_batch) return fail(DSP_E_INVALID, "dsp_mlp_forward: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = forward(q, X, B, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(logits, q->logits, (size_t)B * kMlpOut * 4, cudaMemcpyDeviceToDevice, st);
  bool timed_out = false;
  if (e == cudaSuccess) e = check_status(q, st, &timed_out);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_mlp_forward");
  return timed_out ? fail(DSP_E_TIMEOUT, "dsp_mlp_forward: a tensor-core wait ran out") : DSP_OK;
}

dsp_status dsp_mlp_grad(dsp_mlp* q, const float* X, const int32_t* y, int32_t B, int32_t n_actions, float* loss,
                        float* grad_host, void* stream) {
  if (!q || !X || !y || !loss || B < 1 || B > q->max_batch || n_actions < 1 || n_actions > kMlpOut)
    return fail(DSP_E_INVALID, "dsp_mlp_grad: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = forward(q, X, B, st);
  if (e == cudaSuccess) e = backward(q, y, B, n_actions, st);
  float l = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, q->loss, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, q->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, st);
  bool timed_out = false;
  if (e == cudaSuccess) e = check_status(q, st, &timed_out);
  *loss = l / (float)B;
  if (e != cudaSuccess) return cuda_fail(e, "dsp_mlp_grad");
  return timed_out ? fail(DSP_E_TIMEOUT, "dsp_mlp_grad: a tensor-core wait ran out") : DSP_OK;
}

dsp_status dsp_mlp_train_step(dsp_mlp* q, const float* X, const int32_t* y, int32_t B, int32_t n_actions, float lr,
                              float* loss, void* stream) {
  if (!q || !X || !y || B < 1 || B > q->max_batch || n_actions < 1 || n_actions > kMlpOut || !(lr > 0))
    return fail(DSP_E_INVALID, "dsp_mlp_train_step: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = forward(q, X, B, st);
  if (e == cudaSuccess) e = backward(q, y, B, n_actions, st);
  q->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - (float)std::pow(b1, (double)q->step), c2 = 1.0f - (float)std::pow(b2, (double)q->step);
  if (e == cudaSuccess) {
    adam<<<256, 256, 0, st>>>(q->master, q->adam_m, q->adam_v, q->grad, kMlpParams, lr, b1, b2, 1e-8f, c1, c2);
    pack_weights_bf16<<<128, 256, 0, st>>>(q->master, q->wb, q->wt);
    e = cudaGetLastError();
  }
  if (loss) {
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, q->loss, 4, cudaMemcpyDeviceToHost, st);
    bool timed_out = false;
    if (e == cudaSuccess) e = check_status(q, st, &timed_out);
    *loss = l / (float)B;
    if (e == cudaSuccess && timed_out) return fail(DSP_E_TIMEOUT, "dsp_mlp_train_step: a tensor-core wait ran out");
  }
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_train_step");
}

}  // extern "C"
