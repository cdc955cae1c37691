// Training of the learned default policy pi0: softmax cross-entropy on
// (state features, action label) pairs with this library's own kernels: BF16
// GEMMs on the tensor cores (mma.sync m16n8k16, FP32 accumulation) with fused
// epilogues, softmax cross-entropy, column sums for the bias gradients, and
// Adam on FP32 master weights with BF16 copies for the next step. The labels
// are the caller's: the shipped weights were trained on approximate
// policy-iteration labels (the best allowed action by a leaf expansion's Q
// estimate, else "defer" to the heuristic); planner imitation labels go
// through the same step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "mlp.cuh"
#include "model.hpp"

struct dsp_mlp {
  int max_batch = 0;
  long long step = 0;
  float* master = nullptr;     // device FP32 parameters (packed)
  float* adam_m = nullptr;     // device Adam first moments
  float* adam_v = nullptr;     // device Adam second moments
  float* grad = nullptr;       // device FP32 gradients (packed)
  __nv_bfloat16* wb = nullptr; // device BF16 copies of W1, W2, W3 (input-major)
  __nv_bfloat16 *xb = nullptr, *h1 = nullptr, *h2 = nullptr, *dl = nullptr, *dh1 = nullptr, *dh2 = nullptr;
  float* logits = nullptr;
  float* loss = nullptr;       // device scalar
};

namespace dsp {
namespace {

constexpr int kTile = 64, kTileK = 32, kPad = 8;

// kAddF32 adds the tile into Cf with FP32 atomics: the split-K form, where
// gridDim.z CTAs each reduce one slice of K into the same zeroed output.
enum Epilogue { kStoreF32 = 0, kBiasReluBf16 = 1, kBiasF32 = 2, kMaskReluBf16 = 3, kAddF32 = 4 };

// C[M][N] = op(A)[M][K] op(B)[K][N]. A: row-major [M][K] (TA = false) or
// stored [K][M] (TA = true); B: stored [K][N] (TB = false) or [N][K]
// (TB = true). 128 threads, a 64 x 64 tile, warps 2 x 2 of 32 x 32. The CTA
// at blockIdx.z takes K's slice [z * kslice, (z + 1) * kslice).
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_bf16(const __nv_bfloat16* __restrict__ A, int lda,
                                                 const __nv_bfloat16* __restrict__ B, int ldb, int M, int N, int K,
                                                 float* Cf, __nv_bfloat16* Cb, int ldc, const float* bias,
                                                 const __nv_bfloat16* mask, int kslice) {
  __shared__ __align__(16) __nv_bfloat16 sA[kTile][kTileK + kPad];
  __shared__ __align__(16) __nv_bfloat16 sB[kTile][kTileK + kPad];  // [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * kTile, n0 = blockIdx.x * kTile;
  const int g = lane >> 2, t = lane & 3;
  const int kb = blockIdx.z * kslice, ke = min(K, kb + kslice);
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.0f;
  const __nv_bfloat16 zero = __float2bfloat16(0.0f);
  for (int k0 = kb; k0 < ke; k0 += kTileK) {
    // consecutive threads take consecutive addresses of each operand: along
    // k for a row-major A and a [N][K] B, along m or n for the others
    for (int e = tid; e < kTile * kTileK; e += 128) {
      const int r = TA ? e % kTile : e / kTileK, c = TA ? e / kTile : e % kTileK;
      const int m = m0 + r, k = k0 + c;
      __nv_bfloat16 va = zero;
      if (m < M && k < ke) va = TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k];
      sA[r][c] = va;
    }
    for (int e = tid; e < kTile * kTileK; e += 128) {
      const int r = TB ? e / kTileK : e % kTile, c = TB ? e % kTileK : e / kTile;
      const int n = n0 + r, k = k0 + c;
      __nv_bfloat16 vb = zero;
      if (n < N && k < ke) vb = TB ? B[(size_t)n * ldb + k] : B[(size_t)k * ldb + n];
      sB[r][c] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTileK; kk += 16) {
      uint32_t af[2][4], bf[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        int r = wm + 16 * i + g;
        af[i][0] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * t]);
        af[i][1] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * t]);
        af[i][2] = *reinterpret_cast<const uint32_t*>(&sA[r][kk + 2 * t + 8]);
        af[i][3] = *reinterpret_cast<const uint32_t*>(&sA[r + 8][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int c = wn + 8 * j + g;
        bf[j][0] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * t]);
        bf[j][1] = *reinterpret_cast<const uint32_t*>(&sB[c][kk + 2 * t + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]), "r"(bf[j][0]), "r"(bf[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        int m = m0 + wm + 16 * i + g + (c >= 2 ? 8 : 0);
        int n = n0 + wn + 8 * j + 2 * t + (c & 1);
        if (m >= M || n >= N) continue;
        float v = acc[i][j][c];
        size_t o = (size_t)m * ldc + n;
        if (EPI == kStoreF32) {
          Cf[o] = v;
        } else if (EPI == kAddF32) {
          atomicAdd(Cf + o, v);
        } else if (EPI == kBiasReluBf16) {
          v += bias[n];
          Cb[o] = __float2bfloat16_rn(v > 0.0f ? v : 0.0f);
        } else if (EPI == kBiasF32) {
          Cf[o] = v + bias[n];
        } else {
          Cb[o] = __float2bfloat16_rn(__bfloat162float(mask[o]) > 0.0f ? v : 0.0f);
        }
      }
}

__global__ void to_bf16(const float* x, __nv_bfloat16* y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// Per row: loss -log softmax(logits[:na])[y] (summed into *loss) and
// dlogits = (softmax - onehot) / B (zero past na), in BF16.
__global__ void softmax_ce(const float* logits, const int32_t* y, int B, int na, __nv_bfloat16* dl, float* loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < B;
  const float* l = logits + (size_t)(live ? i : 0) * kMlpOut;
  float mx = l[0];
  for (int a = 1; a < na; ++a) mx = fmaxf(mx, l[a]);
  float z = 0.0f;
  for (int a = 0; a < na; ++a) z += expf(l[a] - mx);
  const int yi = live ? y[i] : 0;
  float li = live ? -(l[yi] - mx - logf(z)) : 0.0f;
  for (int o = 16; o > 0; o >>= 1) li += __shfl_down_sync(0xFFFFFFFFu, li, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(loss, li);  // one atomic per warp
  if (!live) return;
  for (int a = 0; a < kMlpOut; ++a) {
    float p = a < na ? expf(l[a] - mx) / z : 0.0f;
    dl[(size_t)i * kMlpOut + a] = __float2bfloat16_rn((p - (a == yi ? 1.0f : 0.0f)) / (float)B);
  }
}

// out[n] += sum over rows of x[row][n]: CTA b sums rows [b * kColRows,
// (b + 1) * kColRows) for every column (one thread per column) and adds its
// partial sums into the zeroed out.
constexpr int kColRows = 128;
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

__global__ void pack_weights_bf16(const float* master, __nv_bfloat16* wb) {
  const int n1 = kMlpIn * kMlpHid, n2 = kMlpHid * kMlpHid, n3 = kMlpHid * kMlpOut;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n1 + n2 + n3; i += gridDim.x * blockDim.x) {
    float v = i < n1 ? master[kOffW1 + i] : (i < n1 + n2 ? master[kOffW2 + i - n1] : master[kOffW3 + i - n1 - n2]);
    wb[i] = __float2bfloat16_rn(v);
  }
}

template <bool TA, bool TB, int EPI>
cudaError_t gemm(const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, int M, int N, int K, float* Cf,
                 __nv_bfloat16* Cb, int ldc, const float* bias, const __nv_bfloat16* mask, cudaStream_t st) {
  // a long K over few output tiles (the weight gradients, K = batch) is
  // split so that the grid covers the SMs; the slices add into Cf
  int splits = 1;
  const int tiles = ((N + kTile - 1) / kTile) * ((M + kTile - 1) / kTile);
  if (EPI == kAddF32) splits = std::max(1, std::min((K + 511) / 512, (4 * 148 + tiles - 1) / tiles));
  const int kslice = ((K + splits - 1) / splits + kTileK - 1) / kTileK * kTileK;
  splits = (K + kslice - 1) / kslice;
  dim3 grid((N + kTile - 1) / kTile, (M + kTile - 1) / kTile, splits);
  gemm_bf16<TA, TB, EPI><<<grid, 128, 0, st>>>(A, lda, B, ldb, M, N, K, Cf, Cb, ldc, bias, mask, kslice);
  return cudaGetLastError();
}

cudaError_t col_sums(const __nv_bfloat16* x, int rows, int cols, float* out, cudaStream_t st) {
  col_sum<<<(rows + kColRows - 1) / kColRows, cols, 0, st>>>(x, rows, cols, out);
  return cudaGetLastError();
}

// Forward pass on X (device, FP32, B x 64): xb, h1, h2 (BF16) and logits.
cudaError_t forward(dsp_mlp* q, const float* X, int B, cudaStream_t st) {
  const __nv_bfloat16* W1 = q->wb;
  const __nv_bfloat16* W2 = q->wb + kMlpIn * kMlpHid;
  const __nv_bfloat16* W3 = W2 + kMlpHid * kMlpHid;
  to_bf16<<<64, 256, 0, st>>>(X, q->xb, (size_t)B * kMlpIn);
  cudaError_t e = gemm<false, false, kBiasReluBf16>(q->xb, kMlpIn, W1, kMlpHid, B, kMlpHid, kMlpIn, nullptr, q->h1,
                                                    kMlpHid, q->master + kOffB1, nullptr, st);
  if (e == cudaSuccess)
    e = gemm<false, false, kBiasReluBf16>(q->h1, kMlpHid, W2, kMlpHid, B, kMlpHid, kMlpHid, nullptr, q->h2, kMlpHid,
                                          q->master + kOffB2, nullptr, st);
  if (e == cudaSuccess)
    e = gemm<false, false, kBiasF32>(q->h2, kMlpHid, W3, kMlpOut, B, kMlpOut, kMlpHid, q->logits, nullptr, kMlpOut,
                                     q->master + kOffB3, nullptr, st);
  return e;
}

// Loss and packed FP32 gradient into q->grad (after a forward pass).
cudaError_t backward(dsp_mlp* q, const int32_t* y, int B, int na, cudaStream_t st) {
  const __nv_bfloat16* W2 = q->wb + kMlpIn * kMlpHid;
  const __nv_bfloat16* W3 = W2 + kMlpHid * kMlpHid;
  cudaMemsetAsync(q->loss, 0, sizeof(float), st);
  cudaMemsetAsync(q->grad, 0, kMlpParams * sizeof(float), st);  // the split-K GEMMs and column sums add into it
  softmax_ce<<<(B + 127) / 128, 128, 0, st>>>(q->logits, y, B, na, q->dl, q->loss);
  // dW3 = H2^T dL, db3 = colsum(dL)
  cudaError_t e = gemm<true, false, kAddF32>(q->h2, kMlpHid, q->dl, kMlpOut, kMlpHid, kMlpOut, B,
                                               q->grad + kOffW3, nullptr, kMlpOut, nullptr, nullptr, st);
  if (e == cudaSuccess) e = col_sums(q->dl, B, kMlpOut, q->grad + kOffB3, st);
  // dH2 = (dL W3^T) masked by H2 > 0
  if (e == cudaSuccess)
    e = gemm<false, true, kMaskReluBf16>(q->dl, kMlpOut, W3, kMlpOut, B, kMlpHid, kMlpOut, nullptr, q->dh2, kMlpHid,
                                         nullptr, q->h2, st);
  if (e == cudaSuccess)
    e = gemm<true, false, kAddF32>(q->h1, kMlpHid, q->dh2, kMlpHid, kMlpHid, kMlpHid, B, q->grad + kOffW2,
                                     nullptr, kMlpHid, nullptr, nullptr, st);
  if (e == cudaSuccess) e = col_sums(q->dh2, B, kMlpHid, q->grad + kOffB2, st);
  if (e == cudaSuccess)
    e = gemm<false, true, kMaskReluBf16>(q->dh2, kMlpHid, W2, kMlpHid, B, kMlpHid, kMlpHid, nullptr, q->dh1,
                                         kMlpHid, nullptr, q->h1, st);
  if (e == cudaSuccess)
    e = gemm<true, false, kAddF32>(q->xb, kMlpIn, q->dh1, kMlpHid, kMlpIn, kMlpHid, B, q->grad + kOffW1, nullptr,
                                     kMlpHid, nullptr, nullptr, st);
  if (e == cudaSuccess) e = col_sums(q->dh1, B, kMlpHid, q->grad + kOffB1, st);
  if (e == cudaSuccess) e = cudaGetLastError();
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
  const size_t P = kMlpParams * sizeof(float);
  const size_t W = (size_t)(kMlpIn * kMlpHid + kMlpHid * kMlpHid + kMlpHid * kMlpOut) * sizeof(__nv_bfloat16);
  const size_t B = (size_t)max_batch;
  cudaError_t e = cudaMalloc(&q->master, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->adam_m, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->adam_v, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->grad, P);
  if (e == cudaSuccess) e = cudaMalloc(&q->wb, W);
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
  void* ptrs[] = {q->master, q->adam_m, q->adam_v, q->grad, q->wb, q->xb, q->h1, q->h2, q->dh1, q->dh2, q->dl,
                  q->logits, q->loss};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete q;
}

dsp_status dsp_mlp_set_weights(dsp_mlp* q, const float* host) {
  if (!q || !host) return fail(DSP_E_INVALID, "dsp_mlp_set_weights: NULL argument");
  cudaError_t e = cudaMemcpy(q->master, host, kMlpParams * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    pack_weights_bf16<<<128, 256>>>(q->master, q->wb);
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
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_forward");
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
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  *loss = l / (float)B;
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_grad");
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
    pack_weights_bf16<<<128, 256, 0, st>>>(q->master, q->wb);
    e = cudaGetLastError();
  }
  if (loss) {
    float l = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l, q->loss, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    *loss = l / (float)B;
  }
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_mlp_train_step");
}

}  // extern "C"
