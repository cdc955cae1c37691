// The learned default policy pi0: an MLP 64 -> 256 -> 256 -> 32 with ReLU
// hidden layers whose first |A| logits score the actions. Shared by the
// training kernels and the in-rollout policy: sizes, the state features (the
// same FP32 operations on host and device), bfloat16 rounding.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace dsp {

constexpr int kMlpIn = 64, kMlpHid = 256, kMlpOut = 32;
// Packed FP32 parameters, input-major weights: W1[64][256] b1[256]
// W2[256][256] b2[256] W3[256][32] b3[32].
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpIn * kMlpHid, kOffW2 = kOffB1 + kMlpHid,
              kOffB2 = kOffW2 + kMlpHid * kMlpHid, kOffW3 = kOffB2 + kMlpHid, kOffB3 = kOffW3 + kMlpHid * kMlpOut,
              kMlpParams = kOffB3 + kMlpOut;

// Policy features of a one-robot Rock Sample state with belief counters:
// x/n, y/n, then per rock (rock x - x)/n, (rock y - y)/n,
// clamp(counter, -3, 3)/3, sampled (0/1); zero beyond 2 + 4m (m <= 15).
__host__ __device__ __forceinline__ void rs_features(int n, int m, const int* rock_xy, uint32_t pos,
                                                     uint32_t sampled, const int8_t* counters, float* f) {
  const float inv_n = 1.0f / (float)n;
  const float third = 1.0f / 3.0f;
  const int x = (int)(pos & 0xFFu), y = (int)((pos >> 8) & 0xFFu);
  for (int k = 0; k < kMlpIn; ++k) f[k] = 0.0f;
  f[0] = (float)x * inv_n;
  f[1] = (float)y * inv_n;
  for (int r = 0; r < m && r < 15; ++r) {
    int rx = rock_xy[r] & 0xFF, ry = rock_xy[r] >> 8;
    int c = counters[r];
    c = c > 3 ? 3 : (c < -3 ? -3 : c);
    f[2 + 4 * r] = (float)(rx - x) * inv_n;
    f[3 + 4 * r] = (float)(ry - y) * inv_n;
    f[4 + 4 * r] = (float)c * third;
    f[5 + 4 * r] = ((sampled >> r) & 1u) ? 1.0f : 0.0f;
  }
}

}  // namespace dsp
