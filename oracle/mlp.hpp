// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// The learned default policy pi0: an MLP 64 -> 256 -> 256 -> 32 (ReLU hidden
// layers; the first |A| logits are the actions), its softmax cross-entropy
// loss for imitation of the planner's chosen actions, the gradient of that
// loss, and the state features the policy reads. Two forward modes:
//  - exact: FP64 throughout;
//  - bf16: weights, features and hidden activations rounded to bfloat16
//    (round to nearest even), products summed in FP32 in input order, the
//    arithmetic the GPU's BF16 tensor-core layers approximate.
// Weights are input-major: W1[k][n] with k < 64, n < 256, etc.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc {

constexpr int kMlpIn = 64, kMlpHid = 256, kMlpOut = 32;

inline float bf16_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return x;  // inf / nan unchanged
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7FFFu + lsb;
  u &= 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

struct Net {
  const double *W1, *b1, *W2, *b2, *W3, *b3;
};

// exact FP64 forward; keeps the hidden activations for the backward pass
inline void forward64(const Net& w, const double* x, double* h1, double* h2, double* logit) {
  for (int n = 0; n < kMlpHid; ++n) {
    double s = w.b1[n];
    for (int k = 0; k < kMlpIn; ++k) s += x[k] * w.W1[k * kMlpHid + n];
    h1[n] = s > 0 ? s : 0;
  }
  for (int n = 0; n < kMlpHid; ++n) {
    double s = w.b2[n];
    for (int k = 0; k < kMlpHid; ++k) s += h1[k] * w.W2[k * kMlpHid + n];
    h2[n] = s > 0 ? s : 0;
  }
  for (int n = 0; n < kMlpOut; ++n) {
    double s = w.b3[n];
    for (int k = 0; k < kMlpHid; ++k) s += h2[k] * w.W3[k * kMlpOut + n];
    logit[n] = s;
  }
}

inline void forward_bf16(const Net& w, const double* x64, double* logit, double* h1_out = nullptr,
                         double* h2_out = nullptr) {
  float x[kMlpIn], h1[kMlpHid], h2[kMlpHid];
  for (int k = 0; k < kMlpIn; ++k) x[k] = bf16_round((float)x64[k]);
  for (int n = 0; n < kMlpHid; ++n) {
    float s = 0.0f;
    for (int k = 0; k < kMlpIn; ++k) s += x[k] * bf16_round((float)w.W1[k * kMlpHid + n]);
    s += (float)w.b1[n];
    h1[n] = bf16_round(s > 0 ? s : 0.0f);
  }
  for (int n = 0; n < kMlpHid; ++n) {
    float s = 0.0f;
    for (int k = 0; k < kMlpHid; ++k) s += h1[k] * bf16_round((float)w.W2[k * kMlpHid + n]);
    s += (float)w.b2[n];
    h2[n] = bf16_round(s > 0 ? s : 0.0f);
  }
  for (int n = 0; n < kMlpOut; ++n) {
    float s = 0.0f;
    for (int k = 0; k < kMlpHid; ++k) s += h2[k] * bf16_round((float)w.W3[k * kMlpOut + n]);
    logit[n] = (double)(s + (float)w.b3[n]);
  }
  if (h1_out)
    for (int n = 0; n < kMlpHid; ++n) h1_out[n] = (double)h1[n];
  if (h2_out)
    for (int n = 0; n < kMlpHid; ++n) h2_out[n] = (double)h2[n];
}



// logits[B][32] of the policy network (bf16 = 1: the BF16/FP32 arithmetic).
inline int mlp_forward(const double* W1, const double* b1, const double* W2, const double* b2, const double* W3,
                    const double* b3, const double* X, int B, int bf16, double* logits) {
  Net w{W1, b1, W2, b2, W3, b3};
  std::vector<double> h1(kMlpHid), h2(kMlpHid);
  for (int i = 0; i < B; ++i) {
    if (bf16)
      forward_bf16(w, X + (size_t)i * kMlpIn, logits + (size_t)i * kMlpOut);
    else
      forward64(w, X + (size_t)i * kMlpIn, h1.data(), h2.data(), logits + (size_t)i * kMlpOut);
  }
  return 0;
}

// Mean softmax cross-entropy over the batch (softmax over the first n_actions
// logits, target y[i]) and its gradient with respect to every parameter, FP64.
// bf16_forward = 1 takes the activations and logits of the BF16/FP32 forward
// form (the backward stays FP64): the gradient the BF16 network has.
inline int mlp_loss_grad(const double* W1, const double* b1, const double* W2, const double* b2, const double* W3,
                      const double* b3, const double* X, const int32_t* y, int B, int n_actions, double* loss,
                      double* gW1, double* gb1, double* gW2, double* gb2, double* gW3, double* gb3,
                      int bf16_forward = 0) {
  Net w{W1, b1, W2, b2, W3, b3};
  std::memset(gW1, 0, sizeof(double) * kMlpIn * kMlpHid);
  std::memset(gb1, 0, sizeof(double) * kMlpHid);
  std::memset(gW2, 0, sizeof(double) * kMlpHid * kMlpHid);
  std::memset(gb2, 0, sizeof(double) * kMlpHid);
  std::memset(gW3, 0, sizeof(double) * kMlpHid * kMlpOut);
  std::memset(gb3, 0, sizeof(double) * kMlpOut);
  std::vector<double> h1(kMlpHid), h2(kMlpHid), lg(kMlpOut), dl(kMlpOut), dh2(kMlpHid), dh1(kMlpHid);
  double total = 0;
  for (int i = 0; i < B; ++i) {
    const double* x = X + (size_t)i * kMlpIn;
    if (bf16_forward)
      forward_bf16(w, x, lg.data(), h1.data(), h2.data());
    else
      forward64(w, x, h1.data(), h2.data(), lg.data());
    double mx = lg[0];
    for (int a = 1; a < n_actions; ++a) mx = std::max(mx, lg[a]);
    double z = 0;
    for (int a = 0; a < n_actions; ++a) z += std::exp(lg[a] - mx);
    total += -(lg[y[i]] - mx - std::log(z));
    for (int a = 0; a < kMlpOut; ++a) {
      double p = a < n_actions ? std::exp(lg[a] - mx) / z : 0.0;
      dl[a] = (p - (a == y[i] ? 1.0 : 0.0)) / B;
    }
    for (int n = 0; n < kMlpOut; ++n) {
      gb3[n] += dl[n];
      for (int k = 0; k < kMlpHid; ++k) gW3[k * kMlpOut + n] += h2[k] * dl[n];
    }
    for (int k = 0; k < kMlpHid; ++k) {
      double s = 0;
      for (int n = 0; n < kMlpOut; ++n) s += w.W3[k * kMlpOut + n] * dl[n];
      dh2[k] = h2[k] > 0 ? s : 0;
    }
    for (int n = 0; n < kMlpHid; ++n) {
      gb2[n] += dh2[n];
      for (int k = 0; k < kMlpHid; ++k) gW2[k * kMlpHid + n] += h1[k] * dh2[n];
    }
    for (int k = 0; k < kMlpHid; ++k) {
      double s = 0;
      for (int n = 0; n < kMlpHid; ++n) s += w.W2[k * kMlpHid + n] * dh2[n];
      dh1[k] = h1[k] > 0 ? s : 0;
    }
    for (int n = 0; n < kMlpHid; ++n) {
      gb1[n] += dh1[n];
      for (int k = 0; k < kMlpIn; ++k) gW1[k * kMlpHid + n] += x[k] * dh1[n];
    }
  }
  *loss = total / B;
  return 0;
}

// Policy features of Rock Sample states (one robot) with belief counters,
// FP32: robot x/n, y/n, then per rock (rock x - x)/n, (rock y - y)/n,
// clamp(counter, -3, 3)/3, sampled (0/1); zero beyond 2 + 4m.
inline int features_rs(int n, int m, const int32_t* rock_cells, const uint32_t* block, int cap, int count,
                    const int8_t* hist, float* out) {
  const float inv_n = 1.0f / (float)n;
  const float third = 1.0f / 3.0f;
  for (int i = 0; i < count; ++i) {
    float* f = out + (size_t)i * kMlpIn;
    for (int k = 0; k < kMlpIn; ++k) f[k] = 0.0f;
    uint32_t pos = block[i];
    int x = (int)(pos & 0xFF), y = (int)((pos >> 8) & 0xFF);
    uint32_t sampled = block[3 * cap + i];
    f[0] = (float)x * inv_n;
    f[1] = (float)y * inv_n;
    for (int r = 0; r < m && 2 + 4 * r + 3 < kMlpIn; ++r) {
      int rx = rock_cells[r] & 0xFF, ry = (rock_cells[r] >> 8) & 0xFF;
      int c = hist ? hist[(size_t)i * 32 + r] : 0;
      c = c > 3 ? 3 : (c < -3 ? -3 : c);
      f[2 + 4 * r] = (float)(rx - x) * inv_n;
      f[3 + 4 * r] = (float)(ry - y) * inv_n;
      f[4 + 4 * r] = (float)c * third;
      f[5 + 4 * r] = ((sampled >> r) & 1u) ? 1.0f : 0.0f;
    }
  }
  return 0;
}

}  // namespace orc
