// Shared device-side definitions of the leaf-expansion library: the model's
// constant block, Philox4x32-10, fixed-point conversion, small helpers.
#pragma once
#include <cstdint>

#include "../../include/dsp.h"

namespace dsp {

constexpr int kMaxRocks = 32;
constexpr int kMaxSide = 32;
constexpr int kMaxD2 = 2 * (kMaxSide - 1) * (kMaxSide - 1);
constexpr int kGammaLen = 256;
constexpr int kGaussLen = 4096;
constexpr int kMaxPeds = 64;
constexpr int kMaxScen = 512;
// One-robot Rock Sample jobs may hold up to kMaxScenLarge scenarios: those above
// kMaxScen take phase A's global-memory path (their leaf states in the job's
// leaf-state block instead of shared memory).
constexpr int kMaxScenLarge = 8192;
constexpr uint64_t kTermBit = 1ull << 62;

// Device status word bits.
constexpr uint32_t kStatusTimeout = 1u;
constexpr uint32_t kStatusBadJob = 2u;
constexpr uint32_t kStatusOverflow = 4u;
constexpr uint32_t kStatusKeyClash = 8u;

// Constant block of a model, resident in device memory.
struct DevModel {
  int kind, n, m, robots, per_robot, num_actions, P, K, D, words;
  uint64_t seed;
  float gamma;
  float path_len, dt, ped_speed, sigma, stride;
  uint64_t fail_thresh;                 // car: action failure; navigation: move failure
  uint64_t sense_thresh;                // navigation: a wrong adjacent-cell reading
  int rock_xy[kMaxRocks];               // x | y << 8
  uint8_t cell_rock[kMaxSide * kMaxSide]; // rock index at cell y*n+x, 0xFF none
  float G[kGammaLen];                   // gamma^k in FP32
  uint64_t thresh[kMaxD2 + 1];          // sensor thresholds by squared distance
  float gauss[kGaussLen];               // inverse-normal table
  // Heuristic-policy key of rock i seen from cell c, at [i * n * n + c]:
  // Manhattan distance << 7 | i << 2 | the move toward the rock (0 N, 1 E,
  // 2 S, 3 W; x first). The smallest key over a rock set is the nearest rock
  // with the lowest index on ties, and carries the policy's move.
  uint16_t nkey[kMaxRocks * kMaxSide * kMaxSide];
};
// Entries of the policy-key table: a row of n * n keys per rock.
inline int rs_key_words(const DevModel* h) { return h->m * h->n * h->n; }

// Workspace of a model: counters and the status word.
struct DevWork {
  unsigned long long steps;
  unsigned int status;
};

// ------------------------------------------------------------ Philox ----
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3): ten rounds of
// two 32x32->64 multiplies with a Weyl key schedule.
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// phi_depth of scenario `scen` for one purpose and element.
__device__ __forceinline__ U4 scen_random(uint64_t seed, uint32_t scen, uint32_t depth, uint32_t purpose,
                                          uint32_t element, uint32_t plan_step) {
  return philox10(scen, depth, (purpose << 24) | (element & 0xFFFFFFu), plan_step, (uint32_t)seed,
                  (uint32_t)(seed >> 32));
}

// FP32 value -> int64 fixed point 2^-32, round to nearest even: the exact
// rounding of x * 2^32. Done on x's IEEE-754 fields with integer operations:
// the float -> int64 conversion instruction runs on the FP64 pipe, which is
// narrow on this part, and its result latency stalled the rollout warps.
// A finite x = (-1)^s * M * 2^(E - 150) (M with its implicit one; E = 1 and
// no implicit one for subnormals), so x * 2^32 = M * 2^(E - 118): a left
// shift for E >= 118, else M / 2^r (r = 118 - E) rounded half to even, which
// is 0 for r >= 25 (M < 2^24). |x| >= 2^31 (E >= 158, and inf and NaN) takes
// the conversion instruction, whose saturation it keeps.
__device__ __forceinline__ long long to_fixed(float x) {
  const uint32_t b = __float_as_uint(x);
  const int E = (int)((b >> 23) & 0xFFu);
  if (E >= 158) return __float2ll_rn(__fmul_rn(x, 4294967296.0f));
  const uint32_t M = (b & 0x7FFFFFu) | (E ? 0x800000u : 0u);
  const int e = E ? E : 1;
  long long v;
  if (e >= 118) {
    v = (long long)M << (e - 118);
  } else {
    const int r = 118 - e;
    uint32_t q = 0;
    if (r < 25) {
      q = M >> r;
      const uint32_t rem = M & ((1u << r) - 1u), half = 1u << (r - 1);
      q += (rem > half || (rem == half && (q & 1u))) ? 1u : 0u;
    }
    v = (long long)q;
  }
  return (b >> 31) ? -v : v;
}

// Adds v to a child's fixed-point sum: a reduction on global memory with no
// value returned, so the warp does not wait for it (atomicAdd through a
// generic pointer becomes an atomic that returns the old value).
__device__ __forceinline__ void sum_add(int64_t* p, long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}

__device__ __forceinline__ void report(DevWork* w, uint32_t bits) { atomicOr(&w->status, bits); }

// Saturating +-1 update of belief counter i in 32 packed int8 counters.
__device__ __forceinline__ void hist_add(uint32_t (&h)[8], int i, int delta) {
  int sh = 8 * (i & 3);
  int v = (int)(int8_t)((h[i >> 2] >> sh) & 0xFFu) + delta;
  v = v > 127 ? 127 : (v < -127 ? -127 : v);
  h[i >> 2] = (h[i >> 2] & ~(0xFFu << sh)) | ((uint32_t)(uint8_t)(int8_t)v << sh);
}
__device__ __forceinline__ int hist_get(const uint32_t (&h)[8], int i) {
  return (int)(int8_t)((h[i >> 2] >> (8 * (i & 3))) & 0xFFu);
}

// Rollout items of a car expansion with a learned policy: the stepped states
// as a state block of capacity `total` (words fields), then per item the
// meta word depth << 24 | child slot and the job index.
struct CarItems {
  uint32_t* base;  // null: the expansion rolls out with the heuristic policy
  long long total;
  int words;
  __host__ __device__ uint32_t* meta() const { return base + (size_t)words * total; }
  __host__ __device__ uint32_t* job() const { return base + (size_t)(words + 1) * total; }
};

}  // namespace dsp
