// CPU ORACLE — test infrastructure only. Nothing in the product path may include,
// link or call this file; only tests/, the smoke check and the benchmark's CPU
// baseline leg use it.
//
// Philox4x32-10 counter-based generator, written from its published description
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11, section 3: the Philox S-box = two 32x32->64 multiplies, the bijective
// round, the Weyl key schedule, 10 rounds for Philox4x32).
//
// The paper's scenarios (Sec. III-A) are a sampled start state plus the random
// numbers phi_1, phi_2, ... that determinise every later transition and
// observation. Here phi_t of a scenario is the Philox block at counter
// (scenario, depth t, purpose<<24 | element, planning step) under the key
// (seed_lo, seed_hi), so phi_t of a scenario is the same under every action.
#pragma once
#include <cstdint>

namespace orc {

// Op-counting mode: each primitive arithmetic, compare, logic or select
// operation the model definitions need is counted here (per thread), so the
// benchmark can state algorithmic operations per scenario-step.
inline uint64_t& op_counter() {
  static thread_local uint64_t ops = 0;
  return ops;
}
inline void count_ops(uint64_t k) { op_counter() += k; }

struct Block4 {
  uint32_t w[4];
};

// Multipliers and Weyl increments of Philox4x32 (Salmon et al., Table 2 / Sec. 3.3).
static const uint32_t kPhiloxM0 = 0xD2511F53u;
static const uint32_t kPhiloxM1 = 0xCD9E8D57u;
static const uint32_t kPhiloxW0 = 0x9E3779B9u;
static const uint32_t kPhiloxW1 = 0xBB67AE85u;

// One Philox4x32 round: (hi,lo) products of words 0 and 2; the output permutes
// the words and folds in the round key.
inline void philox_round(uint32_t c[4], uint32_t k0, uint32_t k1) {
  uint64_t p0 = (uint64_t)kPhiloxM0 * (uint64_t)c[0];
  uint64_t p1 = (uint64_t)kPhiloxM1 * (uint64_t)c[2];
  uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t out0 = hi1 ^ c[1] ^ k0;
  uint32_t out1 = lo1;
  uint32_t out2 = hi0 ^ c[3] ^ k1;
  uint32_t out3 = lo0;
  c[0] = out0;
  c[1] = out1;
  c[2] = out2;
  c[3] = out3;
}

// R-round Philox4x32 (R = 10 is the standard generator). The key is bumped by
// the Weyl constants before every round after the first.
inline Block4 philox4x32(const uint32_t ctr[4], uint32_t k0, uint32_t k1, int rounds = 10) {
  count_ops((uint64_t)rounds * 10);
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  for (int r = 0; r < rounds; ++r) {
    if (r > 0) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    philox_round(c, k0, k1);
  }
  Block4 b;
  for (int i = 0; i < 4; ++i) b.w[i] = c[i];
  return b;
}

// Purposes of the random streams (third counter word, high byte).
enum Purpose : uint32_t {
  kPurposeInit = 0,        // start-state sampling (belief resampling)
  kPurposeTransition = 1,  // action failure
  kPurposeSensor = 2,      // sensor noise
  kPurposePedestrian = 3,  // pedestrian motion noise
};

// phi_t of scenario `scen` for one purpose/element at depth `depth`.
inline Block4 scenario_random(uint64_t seed, uint32_t scen, uint32_t depth, uint32_t purpose,
                              uint32_t element, uint32_t plan_step) {
  uint32_t ctr[4] = {scen, depth, (purpose << 24) | (element & 0xFFFFFFu), plan_step};
  return philox4x32(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), 10);
}

}  // namespace orc
