// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// Rock Sample with one robot ("grid") or two robots ("multigrid"), the
// multi-agent Rock Sample task of Sec. IV-A: an n x n map, m rocks that are
// good or bad, robots that move, sample, or sense a rock with a sensor whose
// accuracy decays exponentially with distance, +10 for sampling a good rock,
// -10 for a bad one, +10 for leaving by the east border; the world ends when
// every robot has left.
//
// Readings where the paper is silent:
//  * actions per robot: 0 N (y+1), 1 E (x+1), 2 S (y-1), 3 W (x-1), 4 Sample,
//    5+i Sense rock i; joint action a = a0 * (5+m) + a1;
//  * a move off the N/S/W border, or Sample where no rock lies, is illegal:
//    -100 and the robot stays; E from x = n-1 exits (+10);
//  * sampling a good rock turns it bad; robots act in index order, so robot 0
//    wins a rock both sample; an exited robot's actions do nothing;
//  * sense distance is Euclidean; observation per robot 0 none, 1 good, 2 bad;
//    the joint observation is z0 * 3 + z1 and bit 62 of the key marks a
//    terminal outcome.
#pragma once
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "philox.hpp"
#include "tables.hpp"

namespace orc {

static const uint64_t kTerminalBit = 1ull << 62;

struct RSState {
  int x[2], y[2];
  bool exited[2];
  uint32_t good;     // bit i: rock i is good
  uint32_t sampled;  // bit i: rock i has been sampled (known from the action history)
  uint32_t scen;     // scenario id (key of its random stream)
};

// Per-rock belief counters of a history: #good - #bad readings of rock i.
struct Hist {
  int8_t c[32];
};

template <class Real>
struct RockSample {
  int n = 7, m = 8, robots = 1;
  float gamma = 0.95f;
  int K = 100, D = 90;
  uint64_t seed = 0;
  uint32_t plan_step = 0;
  int rock_x[32], rock_y[32];
  std::vector<uint64_t> thresh;  // sensor table indexed by squared distance
  std::vector<Real> G;           // gamma^k

  void init() {
    thresh = sensor_thresholds(2 * (n - 1) * (n - 1));
    G = gamma_powers<Real>(gamma, 256);
  }

  int actions_per_robot() const { return 5 + m; }
  int num_actions() const {
    return robots == 1 ? actions_per_robot() : actions_per_robot() * actions_per_robot();
  }
  bool terminal(const RSState& s) const {
    for (int r = 0; r < robots; ++r)
      if (!s.exited[r]) return false;
    return true;
  }
  int rock_at(int x, int y) const {
    for (int i = 0; i < m; ++i)
      if (rock_x[i] == x && rock_y[i] == y) return i;
    return -1;
  }

  // One robot's part of g: returns its reward, writes its observation.
  int robot_step(RSState& s, int r, int a, int depth, int* z) const {
    *z = 0;
    count_ops(1);
    if (s.exited[r]) return 0;
    int reward = 0;
    count_ops(4);  // decode position, dispatch on the action, re-encode
    if (a == 0) {  // north
      count_ops(2);
      if (s.y[r] == n - 1)
        reward = -100;
      else
        s.y[r] += 1;
    } else if (a == 1) {  // east
      count_ops(2);
      if (s.x[r] == n - 1) {
        reward = 10;
        s.exited[r] = true;
      } else {
        s.x[r] += 1;
      }
    } else if (a == 2) {  // south
      count_ops(2);
      if (s.y[r] == 0)
        reward = -100;
      else
        s.y[r] -= 1;
    } else if (a == 3) {  // west
      count_ops(2);
      if (s.x[r] == 0)
        reward = -100;
      else
        s.x[r] -= 1;
    } else if (a == 4) {  // sample
      count_ops(5);  // cell lookup, good test, mask updates
      int i = rock_at(s.x[r], s.y[r]);
      if (i < 0) {
        reward = -100;
      } else {
        if ((s.good >> i) & 1u) {
          reward = 10;
          s.good &= ~(1u << i);
        } else {
          reward = -10;
        }
        s.sampled |= 1u << i;
      }
    } else {  // sense rock i
      count_ops(10);  // index, dx, dy, d^2, threshold compare, truth test, reading
      int i = a - 5;
      int dx = s.x[r] - rock_x[i], dy = s.y[r] - rock_y[i];
      int d2 = dx * dx + dy * dy;
      Block4 rnd = scenario_random(seed, s.scen, (uint32_t)depth, kPurposeSensor, (uint32_t)r, plan_step);
      bool correct = (uint64_t)rnd.w[0] < thresh[d2];
      bool is_good = (s.good >> i) & 1u;
      bool says_good = correct ? is_good : !is_good;
      *z = says_good ? 1 : 2;
    }
    return reward;
  }

  // g(s, a, phi_depth): successor state, observation key, reward.
  Real step(const RSState& s, int a, int depth, RSState& out, uint64_t* key) const {
    out = s;
    int reward = 0, z0 = 0, z1 = 0;
    if (robots == 1) {
      reward += robot_step(out, 0, a, depth, &z0);
      *key = (uint64_t)z0;
    } else {
      int a0 = a / actions_per_robot(), a1 = a % actions_per_robot();
      reward += robot_step(out, 0, a0, depth, &z0);
      reward += robot_step(out, 1, a1, depth, &z1);
      *key = (uint64_t)(z0 * 3 + z1);
    }
    count_ops(robots == 1 ? 2 : 6);  // key, terminal test (joint: split action, sum)
    if (terminal(out)) *key |= kTerminalBit;
    return (Real)reward;
  }

  // Readings of the robots encoded in an observation key (for belief counters).
  void observe(Hist& h, int a, uint64_t key) const {
    int z = (int)(key & ~kTerminalBit);
    count_ops(2 * robots);
    int acts[2], zs[2];
    if (robots == 1) {
      acts[0] = a;
      zs[0] = z;
    } else {
      acts[0] = a / actions_per_robot();
      acts[1] = a % actions_per_robot();
      zs[0] = z / 3;
      zs[1] = z % 3;
    }
    for (int r = 0; r < robots; ++r) {
      if (acts[r] >= 5 && zs[r] != 0) {
        int i = acts[r] - 5;
        int v = h.c[i] + (zs[r] == 1 ? 1 : -1);
        if (v > 127) v = 127;
        if (v < -127) v = -127;
        h.c[i] = (int8_t)v;
      }
    }
  }

  // Heuristic default policy of one robot: sample a believed-good rock it
  // stands on, else walk to the nearest believed-good unsampled rock
  // (Manhattan distance, lowest index on ties, x-move before y-move), else
  // walk east. "Believed good" = counter > 0 and not yet sampled.
  int robot_policy(const RSState& s, int r, const Hist& h) const {
    count_ops(1);
    if (s.exited[r]) return 0;
    int best = -1, bestd = 1 << 30;
    count_ops(4);  // believed-good mask of the counters and sampled rocks, direction choice
    for (int i = 0; i < m; ++i) {
      if (h.c[i] > 0 && !((s.sampled >> i) & 1u)) {
        count_ops(8);  // |dx| + |dy|, compare, two selects
        int d = std::abs(s.x[r] - rock_x[i]) + std::abs(s.y[r] - rock_y[i]);
        if (d < bestd) {
          bestd = d;
          best = i;
        }
      }
    }
    if (best < 0) return 1;
    if (bestd == 0) return 4;
    if (rock_x[best] > s.x[r]) return 1;
    if (rock_x[best] < s.x[r]) return 3;
    if (rock_y[best] > s.y[r]) return 0;
    return 2;
  }

  int policy(const RSState& s, const Hist& h) const {
    if (robots == 1) return robot_policy(s, 0, h);
    return robot_policy(s, 0, h) * actions_per_robot() + robot_policy(s, 1, h);
  }

  // Upper-bound heuristic u(phi): every good rock collected at its nearest
  // robot's Manhattan distance, plus every robot's exit reward after walking
  // straight east. Summed in rock order, then robot order.
  Real upper(const RSState& s) const {
    count_ops(1);
    if (terminal(s)) return (Real)0;
    Real u = (Real)0;
    for (int i = 0; i < m; ++i) {
      if (!((s.good >> i) & 1u)) continue;
      count_ops(2 + 6 * robots);  // per robot |dx|+|dy| and min; 10*G[d] and the sum
      int bestd = 1 << 30;
      for (int r = 0; r < robots; ++r) {
        if (s.exited[r]) continue;
        int d = std::abs(s.x[r] - rock_x[i]) + std::abs(s.y[r] - rock_y[i]);
        if (d < bestd) bestd = d;
      }
      u = u + (Real)10 * G[bestd];
    }
    for (int r = 0; r < robots; ++r)
      if (!s.exited[r]) u = u + (Real)10 * G[n - 1 - s.x[r]];
    count_ops(4 * robots);
    return u;
  }

  // Value past the horizon: every robot walks east (achievable).
  Real tail(const RSState& s) const {
    Real l = (Real)0;
    count_ops(4 * robots);
    for (int r = 0; r < robots; ++r)
      if (!s.exited[r]) l = l + (Real)10 * G[n - 1 - s.x[r]];
    return l;
  }

  // Words of one scenario in the state block format (field-major, 5 fields):
  // f0/f1 robot r as x | y<<8 | exited<<16, f2 good mask, f3 sampled mask,
  // f4 scenario id.
  static const int kWords = 5;
  RSState unpack(const uint32_t* block, int cap, int i) const {
    RSState s;
    for (int r = 0; r < 2; ++r) {
      uint32_t w = block[r * cap + i];
      s.x[r] = (int)(w & 0xFF);
      s.y[r] = (int)((w >> 8) & 0xFF);
      s.exited[r] = (w >> 16) & 1u;
    }
    if (robots == 1) {
      s.x[1] = s.y[1] = 0;
      s.exited[1] = true;
    }
    s.good = block[2 * cap + i];
    s.sampled = block[3 * cap + i];
    s.scen = block[4 * cap + i];
    return s;
  }
  void pack(const RSState& s, uint32_t* block, int cap, int i) const {
    for (int r = 0; r < 2; ++r) {
      uint32_t w = 0;
      if (r < robots) w = (uint32_t)s.x[r] | ((uint32_t)s.y[r] << 8) | ((uint32_t)s.exited[r] << 16);
      block[r * cap + i] = w;
    }
    block[2 * cap + i] = s.good;
    block[3 * cap + i] = s.sampled;
    block[4 * cap + i] = s.scen;
  }
};

}  // namespace orc
