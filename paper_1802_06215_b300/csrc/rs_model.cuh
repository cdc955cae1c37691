// Rock Sample with R robots (R = 1 "grid", R = 2 "multigrid"): the device
// step function g, observation bookkeeping, heuristic default policy and
// bound heuristics of the multi-agent Rock Sample task (Sec. IV-A).
//
// Rules and readings (the same as the library's documentation states):
// per-robot actions 0 N (y+1), 1 E (x+1), 2 S (y-1), 3 W (x-1), 4 Sample,
// 5+i Sense rock i, joint action a0 * (5+m) + a1; moving off the N/S/W border
// or sampling where no rock lies costs -100 and does nothing; E from the last
// column exits (+10); sampling a good rock gives +10 and makes it bad, a bad
// one -10; robots act in index order; exited robots do nothing; a reading of
// rock i is right iff the Philox word u (purpose 2, element = robot) is below
// the threshold of the squared Euclidean distance; observation per robot
// 0 none / 1 good / 2 bad, joint z0 * 3 + z1, bit 62 = terminal.
#pragma once
#include "common.cuh"

namespace dsp {

// Scenario state in registers: robot words x | y<<8 | exited<<16, rock masks,
// scenario id.
struct RSS {
  uint32_t pos[2];
  uint32_t good, sampled, scen;
};

// Constants a CTA keeps in shared memory.
struct RSShared {
  float G[kGammaLen];
  int rock_xy[kMaxRocks];
  uint8_t cell_rock[kMaxSide * kMaxSide];
};

template <int R>
struct RSModel {
  const RSShared* sh;
  const uint64_t* thresh;  // global, read through the read-only path
  const uint16_t* nkey;    // policy keys of (rock, cell), in shared or global memory
  int n, nn, m, per, D;
  uint64_t seed;
  uint32_t plan_step;

  __device__ __forceinline__ bool terminal(const RSS& s) const {
    bool t = (s.pos[0] >> 16) & 1u;
    if (R == 2) t = t && ((s.pos[1] >> 16) & 1u);
    return t;
  }

  // One robot's part of g. A Sense reading draws the scenario's sensor word
  // (Philox purpose 2, element r) unless the caller passes it in `sense`:
  // the word depends on the scenario and the depth only, so a leaf's actions
  // share it.
  __device__ __forceinline__ int robot_step(RSS& s, int r, int a, int depth, int& z,
                                            const uint32_t* sense = nullptr) const {
    z = 0;
    uint32_t p = s.pos[r];
    if ((p >> 16) & 1u) return 0;
    int x = (int)(p & 0xFFu), y = (int)((p >> 8) & 0xFFu);
    int reward = 0;
    if (a == 0) {
      if (y == n - 1) reward = -100; else y += 1;
    } else if (a == 1) {
      if (x == n - 1) { reward = 10; p |= 1u << 16; } else x += 1;
    } else if (a == 2) {
      if (y == 0) reward = -100; else y -= 1;
    } else if (a == 3) {
      if (x == 0) reward = -100; else x -= 1;
    } else if (a == 4) {
      int i = sh->cell_rock[y * n + x];
      if (i == 0xFF) {
        reward = -100;
      } else {
        uint32_t bit = 1u << i;
        reward = (s.good & bit) ? 10 : -10;
        s.good &= ~bit;
        s.sampled |= bit;
      }
    } else {
      int i = a - 5;
      int rx = sh->rock_xy[i] & 0xFF, ry = sh->rock_xy[i] >> 8;
      int dx = x - rx, dy = y - ry;
      const uint32_t u = sense != nullptr ? sense[r] : sense_word(s.scen, depth, r);
      bool correct = (uint64_t)u < __ldg(thresh + dx * dx + dy * dy);
      bool is_good = (s.good >> i) & 1u;
      z = (correct == is_good) ? 1 : 2;
    }
    s.pos[r] = (p & 0xFFFF0000u) | (uint32_t)x | ((uint32_t)y << 8);
    return reward;
  }

  // The sensor word of scenario `scen` for robot r at `depth`.
  __device__ __forceinline__ uint32_t sense_word(uint32_t scen, int depth, int r) const {
    return scen_random(seed, scen, (uint32_t)depth, 2u, (uint32_t)r, plan_step).x;
  }

  // g(s, a, phi_depth); returns the reward, writes the observation key. The
  // robots' sensor words may be passed in (sense_word of each robot).
  __device__ __forceinline__ float step(RSS& s, int a, int depth, uint64_t& key,
                                        const uint32_t* sense = nullptr) const {
    int z0, z1 = 0, rew;
    if (R == 1) {
      rew = robot_step(s, 0, a, depth, z0, sense);
      key = (uint64_t)z0;
    } else {
      int a0 = a / per, a1 = a - a0 * per;
      rew = robot_step(s, 0, a0, depth, z0, sense);
      rew += robot_step(s, 1, a1, depth, z1, sense);
      key = (uint64_t)(z0 * 3 + z1);
    }
    if (terminal(s)) key |= kTermBit;
    return (float)rew;
  }

  // Belief counters of the history after (a, key); `pmask` tracks which
  // counters are positive.
  __device__ __forceinline__ void observe_robot(uint32_t (&h)[8], uint32_t& pmask, int ar, int zr) const {
    if (ar >= 5 && zr != 0) {
      int i = ar - 5;
      int delta = zr == 1 ? 1 : -1;
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (k == (i >> 2)) {
          uint32_t hw[8];
          hw[k] = h[k];
          int sh8 = 8 * (i & 3);
          int v = (int)(int8_t)((hw[k] >> sh8) & 0xFFu) + delta;
          v = v > 127 ? 127 : (v < -127 ? -127 : v);
          h[k] = (hw[k] & ~(0xFFu << sh8)) | ((uint32_t)(uint8_t)(int8_t)v << sh8);
          pmask = v > 0 ? (pmask | (1u << i)) : (pmask & ~(1u << i));
        }
    }
  }
  __device__ __forceinline__ void observe(uint32_t (&h)[8], uint32_t& pmask, int a, uint64_t key) const {
    int z = (int)(key & ~kTermBit);
    if (R == 1) {
      observe_robot(h, pmask, a, z);
    } else {
      int a0 = a / per;
      observe_robot(h, pmask, a0, z / 3);
      observe_robot(h, pmask, a - a0 * per, z % 3);
    }
  }

  // Default policy of one robot: sample a believed-good rock underfoot, else
  // head for the nearest believed-good unsampled rock (Manhattan, lowest
  // index on ties, x before y), else east.
  __device__ __forceinline__ int robot_policy(const RSS& s, int r, uint32_t pmask) const {
    uint32_t p = s.pos[r];
    if ((p >> 16) & 1u) return 0;
    int x = (int)(p & 0xFFu), y = (int)((p >> 8) & 0xFFu);
    uint32_t cand = pmask & ~s.sampled;
    int best = -1, bestd = 1 << 30;
    while (cand) {
      int i = __ffs(cand) - 1;
      cand &= cand - 1;
      int rxy = sh->rock_xy[i];
      int d = abs(x - (rxy & 0xFF)) + abs(y - (rxy >> 8));
      if (d < bestd) {
        bestd = d;
        best = i;
      }
    }
    if (best < 0) return 1;
    if (bestd == 0) return 4;
    int rxy = sh->rock_xy[best];
    int rx = rxy & 0xFF, ry = rxy >> 8;
    if (rx > x) return 1;
    if (rx < x) return 3;
    if (ry > y) return 0;
    return 2;
  }
  __device__ __forceinline__ int policy(const RSS& s, uint32_t pmask) const {
    if (R == 1) return robot_policy(s, 0, pmask);
    return robot_policy(s, 0, pmask) * per + robot_policy(s, 1, pmask);
  }

  // u(phi): each good rock (of the m) at its nearest live robot's Manhattan
  // distance, read from the policy-key table, then each live robot's exit,
  // summed in that order in FP32.
  __device__ __forceinline__ float upper(const RSS& s) const {
    if (terminal(s)) return 0.0f;
    int cell[R];
    bool live[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t p = s.pos[r];
      live[r] = !((p >> 16) & 1u);
      cell[r] = (int)(p & 0xFFu) + (int)((p >> 8) & 0xFFu) * n;
    }
    float u = 0.0f;
    uint32_t g = s.good & (m == 32 ? 0xFFFFFFFFu : (1u << m) - 1u);
    while (g) {
      const int i = __ffs(g) - 1;
      g &= g - 1;
      int bestd = 1 << 30;
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (live[r]) bestd = min(bestd, (int)nkey[i * nn + cell[r]] >> 7);
      u = __fadd_rn(u, __fmul_rn(10.0f, sh->G[bestd]));
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
      if (live[r]) u = __fadd_rn(u, __fmul_rn(10.0f, sh->G[n - 1 - (int)(s.pos[r] & 0xFFu)]));
    return u;
  }

  // Past the horizon every live robot walks east.
  __device__ __forceinline__ float tail(const RSS& s) const {
    float l = 0.0f;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint32_t p = s.pos[r];
      if (!((p >> 16) & 1u)) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - (int)(p & 0xFFu)]));
    }
    return l;
  }

  // Eq. lb for one scenario from depth t0; pmask marks the rocks whose belief
  // counter is positive. The heuristic policy never senses, so the counters
  // stay fixed and the step only meets moves and Sample. A zero reward adds
  // +0.0 to v, which is never -0.0, so skipping it (and its discount-table
  // load) leaves v unchanged.
  __device__ __forceinline__ float rollout(RSS s, uint32_t pmask, int t0, unsigned long long& steps) const {
    if constexpr (R == 1)
      return rollout_one(s, pmask, t0, steps);
    else
      return rollout_two(s, pmask, t0, steps);
  }

  // The heuristic's decision for one robot at cell y*n+x among the non-empty
  // rock set cand: the smallest key of the model's policy-key table, i.e. the
  // nearest rock (Manhattan, lowest index on ties) with its distance and the
  // move toward it. Rocks are visited from the highest index down; the key
  // order does the tie-breaking.
  __device__ __forceinline__ int nearest_key(int cell, uint32_t cand) const {
    int key = 0xFFFF;
    const uint16_t* col = nkey + cell;
    do {
      const int i = 31 - __clz(cand);
      cand ^= 1u << i;
      key = min(key, (int)col[i * nn]);
    } while (cand);
    return key;
  }

  // The heuristic's target of one robot at cell y*n+x among the non-empty
  // rock set cand (the smallest policy key: nearest rock, lowest index on
  // ties): its coordinates and bit.
  __device__ __forceinline__ void target(int x, int y, uint32_t cand, int& tx, int& ty, uint32_t& tbit) const {
    const int i = (nearest_key(y * n + x, cand) >> 2) & 31;
    const int rxy = sh->rock_xy[i];
    tx = rxy & 0xFF;
    ty = rxy >> 8;
    tbit = 1u << i;
  }

  // One heuristic step of one robot with its target carried between steps
  // (no target: E, the exit from the last column). Between two samples the
  // target cannot change: a step toward it lowers its Manhattan distance by
  // one and any other rock's by at most one, so no other rock overtakes it,
  // and on a tie the lower index that already won keeps winning. So the
  // policy's action equals a fresh scan's at every step; the scan runs only
  // after a sample changed the rock set. On the target's cell: Sample (the
  // rock leaves the set, the robot retargets). Else the move toward it, x
  // before y. Returns the reward.
  __device__ __forceinline__ int heuristic_step(int& x, int& y, bool& ex, int& tx, int& ty, uint32_t& tbit,
                                                uint32_t& good, uint32_t& cand) const {
    if (ex) return 0;
    if (tbit == 0) {
      if (x == n - 1) {
        ex = true;
        return 10;
      }
      x += 1;
      return 0;
    }
    if (x == tx && y == ty) {
      const int r = (good & tbit) ? 10 : -10;
      good &= ~tbit;
      cand &= ~tbit;
      tbit = 0;
      return r;
    }
    if (x != tx)
      x += tx > x ? 1 : -1;
    else
      y += ty > y ? 1 : -1;
    return 0;
  }

  // Steps before a robot's next event under the carried target: the moves to
  // the target cell (Manhattan distance; its Sample follows), or with no
  // target the E moves to the last column (its exit follows); never for an
  // exited robot.
  __device__ __forceinline__ int event_steps(int x, int y, bool ex, int tx, int ty, uint32_t tbit) const {
    if (ex) return 1 << 30;
    if (tbit == 0) return n - 1 - x;
    return abs(tx - x) + abs(ty - y);
  }

  // k of those moves at once (k <= event_steps): toward the target, x before
  // y, or east.
  __device__ __forceinline__ void move_steps(int& x, int& y, bool ex, int tx, int ty, uint32_t tbit, int k) const {
    if (ex || k == 0) return;
    if (tbit == 0) {
      x += k;
      return;
    }
    const int mx = min(k, abs(tx - x));
    x += tx > x ? mx : -mx;
    const int my = k - mx;
    y += ty > y ? my : -my;
  }

  // The same rollout for two robots with the state unpacked into registers:
  // both robots decide on the state before the step (the joint heuristic
  // policy), robot 0 acts first (a rock both stand on is sampled by robot 0,
  // robot 1's Sample then finds it bad), an exited robot does nothing, the
  // rewards are summed, and the world ends when both have exited. Targets
  // are carried between steps (heuristic_step). A sample removes one rock
  // from the shared set; the argmin over the rest is unchanged unless it was
  // that rock, so a robot retakes its target, before the next step, exactly
  // when its target has left the set. Between events (a Sample, an exit)
  // the steps are moves only and are taken together.
  __device__ __forceinline__ float rollout_two(RSS s, uint32_t pmask, int t0, unsigned long long& steps) const {
    int x0 = (int)(s.pos[0] & 0xFFu), y0 = (int)((s.pos[0] >> 8) & 0xFFu);
    int x1 = (int)(s.pos[1] & 0xFFu), y1 = (int)((s.pos[1] >> 8) & 0xFFu);
    bool ex0 = (s.pos[0] >> 16) & 1u, ex1 = (s.pos[1] >> 16) & 1u;
    uint32_t good = s.good, cand = pmask & ~s.sampled;  // cand loses each sampled rock
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    uint32_t tb0 = 0, tb1 = 0;
    float v = 0.0f;
    int t = t0;
    while (t < D && !(ex0 && ex1)) {
      if (!ex0 && (tb0 & cand) == 0) {
        tb0 = 0;
        if (cand != 0) target(x0, y0, cand, tx0, ty0, tb0);
      }
      if (!ex1 && (tb1 & cand) == 0) {
        tb1 = 0;
        if (cand != 0) target(x1, y1, cand, tx1, ty1, tb1);
      }
      // Until the first robot's next event (its Sample on the target cell,
      // or its exit from the last column) both robots only move, one cell
      // per step, and no target changes: jump those steps (their rewards
      // are 0, which leaves v as it is) and move both robots there at once.
      const int k = min(min(event_steps(x0, y0, ex0, tx0, ty0, tb0), event_steps(x1, y1, ex1, tx1, ty1, tb1)), D - t);
      move_steps(x0, y0, ex0, tx0, ty0, tb0, k);
      move_steps(x1, y1, ex1, tx1, ty1, tb1, k);
      t += k;
      if (t >= D) break;
      // the event step: robot 1's target was taken on the state before
      // robot 0 acts, so its Sample of a rock robot 0 just took finds it
      // bad, as the joint step's order has it
      int reward = heuristic_step(x0, y0, ex0, tx0, ty0, tb0, good, cand);
      reward += heuristic_step(x1, y1, ex1, tx1, ty1, tb1, good, cand);
      if (reward != 0) v = __fadd_rn(v, __fmul_rn(sh->G[t - t0], (float)reward));
      t += 1;
    }
    steps += (unsigned long long)(t - t0);
    if (!(ex0 && ex1)) {
      float l = 0.0f;
      if (!ex0) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x0]));
      if (!ex1) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x1]));
      v = __fadd_rn(v, __fmul_rn(sh->G[D - t0], l));
    }
    return v;
  }

  // The same rollout for one robot with the state unpacked into registers.
  // The heuristic policy only moves and samples, and its moves never leave
  // the map except E from the last column (the exit). With the target
  // carried (heuristic_step), a rollout is a run of segments, each step of
  // which is one g step: the moves toward the target, one cell per step, x
  // before y (the direction along each axis is fixed for the segment), then
  // Sample on it, which takes the rock out of the set and retakes the
  // target; with no target left, E until the exit. Rewards, their order and
  // the step count are those of step() and policy() at every step.
  __device__ __forceinline__ float rollout_one(RSS s, uint32_t pmask, int t0, unsigned long long& steps) const {
    const uint32_t p0 = s.pos[0];
    int x = (int)(p0 & 0xFFu), y = (int)((p0 >> 8) & 0xFFu);
    bool ex = (p0 >> 16) & 1u;
    uint32_t good = s.good, cand = pmask & ~s.sampled;  // cand loses each sampled rock
    float v = 0.0f;
    int t = t0;
    if (!ex) {
      while (t < D) {
        if (cand == 0) {
          // E each step; from the last column E exits (+10)
          const int ke = min(n - 1 - x, D - t);
          x += ke;
          t += ke;
          if (t < D) {
            v = __fadd_rn(v, __fmul_rn(sh->G[t - t0], 10.0f));
            ex = true;
            ++t;
          }
          break;
        }
        int tx, ty;
        uint32_t tbit;
        target(x, y, cand, tx, ty, tbit);
        const int sx = tx > x ? 1 : -1, sy = ty > y ? 1 : -1;
        // one move per step toward the target: x first, then y (taken
        // together, up to the horizon)
        const int kx = min(abs(tx - x), D - t);
        x += sx * kx;
        t += kx;
        const int ky = min(abs(ty - y), D - t);
        y += sy * ky;
        t += ky;
        if (t >= D) break;
        // on the target's cell: Sample
        const float r = (good & tbit) ? 10.0f : -10.0f;
        good &= ~tbit;
        cand &= ~tbit;
        v = __fadd_rn(v, __fmul_rn(sh->G[t - t0], r));
        ++t;
      }
    }
    steps += (unsigned long long)(t - t0);
    if (!ex) v = __fadd_rn(v, __fmul_rn(sh->G[D - t0], __fmul_rn(10.0f, sh->G[n - 1 - x])));
    return v;
  }

  // heuristic_step for two scenarios of one child that share the robots'
  // positions, targets and candidate set: the moves and exits are the same,
  // and a Sample gives each scenario its own reward (added to ra, rb) and
  // clears the rock in both good masks.
  __device__ __forceinline__ void heuristic_step2(int& x, int& y, bool& ex, int tx, int ty, uint32_t& tbit,
                                                  uint32_t& good_a, uint32_t& good_b, uint32_t& cand, int& ra,
                                                  int& rb) const {
    if (ex) return;
    if (tbit == 0) {
      if (x == n - 1) {
        ex = true;
        ra += 10;
        rb += 10;
        return;
      }
      x += 1;
      return;
    }
    if (x == tx && y == ty) {
      ra += (good_a & tbit) ? 10 : -10;
      rb += (good_b & tbit) ? 10 : -10;
      good_a &= ~tbit;
      good_b &= ~tbit;
      cand &= ~tbit;
      tbit = 0;
      return;
    }
    if (x != tx)
      x += tx > x ? 1 : -1;
    else
      y += ty > y ? 1 : -1;
  }

  // heuristic_step2 for K scenarios of one child: the same moves and exits,
  // each scenario's own reward at a Sample (added to r[k]), the rock cleared
  // in every good mask.
  template <int K>
  __device__ __forceinline__ void heuristic_stepK(int& x, int& y, bool& ex, int tx, int ty, uint32_t& tbit,
                                                  uint32_t (&good)[K], uint32_t& cand, int (&r)[K]) const {
    if (ex) return;
    if (tbit == 0) {
      if (x == n - 1) {
        ex = true;
#pragma unroll
        for (int k = 0; k < K; ++k) r[k] += 10;
        return;
      }
      x += 1;
      return;
    }
    if (x == tx && y == ty) {
#pragma unroll
      for (int k = 0; k < K; ++k) {
        r[k] += (good[k] & tbit) ? 10 : -10;
        good[k] &= ~tbit;
      }
      cand &= ~tbit;
      tbit = 0;
      return;
    }
    if (x != tx)
      x += tx > x ? 1 : -1;
    else
      y += ty > y ? 1 : -1;
  }

  // rollout_two for K scenarios of one child (rollout_two2's joint
  // trajectory, each scenario's rewards added as rollout_two adds them, a
  // zero reward skipped); steps_each scenarios' steps are counted.
  template <int K>
  __device__ __forceinline__ void rollout_twoK(uint32_t p0, uint32_t p1, const uint32_t (&good_in)[K], uint32_t cand,
                                               int t0, float (&v)[K], unsigned long long steps_each,
                                               unsigned long long& steps) const {
    int x0 = (int)(p0 & 0xFFu), y0 = (int)((p0 >> 8) & 0xFFu);
    int x1 = (int)(p1 & 0xFFu), y1 = (int)((p1 >> 8) & 0xFFu);
    bool ex0 = (p0 >> 16) & 1u, ex1 = (p1 >> 16) & 1u;
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    uint32_t tb0 = 0, tb1 = 0;
    uint32_t good[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      good[k] = good_in[k];
      v[k] = 0.0f;
    }
    int t = t0;
    while (t < D && !(ex0 && ex1)) {
      if (!ex0 && (tb0 & cand) == 0) {
        tb0 = 0;
        if (cand != 0) target(x0, y0, cand, tx0, ty0, tb0);
      }
      if (!ex1 && (tb1 & cand) == 0) {
        tb1 = 0;
        if (cand != 0) target(x1, y1, cand, tx1, ty1, tb1);
      }
      const int k = min(min(event_steps(x0, y0, ex0, tx0, ty0, tb0), event_steps(x1, y1, ex1, tx1, ty1, tb1)), D - t);
      move_steps(x0, y0, ex0, tx0, ty0, tb0, k);
      move_steps(x1, y1, ex1, tx1, ty1, tb1, k);
      t += k;
      if (t >= D) break;
      int r[K];
#pragma unroll
      for (int q = 0; q < K; ++q) r[q] = 0;
      heuristic_stepK<K>(x0, y0, ex0, tx0, ty0, tb0, good, cand, r);
      heuristic_stepK<K>(x1, y1, ex1, tx1, ty1, tb1, good, cand, r);
      const float g = sh->G[t - t0];
#pragma unroll
      for (int q = 0; q < K; ++q)
        if (r[q] != 0) v[q] = __fadd_rn(v[q], __fmul_rn(g, (float)r[q]));
      t += 1;
    }
    steps += steps_each * (unsigned long long)(t - t0);
    if (!(ex0 && ex1)) {
      float l = 0.0f;
      if (!ex0) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x0]));
      if (!ex1) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x1]));
      const float tl = __fmul_rn(sh->G[D - t0], l);
#pragma unroll
      for (int q = 0; q < K; ++q) v[q] = __fadd_rn(v[q], tl);
    }
  }

  // rollout_two for two scenarios of one child: one joint trajectory (the
  // robots' moves read no rock state), each scenario's rewards at the event
  // steps added as rollout_two adds them (a zero reward skipped); both
  // rollouts' steps are counted.
  __device__ __forceinline__ void rollout_two2(uint32_t p0, uint32_t p1, uint32_t good_a, uint32_t good_b,
                                               uint32_t cand, int t0, float& va, float& vb,
                                               unsigned long long& steps) const {
    int x0 = (int)(p0 & 0xFFu), y0 = (int)((p0 >> 8) & 0xFFu);
    int x1 = (int)(p1 & 0xFFu), y1 = (int)((p1 >> 8) & 0xFFu);
    bool ex0 = (p0 >> 16) & 1u, ex1 = (p1 >> 16) & 1u;
    int tx0 = 0, ty0 = 0, tx1 = 0, ty1 = 0;
    uint32_t tb0 = 0, tb1 = 0;
    va = 0.0f;
    vb = 0.0f;
    int t = t0;
    while (t < D && !(ex0 && ex1)) {
      if (!ex0 && (tb0 & cand) == 0) {
        tb0 = 0;
        if (cand != 0) target(x0, y0, cand, tx0, ty0, tb0);
      }
      if (!ex1 && (tb1 & cand) == 0) {
        tb1 = 0;
        if (cand != 0) target(x1, y1, cand, tx1, ty1, tb1);
      }
      const int k = min(min(event_steps(x0, y0, ex0, tx0, ty0, tb0), event_steps(x1, y1, ex1, tx1, ty1, tb1)), D - t);
      move_steps(x0, y0, ex0, tx0, ty0, tb0, k);
      move_steps(x1, y1, ex1, tx1, ty1, tb1, k);
      t += k;
      if (t >= D) break;
      int ra = 0, rb = 0;
      heuristic_step2(x0, y0, ex0, tx0, ty0, tb0, good_a, good_b, cand, ra, rb);
      heuristic_step2(x1, y1, ex1, tx1, ty1, tb1, good_a, good_b, cand, ra, rb);
      const float g = sh->G[t - t0];
      if (ra != 0) va = __fadd_rn(va, __fmul_rn(g, (float)ra));
      if (rb != 0) vb = __fadd_rn(vb, __fmul_rn(g, (float)rb));
      t += 1;
    }
    steps += 2ull * (unsigned long long)(t - t0);
    if (!(ex0 && ex1)) {
      float l = 0.0f;
      if (!ex0) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x0]));
      if (!ex1) l = __fadd_rn(l, __fmul_rn(10.0f, sh->G[n - 1 - x1]));
      const float tl = __fmul_rn(sh->G[D - t0], l);
      va = __fadd_rn(va, tl);
      vb = __fadd_rn(vb, tl);
    }
  }

  // rollout_one for K scenarios of one child (the same position, candidate
  // set and depth, so the same trajectory); each scenario adds its own
  // reward at each Sample with the operations and in the order rollout_one
  // uses. `live` marks the scenarios whose steps are counted.
  template <int K>
  __device__ __forceinline__ void rollout_oneK(uint32_t p0, const uint32_t (&good)[K], uint32_t cand, int t0,
                                               float (&v)[K], unsigned long long steps_each,
                                               unsigned long long& steps) const {
    int x = (int)(p0 & 0xFFu), y = (int)((p0 >> 8) & 0xFFu);
    bool ex = (p0 >> 16) & 1u;
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0f;
    int t = t0;
    if (!ex) {
      while (t < D) {
        if (cand == 0) {
          const int ke = min(n - 1 - x, D - t);
          x += ke;
          t += ke;
          if (t < D) {
            const float e = __fmul_rn(sh->G[t - t0], 10.0f);
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] = __fadd_rn(v[k], e);
            ex = true;
            ++t;
          }
          break;
        }
        int tx, ty;
        uint32_t tbit;
        target(x, y, cand, tx, ty, tbit);
        const int sx = tx > x ? 1 : -1, sy = ty > y ? 1 : -1;
        const int kx = min(abs(tx - x), D - t);
        x += sx * kx;
        t += kx;
        const int ky = min(abs(ty - y), D - t);
        y += sy * ky;
        t += ky;
        if (t >= D) break;
        const float g = __fmul_rn(sh->G[t - t0], 10.0f);
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = __fadd_rn(v[k], (good[k] & tbit) ? g : -g);
        cand &= ~tbit;
        ++t;
      }
    }
    steps += steps_each * (unsigned long long)(t - t0);
    if (!ex) {
      const float tl = __fmul_rn(sh->G[D - t0], __fmul_rn(10.0f, sh->G[n - 1 - x]));
#pragma unroll
      for (int k = 0; k < K; ++k) v[k] = __fadd_rn(v[k], tl);
    }
  }

  // rollout_one for two scenarios of one child: the same position and
  // candidate set, so the same trajectory (the heuristic's moves read no
  // rock state); each scenario adds its own reward at each Sample, with the
  // operations and in the order rollout_one uses, and both rollouts' steps
  // are counted. (A sampled rock leaves the candidate set, so no later
  // reward reads its good bit again.)
  __device__ __forceinline__ void rollout_one2(uint32_t p0, uint32_t good_a, uint32_t good_b, uint32_t cand, int t0,
                                               float& va, float& vb, unsigned long long& steps) const {
    int x = (int)(p0 & 0xFFu), y = (int)((p0 >> 8) & 0xFFu);
    bool ex = (p0 >> 16) & 1u;
    va = 0.0f;
    vb = 0.0f;
    int t = t0;
    if (!ex) {
      while (t < D) {
        if (cand == 0) {
          const int ke = min(n - 1 - x, D - t);
          x += ke;
          t += ke;
          if (t < D) {
            const float e = __fmul_rn(sh->G[t - t0], 10.0f);
            va = __fadd_rn(va, e);
            vb = __fadd_rn(vb, e);
            ex = true;
            ++t;
          }
          break;
        }
        int tx, ty;
        uint32_t tbit;
        target(x, y, cand, tx, ty, tbit);
        const int sx = tx > x ? 1 : -1, sy = ty > y ? 1 : -1;
        const int kx = min(abs(tx - x), D - t);
        x += sx * kx;
        t += kx;
        const int ky = min(abs(ty - y), D - t);
        y += sy * ky;
        t += ky;
        if (t >= D) break;
        const float g = sh->G[t - t0];
        va = __fadd_rn(va, __fmul_rn(g, (good_a & tbit) ? 10.0f : -10.0f));
        vb = __fadd_rn(vb, __fmul_rn(g, (good_b & tbit) ? 10.0f : -10.0f));
        cand &= ~tbit;
        ++t;
      }
    }
    steps += 2ull * (unsigned long long)(t - t0);
    if (!ex) {
      const float tl = __fmul_rn(sh->G[D - t0], __fmul_rn(10.0f, sh->G[n - 1 - x]));
      va = __fadd_rn(va, tl);
      vb = __fadd_rn(vb, tl);
    }
  }

  __device__ __forceinline__ RSS load(const uint32_t* block, int cap, int i) const {
    RSS s;
    s.pos[0] = block[i];
    s.pos[1] = R == 2 ? block[cap + i] : 0u;
    s.good = block[2 * cap + i];
    s.sampled = block[3 * cap + i];
    s.scen = block[4 * cap + i];
    return s;
  }
  __device__ __forceinline__ void store(const RSS& s, uint32_t* block, int cap, int i) const {
    block[i] = s.pos[0];
    block[cap + i] = R == 2 ? s.pos[1] : 0u;
    block[2 * cap + i] = s.good;
    block[3 * cap + i] = s.sampled;
    block[4 * cap + i] = s.scen;
  }
};

__device__ __forceinline__ uint32_t positive_mask(const uint32_t (&h)[8], int m) {
  uint32_t pm = 0;
#pragma unroll
  for (int i = 0; i < kMaxRocks; ++i)
    if (i < m && (int)(int8_t)((h[i >> 2] >> (8 * (i & 3))) & 0xFFu) > 0) pm |= 1u << i;
  return pm;
}

}  // namespace dsp
