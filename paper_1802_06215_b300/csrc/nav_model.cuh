// Navigation in a partially known map (Sec. IV-A) on the device: one thread
// per scenario, the state in registers (position, terminal flag, the
// scenario's occupancy map of n*n <= 256 cells in up to 8 words, scenario id).
//
// Rules (the same as the library's documentation states): actions 0 stay,
// 1 N (y-1), 2 NE, 3 E (x+1), 4 SE, 5 S (y+1), 6 SW, 7 W, 8 NW. Staying costs
// 0.2. A move fails when the Philox word (purpose 1, element 0) is below
// floor(fail_p * 2^32): the robot stays and pays 0.1. A move off the map or
// onto an occupied cell is a crash: -1, the robot stays. Entering the goal
// (n/2, n-1) gives +20 and ends the world; any other move costs 0.1. The
// observation is one bit per neighbour in action order (bit k-1 for action k,
// 1 = occupied, off-map cells occupied), each flipped when its Philox word
// (purpose 2, elements 0 and 1, four words each) is below floor(sense_p *
// 2^32); a terminal outcome observes nothing (key bit 62). The default policy
// sees only the last reading: the first of S, SE, SW, E, W, NE, NW, N read
// free, else stay. u = 20 gamma^(d-1), d the 8-connected distance to the goal
// through the open gate (the free one of x = n/4 and n-1-n/4 on the wall row
// n/2) while the robot is above the wall; the horizon tail is 0.
#pragma once
#include "common.cuh"

namespace dsp {

constexpr int kNavMaxWords = 8;  // occupancy words: n * n <= 256

struct NavS {
  int x, y;
  bool term;
  uint32_t occ[kNavMaxWords];
  uint32_t scen;
};

struct NavModel {
  const float* G;  // gamma^k in shared memory
  int n, mw, D;
  uint64_t seed, fail_thresh, sense_thresh;
  uint32_t plan_step;

  __device__ __forceinline__ static int dx(int a) {
    // stay, N, NE, E, SE, S, SW, W, NW
    return a == 0 ? 0 : (a == 1 || a == 5) ? 0 : (a <= 4 ? 1 : -1);
  }
  __device__ __forceinline__ static int dy(int a) {
    return a == 0 ? 0 : (a == 3 || a == 7) ? 0 : ((a <= 2 || a == 8) ? -1 : 1);
  }

  __device__ __forceinline__ bool occupied(const NavS& s, int x, int y) const {
    if (x < 0 || y < 0 || x >= n || y >= n) return true;
    const int c = y * n + x;
    const int k = c >> 5;
    // a select tree over the eight words keeps the map in registers
    const uint32_t a01 = (k & 1) ? s.occ[1] : s.occ[0];
    const uint32_t a23 = (k & 1) ? s.occ[3] : s.occ[2];
    const uint32_t a45 = (k & 1) ? s.occ[5] : s.occ[4];
    const uint32_t a67 = (k & 1) ? s.occ[7] : s.occ[6];
    const uint32_t b03 = (k & 2) ? a23 : a01;
    const uint32_t b47 = (k & 2) ? a67 : a45;
    const uint32_t w = (k & 4) ? b47 : b03;
    return (w >> (c & 31)) & 1u;
  }

  __device__ __forceinline__ NavS load(const uint32_t* b, int cap, int i) const {
    NavS s;
    const uint32_t w = b[i];
    s.x = (int)(w & 0xFFu);
    s.y = (int)((w >> 8) & 0xFFu);
    s.term = (w >> 16) & 1u;
#pragma unroll
    for (int k = 0; k < kNavMaxWords; ++k) s.occ[k] = k < mw ? b[(size_t)(1 + k) * cap + i] : 0u;
    s.scen = b[(size_t)(1 + mw) * cap + i];
    return s;
  }
  __device__ __forceinline__ void store(const NavS& s, uint32_t* b, int cap, int i) const {
    b[i] = (uint32_t)s.x | ((uint32_t)s.y << 8) | ((uint32_t)s.term << 16);
#pragma unroll
    for (int k = 0; k < kNavMaxWords; ++k)
      if (k < mw) b[(size_t)(1 + k) * cap + i] = s.occ[k];
    b[(size_t)(1 + mw) * cap + i] = s.scen;
  }

  // Bit k-1 of the observation: neighbour k's occupancy, flipped by its word.
  __device__ __forceinline__ uint32_t reading(const NavS& s, int k, uint32_t u) const {
    const bool occ = occupied(s, s.x + dx(k), s.y + dy(k));
    const bool flip = (uint64_t)u < sense_thresh;
    return (uint32_t)(occ != flip) << (k - 1);
  }

  // g(s, a, phi_t); returns the reward, writes the observation key.
  __device__ __forceinline__ float step(NavS& s, int a, int t, uint64_t& key) const {
    if (s.term) {
      key = kTermBit;
      return 0.0f;
    }
    float r;
    if (a == 0) {
      r = -0.2f;
    } else {
      const uint32_t u = scen_random(seed, s.scen, (uint32_t)t, 1u, 0u, plan_step).x;
      if ((uint64_t)u < fail_thresh) {
        r = -0.1f;
      } else {
        const int nx = s.x + dx(a), ny = s.y + dy(a);
        if (occupied(s, nx, ny)) {
          r = -1.0f;
        } else {
          s.x = nx;
          s.y = ny;
          if (nx == n / 2 && ny == n - 1) {
            s.term = true;
            r = 20.0f;
          } else {
            r = -0.1f;
          }
        }
      }
    }
    if (s.term) {
      key = kTermBit;
      return r;
    }
    const U4 w0 = scen_random(seed, s.scen, (uint32_t)t, 2u, 0u, plan_step);
    const U4 w1 = scen_random(seed, s.scen, (uint32_t)t, 2u, 1u, plan_step);
    uint32_t z = 0;
    z |= reading(s, 1, w0.x);
    z |= reading(s, 2, w0.y);
    z |= reading(s, 3, w0.z);
    z |= reading(s, 4, w0.w);
    z |= reading(s, 5, w1.x);
    z |= reading(s, 6, w1.y);
    z |= reading(s, 7, w1.z);
    z |= reading(s, 8, w1.w);
    key = z;
    return r;
  }

  // The default policy on the last reading.
  __device__ __forceinline__ static int policy(uint32_t last) {
    constexpr int kOrder[8] = {5, 4, 6, 3, 7, 2, 8, 1};
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (!((last >> (kOrder[i] - 1)) & 1u)) return kOrder[i];
    return 0;
  }

  __device__ __forceinline__ static int cheb(int x0, int y0, int x1, int y1) {
    return max(abs(x1 - x0), abs(y1 - y0));
  }

  __device__ __forceinline__ float upper(const NavS& s) const {
    if (s.term) return 0.0f;
    const int wall = n / 2, gx = n / 2, gy = n - 1;
    int d;
    if (s.y < wall) {
      const int g = occupied(s, n / 4, wall) ? n - 1 - n / 4 : n / 4;
      d = cheb(s.x, s.y, g, wall) + cheb(g, wall, gx, gy);
    } else {
      d = cheb(s.x, s.y, gx, gy);
    }
    d = max(d, 1);  // a live robot standing on the goal (not reachable by g)
    return __fmul_rn(20.0f, G[d - 1]);
  }

  // Eq. lb from depth t0 with the last reading `last`; the tail is 0.
  __device__ __forceinline__ float rollout(NavS& s, uint32_t last, int t0, unsigned long long& steps) const {
    float v = 0.0f;
    int t = t0;
    while (t < D && !s.term) {
      const int a = policy(last);
      uint64_t key;
      const float r = step(s, a, t, key);
      steps += 1;
      if (!(key & kTermBit)) last = (uint32_t)(key & 0xFFu);
      v = __fadd_rn(v, __fmul_rn(G[t - t0], r));
      t += 1;
    }
    return v;
  }
};

__device__ __forceinline__ NavModel make_nav(const DevModel* gm, const float* G, uint32_t plan_step) {
  NavModel M;
  M.G = G;
  M.n = gm->n;
  M.mw = (gm->n * gm->n + 31) / 32;
  M.D = gm->D;
  M.seed = gm->seed;
  M.fail_thresh = gm->fail_thresh;
  M.sense_thresh = gm->sense_thresh;
  M.plan_step = plan_step;
  return M;
}

}  // namespace dsp
