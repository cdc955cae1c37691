// Navigation in a partially known map (Sec. IV-A) on the device: one thread
// per scenario, the state in registers (position, terminal flag, the
// scenario's occupancy map, the true occupancy of the eight neighbours,
// scenario id).
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
//
// Register layout of the map: row r (n <= 16 cells, bit c = column c, bits
// n..15 set: off the map) is the 16-bit half (r + 1) & 1 of word (r + 1) >> 1,
// with the rows -1 and n.. all set, so that the three rows around the robot
// are one 64-bit window of two adjacent words. The state block keeps the map
// packed cell-major (cell y * n + x at bit c & 31 of word c >> 5); the map
// never changes within a scenario, so stores copy the packed words.
#pragma once
#include "common.cuh"

namespace dsp {

constexpr int kNavMaxWords = 8;  // packed occupancy words: n * n <= 256
constexpr int kNavRowWords = 9;  // rows -1..16, two per word

// Per-CTA lookup tables in shared memory.
struct NavTables {
  float G[kGammaLen];  // gamma^k
  uint8_t nb[512];     // 3x3 block (rows y-1, y, y+1; columns x-1..x+1) -> neighbours in action order
  uint8_t pol[256];    // last reading -> default-policy action
};

__device__ __forceinline__ void load_nav_tables(NavTables& T, const DevModel* gm) {
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) T.G[k] = gm->G[k];
  for (int b = threadIdx.x; b < 512; b += blockDim.x) {
    const uint32_t t = b & 7, m = (b >> 3) & 7, s = (b >> 6) & 7;  // bit 0: column x-1
    T.nb[b] = (uint8_t)(((t >> 1) & 1u) | (((t >> 2) & 1u) << 1) | (((m >> 2) & 1u) << 2) | (((s >> 2) & 1u) << 3) |
                        (((s >> 1) & 1u) << 4) | ((s & 1u) << 5) | ((m & 1u) << 6) | ((t & 1u) << 7));
  }
  for (int l = threadIdx.x; l < 256; l += blockDim.x) {
    constexpr int kOrder[8] = {5, 4, 6, 3, 7, 2, 8, 1};
    int a = 0;
    for (int i = 7; i >= 0; --i)
      if (!((l >> (kOrder[i] - 1)) & 1)) a = kOrder[i];
    T.pol[l] = (uint8_t)a;
  }
}

struct NavS {
  int x, y;
  bool term;
  uint32_t nb;  // true occupancy of the neighbours, bit k-1 for action k
  uint32_t R[kNavRowWords];
  uint32_t scen;
};

struct NavModel {
  const NavTables* T;
  int n, mw, D;
  uint64_t seed;
  uint32_t fail_th, sense_th;  // below: fails / flips (when not all)
  bool fail_all, sense_all;    // p = 1
  uint32_t plan_step;

  // stay, N, NE, E, SE, S, SW, W, NW: 2 bits per action of dx + 1 and dy + 1
  __device__ __forceinline__ static int dx(int a) { return (int)((0x6A5u >> (2 * a)) & 3u) - 1; }
  __device__ __forceinline__ static int dy(int a) { return (int)((0x6A41u >> (2 * a)) & 3u) - 1; }

  // word j (0..7) of R, or word j + 1 (base = 1), by a select tree
  __device__ __forceinline__ static uint32_t sel(const uint32_t (&R)[kNavRowWords], int base, int j) {
    const uint32_t a01 = (j & 1) ? R[base + 1] : R[base + 0];
    const uint32_t a23 = (j & 1) ? R[base + 3] : R[base + 2];
    const uint32_t a45 = (j & 1) ? R[base + 5] : R[base + 4];
    const uint32_t a67 = (j & 1) ? R[base + 7] : R[base + 6];
    const uint32_t b03 = (j & 2) ? a23 : a01;
    const uint32_t b47 = (j & 2) ? a67 : a45;
    return (j & 4) ? b47 : b03;
  }

  // The map rows from the packed words; word(k) is packed word k (k <= mw:
  // the word after the map may be read, its bits are not used).
  template <class W>
  __device__ __forceinline__ void set_rows(NavS& s, W word) const {
    const uint32_t pad = 0xFFFFu & ~((1u << n) - 1u);
#pragma unroll
    for (int k = 0; k < kNavRowWords; ++k) s.R[k] = 0xFFFFFFFFu;
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (r < n) {
        const int b = r * n;
        const uint32_t row = (__funnelshift_r(word(b >> 5), word((b >> 5) + 1), b & 31) & 0xFFFFu) | pad;
        const int i = r + 1;  // a constant once unrolled
        s.R[i >> 1] = (i & 1) ? ((s.R[i >> 1] & 0x0000FFFFu) | (row << 16)) : ((s.R[i >> 1] & 0xFFFF0000u) | row);
      }
    }
  }

  // occupancy of cell (x, y); off the map reads occupied
  __device__ __forceinline__ bool occupied(const NavS& s, int x, int y) const {
    if (x < 0 || y < 0 || x >= n || y >= n) return true;
    const int i = y + 1;
    const uint32_t w = (i >> 1) < 8 ? sel(s.R, 0, i >> 1) : s.R[8];
    return (w >> (16 * (i & 1) + x)) & 1u;
  }

  // the neighbours' occupancy in action order, from the 3x3 block around (x, y)
  __device__ __forceinline__ uint32_t neighbourhood(const NavS& s) const {
    const int j = s.y >> 1;  // rows y-1, y, y+1 are indices y..y+2, in words j and j + 1
    const uint32_t lo = sel(s.R, 0, j), hi = sel(s.R, 1, j);
    const uint32_t odd = (uint32_t)s.y & 1u;
    const uint32_t r01 = __funnelshift_r(lo, hi, 16 * odd);
    const uint32_t r2 = odd ? (hi >> 16) : hi;
    // column c at bit c + 1; column -1 and columns >= 16 read occupied
    const uint32_t t = ((((r01 & 0xFFFFu) << 1) | 0xFFFE0001u) >> s.x) & 7u;
    const uint32_t m = ((((r01 >> 16) << 1) | 0xFFFE0001u) >> s.x) & 7u;
    const uint32_t b = ((((r2 & 0xFFFFu) << 1) | 0xFFFE0001u) >> s.x) & 7u;
    return T->nb[t | (m << 3) | (b << 6)];
  }

  __device__ __forceinline__ NavS load(const uint32_t* b, int cap, int i) const {
    NavS s;
    const uint32_t w = b[i];
    s.x = (int)(w & 0xFFu);
    s.y = (int)((w >> 8) & 0xFFu);
    s.term = (w >> 16) & 1u;
    set_rows(s, [&](int k) { return b[(size_t)(1 + k) * cap + i]; });
    s.scen = b[(size_t)(1 + mw) * cap + i];
    s.nb = s.term ? 0u : neighbourhood(s);
    return s;
  }
  // position word and scenario id; the map words are copied by copy_map
  __device__ __forceinline__ void store_pos(const NavS& s, uint32_t* b, int cap, int i) const {
    b[i] = (uint32_t)s.x | ((uint32_t)s.y << 8) | ((uint32_t)s.term << 16);
    b[(size_t)(1 + mw) * cap + i] = s.scen;
  }
  __device__ __forceinline__ void copy_map(const uint32_t* src, int scap, int si, uint32_t* dst, int dcap,
                                           int di) const {
#pragma unroll
    for (int k = 0; k < kNavMaxWords; ++k)
      if (k < mw) dst[(size_t)(1 + k) * dcap + di] = src[(size_t)(1 + k) * scap + si];
  }

  // g(s, a, phi_t); returns the reward, writes the observation key.
  __device__ __forceinline__ float step(NavS& s, int a, int t, uint64_t& key) const {
    if (s.term) {
      key = kTermBit;
      return 0.0f;
    }
    // the step's three Philox draws (move failure, two blocks of sensor
    // words), independent chains issued together; staying does not use the
    // first, a terminal outcome not the others
    const uint32_t u = scen_random(seed, s.scen, (uint32_t)t, 1u, 0u, plan_step).x;
    const U4 w0 = scen_random(seed, s.scen, (uint32_t)t, 2u, 0u, plan_step);
    const U4 w1 = scen_random(seed, s.scen, (uint32_t)t, 2u, 1u, plan_step);
    float r;
    if (a == 0) {
      r = -0.2f;
    } else {
      if (fail_all || u < fail_th) {
        r = -0.1f;
      } else if ((s.nb >> (a - 1)) & 1u) {
        r = -1.0f;
      } else {
        s.x += dx(a);
        s.y += dy(a);
        if (s.x == n / 2 && s.y == n - 1) {
          s.term = true;
          r = 20.0f;
        } else {
          r = -0.1f;
          s.nb = neighbourhood(s);
        }
      }
    }
    if (s.term) {
      key = kTermBit;
      return r;
    }
    uint32_t f;
    if (sense_all) {
      f = 0xFFu;
    } else {
      f = (uint32_t)(w0.x < sense_th) | ((uint32_t)(w0.y < sense_th) << 1) | ((uint32_t)(w0.z < sense_th) << 2) |
          ((uint32_t)(w0.w < sense_th) << 3) | ((uint32_t)(w1.x < sense_th) << 4) |
          ((uint32_t)(w1.y < sense_th) << 5) | ((uint32_t)(w1.z < sense_th) << 6) |
          ((uint32_t)(w1.w < sense_th) << 7);
    }
    key = s.nb ^ f;
    return r;
  }

  // The default policy on the last reading.
  __device__ __forceinline__ int policy(uint32_t last) const { return T->pol[last & 0xFFu]; }

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
    return __fmul_rn(20.0f, T->G[d - 1]);
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
      v = __fadd_rn(v, __fmul_rn(T->G[t - t0], r));
      t += 1;
    }
    return v;
  }
};

__device__ __forceinline__ NavModel make_nav(const DevModel* gm, const NavTables* T, uint32_t plan_step) {
  NavModel M;
  M.T = T;
  M.n = gm->n;
  M.mw = (gm->n * gm->n + 31) / 32;
  M.D = gm->D;
  M.seed = gm->seed;
  M.fail_all = gm->fail_thresh > 0xFFFFFFFFull;
  M.sense_all = gm->sense_thresh > 0xFFFFFFFFull;
  M.fail_th = (uint32_t)gm->fail_thresh;
  M.sense_th = (uint32_t)gm->sense_thresh;
  M.plan_step = plan_step;
  return M;
}

}  // namespace dsp
