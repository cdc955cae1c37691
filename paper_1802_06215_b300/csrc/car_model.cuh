// Car among pedestrians (Sec. IV-A, "Autonomous Driving in a Crowd") on the
// device, with within-step parallelism (Sec. III-D, element level): TPS
// consecutive lanes of a warp share one scenario, each lane owning pedestrian
// pairs {2q, 2q+1} for q = lane_in_group, lane_in_group + TPS, ... (one
// Philox block feeds the noise of one pair). Group-wide facts (collision,
// danger ahead) are warp ballots restricted to the group's lanes.
//
// Every FP32 operation is one IEEE-rounded __f*_rn intrinsic in the order the
// model fixes: speed change (fails iff the Philox word of purpose 1 is below
// floor(fail_p * 2^32)), s += v*dt, each pedestrian walks stride toward its
// goal corner (or lands on it) and gets sigma * table[u >> 20] noise per axis,
// collision = squared distance < 1 (-1000, terminal), goal = s >= path length
// (+1000, terminal), -0.1 for choosing decelerate. Observation key: SplitMix64
// mix of (speed + 1) plus the mixes of every (index+1)<<48 | cell x<<16 |
// cell y, cells = floor(2 * position); bit 62 = terminal.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace dsp {

struct CarShared {
  float G[kGammaLen];
  float gauss[kGaussLen];
};

__device__ __forceinline__ uint64_t splitmix_mix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Pairs a lane may own with TPS lanes per scenario: enough for kMaxPeds by
// default, or KP when the model's crowd is known to fit (KP * TPS pairs).
template <int TPS>
constexpr int kDefaultPairs = (kMaxPeds / 2 + TPS - 1) / TPS;

template <int TPS, int KP = kDefaultPairs<TPS>>
struct CarLane {
  static constexpr int kPairs = KP;  // pairs a lane may own
  float px[2 * kPairs], py[2 * kPairs];
  // 2 bits per owned pedestrian: 64 bits once a lane owns more than 16
  using Goals = typename std::conditional<(2 * kPairs > 16), unsigned long long, uint32_t>::type;
  Goals goals;
  float s;
  int v;
  bool term;
  uint32_t scen;
};

template <int TPS, int KP = kDefaultPairs<TPS>>
struct CarModel {
  const CarShared* sh;
  int P, D;
  float path_len, dt, sigma, stride;
  uint64_t fail_thresh, seed;
  uint32_t plan_step;
  int gl;            // lane index inside the group
  uint32_t gmask;    // the group's lanes in the warp
  int gbase;         // first lane of the group

  __device__ __forceinline__ bool group_any(bool f) const {
    uint32_t b = __ballot_sync(0xFFFFFFFFu, f);
    return (b & gmask) != 0u;
  }

  // Loads scenario i of a state block into the lane's share of the group.
  __device__ __forceinline__ void load(CarLane<TPS, KP>& L, const uint32_t* b, int cap, int i) const {
    L.s = __uint_as_float(b[i]);
    uint32_t w1 = b[cap + i];
    L.v = (int)(w1 & 0xFFu);
    L.term = (w1 >> 8) & 1u;
    L.scen = b[2 * cap + i];
    L.goals = 0;
#pragma unroll
    for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k) {
      int q = gl + k * TPS;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int j = 2 * q + e;
        if (j < P) {
          L.px[2 * k + e] = __uint_as_float(b[(size_t)(4 + j) * cap + i]);
          L.py[2 * k + e] = __uint_as_float(b[(size_t)(4 + P + j) * cap + i]);
          uint32_t gw = b[(size_t)(4 + 2 * P + j / 4) * cap + i];
          L.goals |= (typename CarLane<TPS, KP>::Goals)((gw >> (8 * (j % 4))) & 3u) << (2 * (2 * k + e));
        } else {
          L.px[2 * k + e] = 0.0f;
          L.py[2 * k + e] = 0.0f;
        }
      }
    }
  }

  // Writes the group's scenario to slot i; lanes with valid = false write
  // nothing but still take part in the goal-word shuffles.
  __device__ __forceinline__ void store(const CarLane<TPS, KP>& L, uint32_t* b, int cap, int i, bool valid) const {
    if (valid && gl == 0) {
      b[i] = __float_as_uint(L.s);
      b[cap + i] = (uint32_t)L.v | ((uint32_t)L.term << 8);
      b[2 * cap + i] = L.scen;
      b[3 * cap + i] = 0u;
    }
#pragma unroll
    for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k) {
      int q = gl + k * TPS;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int j = 2 * q + e;
        if (valid && j < P) {
          b[(size_t)(4 + j) * cap + i] = __float_as_uint(L.px[2 * k + e]);
          b[(size_t)(4 + P + j) * cap + i] = __float_as_uint(L.py[2 * k + e]);
        }
      }
    }
    // goal words: four pedestrians (two pairs) per word; the lane owning the
    // word's first pair gathers the second pair's goals from its owner
#pragma unroll
    for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k) {
      int q = gl + k * TPS;
      uint32_t mine = (uint32_t)(L.goals >> (4 * k)) & 15u;
      int q2 = q + 1;
      int src = gbase + (q2 % TPS);
      int k2 = q2 / TPS;
      const typename CarLane<TPS, KP>::Goals other_all = __shfl_sync(0xFFFFFFFFu, L.goals, src);
      uint32_t other = (uint32_t)(other_all >> (4 * k2)) & 15u;
      if (valid && (q & 1) == 0 && 2 * q < P) {
        uint32_t w = (mine & 3u) | ((mine >> 2) << 8);
        if (2 * q2 < P) w |= ((other & 3u) << 16) | ((other >> 2) << 24);
        b[(size_t)(4 + 2 * P + q / 2) * cap + i] = w;
      }
    }
  }

  // The Philox word deciding an action failure at depth t.
  __device__ __forceinline__ uint32_t fail_word(uint32_t scen, int t) const {
    return scen_random(seed, scen, (uint32_t)t, 1u, 0u, plan_step).x;
  }

  // g(s, a, phi_t) for one group (all lanes call it; `live` lanes change).
  // Returns the reward; sets danger (policy input of the next state) and, with
  // kKey, the observation key.
  template <bool kKey>
  __device__ __forceinline__ float step(CarLane<TPS, KP>& L, bool live, int a, int t, uint32_t ufail,
                                        bool& danger, uint64_t& key) const {
    float r = 0.0f;
    bool fails = (uint64_t)ufail < fail_thresh;
    if (live) {
      if (a == 0 && !fails && L.v < 3) L.v += 1;
      if (a == 2 && !fails && L.v > 0) L.v -= 1;
      L.s = __fadd_rn(L.s, __fmul_rn((float)L.v, dt));
    }
    float cx = __fadd_rn(-10.0f, L.s), cy = 20.0f;
    bool coll = false, dang = false;
    uint64_t ksum = 0;
#pragma unroll
    for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k) {
      int q = gl + k * TPS;
      if (2 * q < P) {
        U4 rp = live ? scen_random(seed, L.scen, (uint32_t)t, 3u, (uint32_t)q, plan_step) : U4{0, 0, 0, 0};
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          int j = 2 * q + e;
          if (j < P) {
            float& x = L.px[2 * k + e];
            float& y = L.py[2 * k + e];
            if (live) {
              int gi = (int)(L.goals >> (2 * (2 * k + e))) & 3;
              float gx = (gi & 1) ? 40.0f : 0.0f, gy = (gi & 2) ? 40.0f : 0.0f;
              float dx = __fsub_rn(gx, x), dy = __fsub_rn(gy, y);
              float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
              float dist = __fsqrt_rn(d2);
              if (dist > stride) {
                x = __fadd_rn(x, __fmul_rn(stride, __fdiv_rn(dx, dist)));
                y = __fadd_rn(y, __fmul_rn(stride, __fdiv_rn(dy, dist)));
              } else {
                x = gx;
                y = gy;
              }
              uint32_t ux = e ? rp.z : rp.x, uy = e ? rp.w : rp.y;
              x = __fadd_rn(x, __fmul_rn(sigma, sh->gauss[ux >> 20]));
              y = __fadd_rn(y, __fmul_rn(sigma, sh->gauss[uy >> 20]));
            }
            float ex = __fsub_rn(x, cx), ey = __fsub_rn(y, cy);
            coll = coll || (__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)) < 1.0f);
            dang = dang || (ex > 0.0f && ex <= 4.0f && ey >= -1.0f && ey <= 1.0f);
            if (kKey) {
              int qx = (int)floorf(__fmul_rn(2.0f, x)), qy = (int)floorf(__fmul_rn(2.0f, y));
              uint64_t w = ((uint64_t)(j + 1) << 48) | ((uint64_t)(uint16_t)(int16_t)qx << 16) |
                           (uint64_t)(uint16_t)(int16_t)qy;
              ksum += splitmix_mix(w);
            }
          }
        }
      }
    }
    bool gcoll = group_any(coll);
    danger = group_any(dang);
    if (live) {
      r = (a == 2) ? -0.1f : 0.0f;
      if (gcoll) {
        r = __fadd_rn(r, -1000.0f);
        L.term = true;
      } else if (L.s >= path_len) {
        r = __fadd_rn(r, 1000.0f);
        L.term = true;
      }
    }
    if (kKey) {
#pragma unroll
      for (int o = TPS / 2; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xFFFFFFFFu, ksum, o);
      uint64_t sum = splitmix_mix((uint64_t)(L.v + 1)) + ksum;
      key = (sum & (kTermBit - 1)) | (L.term ? kTermBit : 0ull);
    }
    return r;
  }

  __device__ __forceinline__ int policy(const CarLane<TPS, KP>& L, bool danger) const {
    return danger ? 2 : (L.v < 3 ? 0 : 1);
  }

  // u: the goal bonus at the earliest step the car could reach the goal
  // accelerating every step.
  __device__ __forceinline__ float upper(const CarLane<TPS, KP>& L) const {
    if (L.term) return 0.0f;
    float ss = L.s;
    int vv = L.v, t = 0;
    while (true) {
      if (vv < 3) vv += 1;
      ss = __fadd_rn(ss, __fmul_rn((float)vv, dt));
      t += 1;
      if (ss >= path_len || t >= kGammaLen) break;
    }
    return __fmul_rn(1000.0f, sh->G[t - 1]);
  }

  // Danger ahead in the current state (policy input), group-wide.
  __device__ __forceinline__ bool danger_now(const CarLane<TPS, KP>& L) const {
    float cx = __fadd_rn(-10.0f, L.s), cy = 20.0f;
    bool dang = false;
#pragma unroll
    for (int k = 0; k < CarLane<TPS, KP>::kPairs; ++k) {
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        int j = 2 * (gl + k * TPS) + e;
        if (j < P) {
          float ex = __fsub_rn(L.px[2 * k + e], cx), ey = __fsub_rn(L.py[2 * k + e], cy);
          dang = dang || (ex > 0.0f && ex <= 4.0f && ey >= -1.0f && ey <= 1.0f);
        }
      }
    }
    return group_any(dang);
  }

  // Eq. lb from depth t0 for the group's scenario. Every lane of the warp runs
  // the same number of iterations (until every group in the warp is done);
  // `valid` is false for lanes without a scenario. The action-failure words of
  // TPS depths are drawn at once, one per lane, and broadcast.
  __device__ __forceinline__ float rollout(CarLane<TPS, KP>& L, bool valid, bool danger, int t0,
                                           unsigned long long& steps) const {
    float v = 0.0f;
    int t = t0;
    uint32_t ufail_mine = 0;
    int tbase = t0 - TPS;
    while (true) {
      bool live = valid && !L.term && t < D;
      if (!__any_sync(0xFFFFFFFFu, live)) break;
      if (t - tbase >= TPS) {
        tbase = t;
        ufail_mine = fail_word(L.scen, t + gl);
      }
      uint32_t ufail = __shfl_sync(0xFFFFFFFFu, ufail_mine, gbase + (t - tbase));
      int a = policy(L, danger);
      uint64_t key;
      float r = step<false>(L, live, a, t, ufail, danger, key);
      if (live) {
        v = __fadd_rn(v, __fmul_rn(sh->G[t - t0], r));
        if (gl == 0) steps += 1;
      }
      t += 1;
    }
    return v;
  }
};

// A group's view of the model: TPS consecutive lanes share one scenario.
template <int TPS, int KP = kDefaultPairs<TPS>>
__device__ __forceinline__ CarModel<TPS, KP> make_car_model(const DevModel* gm, const CarShared* sh,
                                                            uint32_t plan_step) {
  CarModel<TPS, KP> M;
  M.sh = sh;
  M.P = gm->P;
  M.D = gm->D;
  M.path_len = gm->path_len;
  M.dt = gm->dt;
  M.sigma = gm->sigma;
  M.stride = gm->stride;
  M.fail_thresh = gm->fail_thresh;
  M.seed = gm->seed;
  M.plan_step = plan_step;
  int lane = threadIdx.x & 31;
  M.gl = lane % TPS;
  M.gbase = lane - M.gl;
  M.gmask = (TPS == 32 ? 0xFFFFFFFFu : ((1u << TPS) - 1u)) << M.gbase;
  return M;
}

__device__ __forceinline__ void load_car_consts(CarShared& c, const DevModel* gm) {
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) c.G[k] = gm->G[k];
  for (int k = threadIdx.x; k < kGaussLen; k += blockDim.x) c.gauss[k] = gm->gauss[k];
}

}  // namespace dsp
