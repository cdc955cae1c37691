// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// Driving among pedestrians (Sec. IV-A, "Autonomous Driving in a Crowd"): a car
// drives along a fixed path and picks accelerate / maintain / decelerate;
// accelerate and decelerate fail with a small probability; pedestrians walk
// toward hidden goals with Gaussian noise; the car sees its speed and the
// pedestrians' positions.
//
// Templated on the arithmetic type: Real = float is the FP32 oracle whose
// operation order the GPU kernels follow (every operation one IEEE-rounded
// + - * / sqrt, no contraction), Real = double is the FP64 oracle that checks
// the FP32 one.
//
// Readings where the paper is silent: the path is the
// line y = 20 from x = -10 for 60 m through the region [0,40]^2; speeds are
// 0..3 m/s in 1 m/s steps; the four goals are the region's corners; a
// pedestrian walks ped_speed*dt toward its goal (or lands on it when closer)
// and then gets N(0, sigma^2) noise per axis from a 4096-entry inverse-normal
// table indexed by the top 12 bits of a Philox word; collision = squared
// distance below 1 m^2 (-1000, terminal); goal = s >= 60 m (+1000,
// terminal); -0.1 for choosing decelerate; the observation is the speed and
// every pedestrian's position floored to 0.5 m cells.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "philox.hpp"
#include "rocksample.hpp"
#include "tables.hpp"

namespace orc {

inline uint64_t splitmix64_mix(uint64_t x) {
  // SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class Real>
struct CarState {
  Real s;      // distance travelled along the path
  int v;       // speed, m/s
  bool term;   // terminal
  uint32_t scen;
  std::vector<Real> px, py;
  std::vector<int> goal;
};

template <class Real>
struct Car {
  int P = 50;
  float gamma = 0.95f;
  int K = 500, D = 50;
  uint64_t seed = 0;
  uint32_t plan_step = 0;
  float path_len = 60.0f, dt = 0.33f, ped_speed = 1.2f, sigma = 0.1f;
  double fail_p = 0.01;
  uint64_t fail_thresh = 0;
  std::vector<Real> G;
  std::vector<Real> gauss;

  static const int kAccel = 0, kMaintain = 1, kDecel = 2;
  static const int kMaxSpeed = 3;

  void init() {
    G = gamma_powers<Real>(gamma, 256);
    std::vector<double> g64 = gauss_table_f64();
    gauss.resize(4096);
    for (int i = 0; i < 4096; ++i) gauss[i] = (Real)g64[i];
    fail_thresh = (uint64_t)std::floor(fail_p * 4294967296.0);
  }

  int num_actions() const { return 3; }
  bool terminal(const CarState<Real>& s) const { return s.term; }

  Real goal_x(int g) const { return (g & 1) ? (Real)40 : (Real)0; }
  Real goal_y(int g) const { return (g & 2) ? (Real)40 : (Real)0; }
  Real car_x(const CarState<Real>& s) const { return (Real)(-10) + s.s; }
  Real car_y() const { return (Real)20; }

  struct Obs {
    int v;
    std::vector<int> qx, qy;
    bool term;
    bool operator==(const Obs& o) const { return v == o.v && qx == o.qx && qy == o.qy && term == o.term; }
  };

  Obs observe_state(const CarState<Real>& s) const {
    Obs o;
    o.v = s.v;
    o.term = s.term;
    o.qx.resize(P);
    o.qy.resize(P);
    for (int i = 0; i < P; ++i) {
      o.qx[i] = (int)std::floor((Real)2 * s.px[i]);
      o.qy[i] = (int)std::floor((Real)2 * s.py[i]);
    }
    return o;
  }

  // 64-bit observation key: a sum of SplitMix64 mixes of the speed and of each
  // pedestrian's (index, cell x, cell y), so any summation order gives it;
  // bit 62 marks a terminal outcome.
  uint64_t obs_key(const Obs& o) const {
    uint64_t sum = splitmix64_mix((uint64_t)(o.v + 1));
    for (int i = 0; i < P; ++i) {
      uint64_t w = ((uint64_t)(i + 1) << 48) | ((uint64_t)(uint16_t)(int16_t)o.qx[i] << 16) |
                   (uint64_t)(uint16_t)(int16_t)o.qy[i];
      sum += splitmix64_mix(w);
    }
    return (sum & (kTerminalBit - 1)) | (o.term ? kTerminalBit : 0);
  }

  // g(s, a, phi_depth).
  Real step(const CarState<Real>& s, int a, int depth, CarState<Real>& out, uint64_t* key,
            Obs* obs = nullptr) const {
    out = s;
    if (s.term) {
      Obs o = observe_state(out);
      *key = obs_key(o);
      if (obs) *obs = o;
      return (Real)0;
    }
    count_ops(10);  // speed change with failure test, advance, car position
    // 1. speed change, failing with probability fail_p
    Block4 ra = scenario_random(seed, s.scen, (uint32_t)depth, kPurposeTransition, 0, plan_step);
    bool fails = (uint64_t)ra.w[0] < fail_thresh;
    if (a == kAccel && !fails && out.v < kMaxSpeed) out.v += 1;
    if (a == kDecel && !fails && out.v > 0) out.v -= 1;
    // 2. the car advances
    Real ds = (Real)out.v * (Real)dt;
    out.s = out.s + ds;
    Real cx = car_x(out), cy = car_y();
    // 3. pedestrians walk toward their goals, then get noise
    Real stride = (Real)ped_speed * (Real)dt;
    Block4 rp{};
    for (int i = 0; i < P; ++i) {
      count_ops(28);  // goal, dx, dy, distance (3 + sqrt), compare, 2 div, 2 mul, 2 add, noise 2x(index, load, mul, add)
      Real gx = goal_x(out.goal[i]), gy = goal_y(out.goal[i]);
      Real dx = gx - out.px[i];
      Real dy = gy - out.py[i];
      Real d2 = dx * dx + dy * dy;
      Real dist = std::sqrt(d2);
      if (dist > stride) {
        out.px[i] = out.px[i] + stride * (dx / dist);
        out.py[i] = out.py[i] + stride * (dy / dist);
      } else {
        out.px[i] = gx;
        out.py[i] = gy;
      }
      if ((i & 1) == 0)
        rp = scenario_random(seed, s.scen, (uint32_t)depth, kPurposePedestrian, (uint32_t)(i >> 1), plan_step);
      uint32_t ux = rp.w[2 * (i & 1)], uy = rp.w[2 * (i & 1) + 1];
      out.px[i] = out.px[i] + (Real)sigma * gauss[ux >> 20];
      out.py[i] = out.py[i] + (Real)sigma * gauss[uy >> 20];
    }
    // 4. reward and termination
    Real r = (a == kDecel) ? (Real)(-0.1f) : (Real)0;
    bool collide = false;
    for (int i = 0; i < P; ++i) {
      count_ops(7);
      Real ex = out.px[i] - cx, ey = out.py[i] - cy;
      if (ex * ex + ey * ey < (Real)1) collide = true;
    }
    count_ops(6);  // reward, goal test
    if (collide) {
      r = r + (Real)(-1000);
      out.term = true;
    } else if (out.s >= (Real)path_len) {
      r = r + (Real)1000;
      out.term = true;
    }
    Obs o = observe_state(out);
    *key = obs_key(o);
    if (obs) *obs = o;
    return r;
  }

  void observe(Hist&, int, uint64_t) const {}

  // Heuristic default policy: decelerate when a pedestrian is within 4 m ahead
  // in the 2 m corridor around the path, else accelerate up to 3 m/s, else
  // maintain.
  int policy(const CarState<Real>& s, const Hist&) const {
    Real cx = car_x(s), cy = car_y();
    count_ops(4);
    for (int i = 0; i < P; ++i) {
      count_ops(6);
      Real ex = s.px[i] - cx, ey = s.py[i] - cy;
      if (ex > (Real)0 && ex <= (Real)4 && ey >= (Real)(-1) && ey <= (Real)1) return kDecel;
    }
    return s.v < kMaxSpeed ? kAccel : kMaintain;
  }

  // Upper bound: the goal bonus at the earliest step the car could reach the
  // goal accelerating every step.
  Real upper(const CarState<Real>& s) const {
    if (s.term) return (Real)0;
    Real ss = s.s;
    int vv = s.v, t = 0;
    while (true) {
      count_ops(6);
      if (vv < kMaxSpeed) vv += 1;
      ss = ss + (Real)vv * (Real)dt;
      t += 1;
      if (ss >= (Real)path_len) break;
    }
    return (Real)1000 * G[t - 1];
  }

  // Value past the horizon: truncated to zero.
  Real tail(const CarState<Real>&) const { return (Real)0; }

  // State block format (field-major): f0 s (f32 bits), f1 v | terminal<<8,
  // f2 scenario id, f3 zero, then P words of pedestrian x, P of y (f32 bits),
  // then the goals packed four to a word (byte i%4 of word i/4).
  int words() const { return 4 + 2 * P + (P + 3) / 4; }

  static float bits_f(uint32_t w) {
    float f;
    std::memcpy(&f, &w, 4);
    return f;
  }
  static uint32_t f_bits(float f) {
    uint32_t w;
    std::memcpy(&w, &f, 4);
    return w;
  }

  CarState<Real> unpack(const uint32_t* block, int cap, int i) const {
    CarState<Real> s;
    s.s = (Real)bits_f(block[0 * cap + i]);
    uint32_t w1 = block[1 * cap + i];
    s.v = (int)(w1 & 0xFF);
    s.term = (w1 >> 8) & 1u;
    s.scen = block[2 * cap + i];
    s.px.resize(P);
    s.py.resize(P);
    s.goal.resize(P);
    for (int j = 0; j < P; ++j) {
      s.px[j] = (Real)bits_f(block[(4 + j) * cap + i]);
      s.py[j] = (Real)bits_f(block[(4 + P + j) * cap + i]);
      uint32_t gw = block[(4 + 2 * P + j / 4) * cap + i];
      s.goal[j] = (int)((gw >> (8 * (j % 4))) & 0xFF);
    }
    return s;
  }
  void pack(const CarState<Real>& s, uint32_t* block, int cap, int i) const {
    block[0 * cap + i] = f_bits((float)s.s);
    block[1 * cap + i] = (uint32_t)s.v | ((uint32_t)s.term << 8);
    block[2 * cap + i] = s.scen;
    block[3 * cap + i] = 0;
    for (int j = 0; j < P; ++j) {
      block[(4 + j) * cap + i] = f_bits((float)s.px[j]);
      block[(4 + P + j) * cap + i] = f_bits((float)s.py[j]);
    }
    for (int w = 0; w < (P + 3) / 4; ++w) {
      uint32_t gw = 0;
      for (int b = 0; b < 4; ++b)
        if (4 * w + b < P) gw |= (uint32_t)(s.goal[4 * w + b] & 0xFF) << (8 * b);
      block[(4 + 2 * P + w) * cap + i] = gw;
    }
  }
};

}  // namespace orc
