// CPU ORACLE — test infrastructure only (see philox.hpp for the rule).
//
// Navigation in a partially known map (Sec. IV-A): a robot starts on the top
// border of an n x n map (13 x 13 in the paper) and travels to a goal at the
// bottom through one of two gates in a middle wall, only one of which is open.
// Some cells are known to the robot (they help it localise but look alike);
// the others are occupied with probability 0.1. Each step the robot stays or
// moves to one of its eight neighbours. A move fails with probability 0.03;
// each of the eight adjacent-cell readings (occupied or free) is wrong with
// probability 0.03. Staying costs 0.2, a move 0.1, a crash 1; reaching the goal
// gives 20 and ends the world.
//
// Readings where the paper is silent:
//  * layout: wall row y = n/2 occupied except the gates at x = n/4 and
//    x = n-1-n/4, exactly one of them open; goal (n/2, n-1); start row y = 0;
//    the state holds the full occupancy map (known and unknown cells alike);
//  * actions: 0 stay, 1 N (y-1), 2 NE, 3 E (x+1), 4 SE, 5 S (y+1), 6 SW, 7 W,
//    8 NW; a failed move (Philox purpose 1 word below floor(p * 2^32)) leaves
//    the robot in place and costs 0.1; a move off the map or onto an occupied
//    cell is a crash: -1 and the robot stays; entering the goal gives +20
//    (instead of the move cost) and ends the world;
//  * observation: one bit per neighbour in action order N..NW (bit k-1 for
//    action k), 1 = occupied (off-map cells read occupied), each bit flipped
//    when its Philox purpose-2 word (elements 0 and 1, words 0..3 each) is
//    below floor(q * 2^32); a terminal outcome observes nothing (bit 62 only);
//  * default policy (history-based: it sees only the last reading, kept in
//    counter 0 of the history): the first of S, SE, SW, E, W, NE, NW, N whose
//    last reading was free, else stay;
//  * u(phi) = 20 gamma^(d-1), d the 8-connected (Chebyshev) distance to the
//    goal, through the open gate while the robot is above the wall; l at the
//    horizon is 0 (values count to depth D only).
#pragma once
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "philox.hpp"
#include "rocksample.hpp"
#include "tables.hpp"

namespace orc {

struct NavState {
  int x, y;
  bool term;
  uint32_t occ[8];  // occupancy, bit c of the map's cell c = y * n + x
  uint32_t scen;
};

template <class Real>
struct Nav {
  int n = 13;
  float gamma = 0.95f;
  int K = 100, D = 90;
  uint64_t seed = 0;
  uint32_t plan_step = 0;
  double fail_p = 0.03, sense_p = 0.03;
  uint64_t fail_thresh = 0, sense_thresh = 0;
  std::vector<Real> G;

  static constexpr int kDx[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};
  static constexpr int kDy[9] = {0, -1, -1, 0, 1, 1, 1, 0, -1};

  void init() {
    G = gamma_powers<Real>(gamma, 256);
    fail_thresh = (uint64_t)std::floor(fail_p * 4294967296.0);
    sense_thresh = (uint64_t)std::floor(sense_p * 4294967296.0);
  }

  int num_actions() const { return 9; }
  int wall_row() const { return n / 2; }
  int gate_x(int g) const { return g == 0 ? n / 4 : n - 1 - n / 4; }
  int goal_x() const { return n / 2; }
  int goal_y() const { return n - 1; }
  int map_words() const { return (n * n + 31) / 32; }

  bool terminal(const NavState& s) const { return s.term; }
  bool occupied(const NavState& s, int x, int y) const {
    if (x < 0 || y < 0 || x >= n || y >= n) return true;
    const int c = y * n + x;
    return (s.occ[c >> 5] >> (c & 31)) & 1u;
  }

  // g(s, a, phi_depth): successor state, observation key, reward.
  Real step(const NavState& s, int a, int depth, NavState& out, uint64_t* key) const {
    out = s;
    count_ops(2);  // terminal test, action dispatch
    if (s.term) {
      *key = kTerminalBit;
      return (Real)0;
    }
    Real r;
    if (a == 0) {
      r = (Real)-0.2f;
    } else {
      count_ops(3);  // failure compare, target x and y
      Block4 f = scenario_random(seed, s.scen, (uint32_t)depth, kPurposeTransition, 0u, plan_step);
      if ((uint64_t)f.w[0] < fail_thresh) {
        r = (Real)-0.1f;
      } else {
        const int nx = s.x + kDx[a], ny = s.y + kDy[a];
        count_ops(6);  // bounds, map bit, goal test
        if (occupied(s, nx, ny)) {
          r = (Real)-1.0f;
        } else {
          out.x = nx;
          out.y = ny;
          if (nx == goal_x() && ny == goal_y()) {
            out.term = true;
            r = (Real)20.0f;
          } else {
            r = (Real)-0.1f;
          }
        }
      }
    }
    if (out.term) {
      *key = kTerminalBit;
      return r;
    }
    Block4 w0 = scenario_random(seed, s.scen, (uint32_t)depth, kPurposeSensor, 0u, plan_step);
    Block4 w1 = scenario_random(seed, s.scen, (uint32_t)depth, kPurposeSensor, 1u, plan_step);
    uint64_t z = 0;
    for (int k = 1; k <= 8; ++k) {
      count_ops(7);  // neighbour, bounds, map bit, noise compare, flip, place
      const uint32_t u = k <= 4 ? w0.w[k - 1] : w1.w[k - 5];
      bool bit = occupied(out, out.x + kDx[k], out.y + kDy[k]);
      if ((uint64_t)u < sense_thresh) bit = !bit;
      if (bit) z |= 1ull << (k - 1);
    }
    *key = z;
    return r;
  }

  // The last reading is the history the default policy sees.
  void observe(Hist& h, int, uint64_t key) const {
    count_ops(1);
    if (!(key & kTerminalBit)) h.c[0] = (int8_t)(uint8_t)(key & 0xFFu);
  }

  int policy(const NavState&, const Hist& h) const {
    static const int kOrder[8] = {5, 4, 6, 3, 7, 2, 8, 1};
    const uint32_t last = (uint32_t)(uint8_t)h.c[0];
    for (int i = 0; i < 8; ++i) {
      count_ops(2);
      const int a = kOrder[i];
      if (!((last >> (a - 1)) & 1u)) return a;
    }
    return 0;
  }

  static int cheb(int x0, int y0, int x1, int y1) {
    const int dx = std::abs(x1 - x0), dy = std::abs(y1 - y0);
    return dx > dy ? dx : dy;
  }

  // 20 gamma^(d-1) with d the 8-connected distance to the goal, through the
  // open gate from above the wall.
  Real upper(const NavState& s) const {
    count_ops(1);
    if (s.term) return (Real)0;
    int d;
    count_ops(12);  // open gate, two Chebyshev distances, sum, table lookup, product
    if (s.y < wall_row()) {
      const int g = occupied(s, gate_x(0), wall_row()) ? 1 : 0;
      d = cheb(s.x, s.y, gate_x(g), wall_row()) + cheb(gate_x(g), wall_row(), goal_x(), goal_y());
    } else {
      d = cheb(s.x, s.y, goal_x(), goal_y());
    }
    if (d < 1) d = 1;  // a live robot standing on the goal (not reachable by g)
    return (Real)20 * G[d - 1];
  }

  Real tail(const NavState&) const { return (Real)0; }

  // Words of one scenario (field-major): f0 x | y << 8 | terminal << 16,
  // f1..f(mw) the occupancy map, f(mw+1) the scenario id; mw = ceil(n*n/32).
  NavState unpack(const uint32_t* block, int cap, int i) const {
    NavState s{};
    const uint32_t w = block[i];
    s.x = (int)(w & 0xFF);
    s.y = (int)((w >> 8) & 0xFF);
    s.term = (w >> 16) & 1u;
    const int mw = map_words();
    for (int k = 0; k < 8; ++k) s.occ[k] = k < mw ? block[(size_t)(1 + k) * cap + i] : 0u;
    s.scen = block[(size_t)(1 + mw) * cap + i];
    return s;
  }
  void pack(const NavState& s, uint32_t* block, int cap, int i) const {
    block[i] = (uint32_t)s.x | ((uint32_t)s.y << 8) | ((uint32_t)s.term << 16);
    const int mw = map_words();
    for (int k = 0; k < mw; ++k) block[(size_t)(1 + k) * cap + i] = s.occ[k];
    block[(size_t)(1 + mw) * cap + i] = s.scen;
  }
};

template <class Real>
constexpr int Nav<Real>::kDx[9];
template <class Real>
constexpr int Nav<Real>::kDy[9];

}  // namespace orc
