// Leaf expansion for Rock Sample models (one or two robots), Sec. III-D, in
// two phases.
//
// Phase A (rs_group_kernel, persistent over jobs, largest first): a CTA takes
// a leaf job, gathers its scenarios from the parent list and applies the last
// action ("update") once. Each warp then expands whole actions of the job in
// two passes over 32-scenario chunks:
//  1. Step every (action, scenario) pair with g (Eq. expand) and count each
//     observation code (z, and whether the step ended the world): its
//     scenarios, first position and exact reward sum, by ballots (one robot,
//     6 codes, in registers) or __match_any_sync leaders (two robots, 18
//     codes, in the warp's rows of shared tables).
//  2. Number the children by first position (Eq. newnodes), then write the
//     grouped positions and one rollout item per (action, scenario), in
//     child-grouped order, and list each child's items as slices of up to
//     128. Actions that draw no random numbers are re-applied; Sense leaves
//     the state unchanged. Where the job's scenarios share the robots' cells
//     and sampled mask (a tree node's), a child's items share their state
//     after the step: the slice holds it and an item only its good mask.
// No barrier is needed inside a job. Phase A also writes the children's
// counts, offsets, keys and reward sums.
//
// Phase B (rs_rollout_slices_kernel): warps take slices (no barriers), four
// items a lane, all one child's, so one trajectory of the default policy
// (Eq. lb, whose moves read no rock state) gives every item's value, with
// each item's own rewards; u (Eq. ub) comes from per-rock terms computed once
// per slice, and the child's int64 fixed-point sums take one warp sum and one
// reduction each (exact in any order). Without a slice list (the
// no-allocation entry point) rs_rollout_items_kernel takes 32-item chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "rs_common.cuh"
#include "rs_model.cuh"

namespace dsp {

namespace {

constexpr int kBlockA = 512;          // phase-A CTA: 16 warps
constexpr int kWarpsA = kBlockA / 32;
constexpr int kCodes = 18;            // observation code z + 9 * terminal, z <= 8

struct RSGroupSmem {
  RSShared c;
  uint32_t leaf[5][kMaxScen];          // the leaf's states, field-major
  uint32_t sense[2][kMaxScen];         // each scenario's sensor word per robot at the leaf's depth
  // two robots, per warp and observation code of the warp's current action:
  int wcnt[kWarpsA][kCodes];           // scenarios holding the code
  int wfirst[kWarpsA][kCodes];         // first position of the code
  int wpre[kWarpsA][kCodes];           // scenarios of the code placed so far (pass 2)
  int aoff[kWarpsA][kCodes];           // offset of the code's child in the grouped order
  int acid[kWarpsA][kCodes];           // child index of the code
  unsigned long long sr[kWarpsA][kCodes];  // exact reward sum (fixed point)
  uint32_t pm_job;
  int job, part;
  dsp_leaf_job J;
  uint8_t code1[kWarpsA][kMaxScen];    // each warp's observation codes of its current action
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Writes job j's compact leaf states (given one at a time by the caller's
// loop over p) and its block table entries.
__device__ __forceinline__ void put_leaf(const LeafBlocks& lb, int j, int n, int p, uint32_t pos, uint32_t good,
                                         uint32_t sampled) {
  uint32_t* L = lb.leaf + 3 * lb.scen_base[j];
  L[p] = pos;
  L[n + p] = good;
  L[2 * n + p] = sampled;
}
__device__ __forceinline__ void put_blocks(const LeafBlocks& lb, int j, int n, int A) {
  const long long u0 = lb.unit_base[j];
  const int nu = A * ((n + 31) >> 5);
  for (int u = threadIdx.x; u < nu; u += (int)blockDim.x) lb.chunk_job[u0 + u] = j;
}

// Gather + update of the job in S.J into S.leaf (and J.leaf_states), and the
// job's positive-counter mask. Ends with a barrier. Only the job's first unit
// (`first`) counts the update steps and writes the leaf's states.
template <int R>
__device__ __forceinline__ void gather_update(RSGroupSmem& S, const RSModel<R>& M, bool first,
                                              unsigned long long& steps) {
  const int tid = threadIdx.x;
  const dsp_leaf_job& J = S.J;
  const int n = J.n_scen, depth = J.depth;
  for (int p = tid; p < n; p += (int)blockDim.x) {
    RSS s = M.load(J.parent, J.parent_cap, J.idx[p]);
    if (J.last_action >= 0) {
      if (!M.terminal(s) && first) steps += 1;
      uint64_t k;
      M.step(s, J.last_action, depth - 1, k);
    }
    S.leaf[0][p] = s.pos[0];
    S.leaf[1][p] = s.pos[1];
    S.leaf[2][p] = s.good;
    S.leaf[3][p] = s.sampled;
    S.leaf[4][p] = s.scen;
#pragma unroll
    for (int r = 0; r < R; ++r) S.sense[r][p] = M.sense_word(s.scen, depth, r);
    if (first && J.leaf_states != nullptr) M.store(s, J.leaf_states, n, p);
  }
  if (tid == 0) {
    uint32_t h[8];
    const uint32_t* hw = reinterpret_cast<const uint32_t*>(J.hist);
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = hw[k];
    S.pm_job = positive_mask(h, M.m);
  }
  __syncthreads();
}

// An action's slices for the rollout phase: each child's grouped positions
// (count cnt[c] from offset off[c]) in runs of at most kSliceItems items.
// Called by one lane; one atomic per action takes the slots. `shared`: the
// job's scenarios share the robot's cell and sampled mask, so every item of
// child c has the position pos, the candidate mask pm_z[c % 3] & ~sampled
// and the child's depth and slot, which the slice carries.
template <int kC>
__device__ __forceinline__ void put_slices(const Slices& sl, long long ibase, int a, int n, const int (&cnt)[kC],
                                           const int (&off)[kC], const int (&cid)[kC], int cap, int depth, int j,
                                           bool shared, uint32_t pos, const uint32_t (&pm_z)[3], uint32_t sampled,
                                           DevWork* work) {
  if (sl.list == nullptr) return;
  int ns = 0;
#pragma unroll
  for (int c = 0; c < kC; ++c) ns += (cnt[c] + kSliceItems - 1) / kSliceItems;
  if (ns == 0) return;
  unsigned int k = atomicAdd(sl.count, (unsigned int)ns);
  if (k + (unsigned int)ns > sl.cap) {
    report(work, kStatusOverflow);
    return;
  }
  const long long first = ibase + (long long)a * n;
#pragma unroll
  for (int c = 0; c < kC; ++c) {
    const uint32_t meta = ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(cid[c], cap - 1));
    const uint32_t cand = pm_z[c % 3] & ~sampled;
    for (int s = 0; s < cnt[c]; s += kSliceItems) {
      const uint32_t count = (uint32_t)min(kSliceItems, cnt[c] - s) | (shared ? kSliceShared : 0u);
      sl.list[2 * k] = make_uint4((uint32_t)(first + off[c] + s), count, pos, cand);
      sl.list[2 * k + 1] = make_uint4(meta, (uint32_t)j, 0u, 0u);
      ++k;
    }
  }
}

// Phase A for one robot, where an action's scenarios fall into at most a few
// children: observation z in {0, 1, 2} and whether the step ended the world
// give 6 codes (a move or Sample gives every scenario of a job one code, a
// Sense at most two). Each warp expands whole actions: pass 1 steps the
// action's scenarios 32 at a time, keeps each scenario's code in shared memory
// and counts codes, first positions and exact reward sums with ballots and
// warp reductions; pass 2 numbers the children by first position and writes
// the grouped positions and the rollout items, re-stepping only the actions
// that draw no random numbers (a Sense leaves the state as it was). The result
// is identical to the general grouping; no barrier is needed inside the job.
__device__ void rs1_group_job(RSGroupSmem& S, const RSModel<1>& M, int j, long long ibase, Items<1> items,
                              DevWork* work, unsigned long long& steps, const LeafBlocks& lb, const Slices& sl) {
  constexpr int kC = 6;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  gather_update<1>(S, M, true, steps);
  const dsp_leaf_job& J = S.J;
  const int n = J.n_scen, depth = J.depth, A = J.n_actions, cap = J.child_cap;
  const bool blocks = lb.leaf != nullptr;
  if (blocks) {
    for (int p = tid; p < n; p += (int)blockDim.x) put_leaf(lb, j, n, p, S.leaf[0][p], S.leaf[2][p], S.leaf[3][p]);
    put_blocks(lb, j, n, A);
  }
  // A tree node's scenarios share the robot's position and sampled mask (both
  // observed); they differ in the rocks' states and random streams. When the
  // job's leaves do (checked here), a move or a terminal leaf gives every
  // scenario the same step (one child, the grouped positions in their
  // original order) and a Sense compares each scenario's sensor word with
  // one threshold. The results are those of the general path below.
  bool same = true;
  for (int p = tid; p < n; p += (int)blockDim.x)
    same = same && S.leaf[0][p] == S.leaf[0][0] && S.leaf[3][p] == S.leaf[3][0];
  const bool uniform = __syncthreads_and(same ? 1 : 0) != 0;
  // the shared position and sampled mask (a move's or a terminal leaf's step
  // reads neither the rocks' states nor the random streams)
  RSS rep;
  rep.pos[0] = S.leaf[0][0];
  rep.pos[1] = 0u;
  rep.good = 0u;
  rep.sampled = S.leaf[3][0];
  rep.scen = 0u;
  const uint32_t lt = lanemask_lt();
  uint8_t* codes = S.code1[warp];
  const uint32_t pm_job = S.pm_job;
  const int nwarps = (int)(blockDim.x >> 5);
  for (int a = warp; a < A; a += nwarps) {
    const int aa = J.first_action + a;
    int cnt[kC], first[kC], rsum[kC];  // |reward sum| <= 100 * 512 fits 32 bits
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      cnt[c] = 0;
      first[c] = 0x7FFFFFFF;
      rsum[c] = 0;
    }
    const bool rep_term = M.terminal(rep);
    const bool same_step = uniform && (aa < 4 || rep_term);  // one code and reward for all
    const bool same_sense = uniform && aa >= 5 && !rep_term;
    RSS rep_next = rep;
    int rep_code = 0, rep_r = 0;
    uint64_t sense_thr = 0;
    uint32_t sense_bit = 0;
    if (same_step) {
      uint64_t key;
      rep_r = (int)M.step(rep_next, aa, depth, key);
      rep_code = (int)(key & 3u) + 3 * (int)(key >> 62);
    } else if (same_sense) {
      const int i = aa - 5;
      const int x = (int)(rep.pos[0] & 0xFFu), y = (int)((rep.pos[0] >> 8) & 0xFFu);
      const int dx = x - (S.c.rock_xy[i] & 0xFF), dy = y - (S.c.rock_xy[i] >> 8);
      sense_thr = __ldg(M.thresh + dx * dx + dy * dy);
      sense_bit = 1u << i;
    }
    if (same_step) {
      // (an unrolled loop over the codes keeps the arrays in registers)
#pragma unroll
      for (int c = 0; c < kC; ++c)
        if (c == rep_code) {
          cnt[c] = n;
          first[c] = 0;
          rsum[c] = n * rep_r;
        }
      if (!rep_term && lane == 0) steps += (unsigned long long)n;
    }
    for (int w = 0; !same_step && w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      int code = kC, rint = 0;
      if (p < n && same_sense) {
        // Sense of rock i: the reading is correct iff the sensor word is
        // below the threshold of the (shared) distance; z = 1 reads good
        steps += 1;
        const bool correct = (uint64_t)S.sense[0][p] < sense_thr;
        const bool is_good = (S.leaf[2][p] & sense_bit) != 0u;
        code = correct == is_good ? 1 : 2;
        codes[p] = (uint8_t)code;
      } else if (p < n) {
        RSS s;
        s.pos[0] = S.leaf[0][p];
        s.pos[1] = 0u;
        s.good = S.leaf[2][p];
        s.sampled = S.leaf[3][p];
        s.scen = S.leaf[4][p];
        if (!M.terminal(s)) steps += 1;
        uint64_t key;
        const uint32_t sw[2] = {S.sense[0][p], 0u};
        rint = (int)M.step(s, aa, depth, key, sw);
        code = (int)(key & 3u) + 3 * (int)(key >> 62);
        codes[p] = (uint8_t)code;
      }
      // codes held by the chunk (warp-uniform): absent codes are skipped
      const uint32_t present = __reduce_or_sync(0xFFFFFFFFu, code < kC ? 1u << code : 0u);
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        if (present & (1u << c)) {
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, code == c);
          if (cnt[c] == 0) first[c] = w * 32 + __ffs(b) - 1;
          cnt[c] += __popc(b);
          rsum[c] += __reduce_add_sync(0xFFFFFFFFu, code == c ? rint : 0);
        }
      }
    }
    __syncwarp();
    // children in order of first position
    int cid[kC], off[kC], nch = 0;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      cid[c] = -1;
      off[c] = 0;
      if (cnt[c] > 0) {
        nch += 1;
        int k = 0, o = 0;
#pragma unroll
        for (int c2 = 0; c2 < kC; ++c2)
          if (cnt[c2] > 0 && first[c2] < first[c]) {
            k += 1;
            o += cnt[c2];
          }
        cid[c] = k;
        off[c] = o;
      }
    }
    // per-action results: counts, offsets, keys, exact reward sums; u and l start at 0
    if (lane == 0) {
      J.child_count[a] = nch;
      if (nch > cap) report(work, kStatusOverflow);
      if (nch <= cap) J.child_off[(size_t)a * (cap + 1) + nch] = n;
#pragma unroll
      for (int c = 0; c < kC; ++c)
        if (cnt[c] > 0 && cid[c] < cap) {
          const size_t o = (size_t)a * cap + cid[c];
          J.child_off[(size_t)a * (cap + 1) + cid[c]] = off[c];
          J.child_key[o] = (uint64_t)(c % 3) | ((uint64_t)(c / 3) << 62);
          J.rew_sum[o] = (long long)rsum[c] * 4294967296LL;
          J.u_sum[o] = 0;
          J.l_sum[o] = 0;
        }
    }
    // the item's positive-counter mask: a Sense reading moves rock i's counter
    // by +-1 (clamped to +-127, as the belief bookkeeping does)
    uint32_t pm_z[3] = {pm_job, pm_job, pm_job};
    if (aa >= 5) {
      const int i = aa - 5;
      const int c0 = (int)J.hist[i];
      const int cg = min(c0 + 1, 127), cb = max(c0 - 1, -127);
      pm_z[1] = cg > 0 ? (pm_job | (1u << i)) : (pm_job & ~(1u << i));
      pm_z[2] = cb > 0 ? (pm_job | (1u << i)) : (pm_job & ~(1u << i));
    }
    // a shared-position job's children: the state after the step is the job's
    // (a move or a terminal leaf: rep_next; a Sense: as it was; a Sample on a
    // rock: that rock sampled, and bad in every scenario), so with a slice
    // list the items hold only the good masks and the slices the rest
    const int rock_here = S.c.cell_rock[(int)((rep.pos[0] >> 8) & 0xFFu) * M.n + (int)(rep.pos[0] & 0xFFu)];
    const uint32_t sample_bit = (uniform && aa == 4 && !rep_term && rock_here != 0xFF) ? (1u << rock_here) : 0u;
    const bool slim = uniform && sl.list != nullptr && !items.full;
    if (lane == 0)
      put_slices<kC>(sl, ibase, a, n, cnt, off, cid, cap, depth, j, slim, same_step ? rep_next.pos[0] : rep.pos[0],
                     pm_z, same_step ? rep_next.sampled : (rep.sampled | sample_bit), work);
    // grouped positions and rollout items
    int run[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) run[c] = 0;
    for (int w = 0; w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      const int code = p < n ? (same_step ? rep_code : (int)codes[p]) : kC;
      int q = p, mycid = 0;  // one child: the original order
      if (!same_step) {
        q = 0;
#pragma unroll
        for (int c = 0; c < kC; ++c) {
          if (cnt[c] > 0) {  // the action's codes (warp-uniform)
            const uint32_t b = __ballot_sync(0xFFFFFFFFu, code == c);
            if (code == c) {
              q = off[c] + run[c] + __popc(b & lt);
              mycid = cid[c];
            }
            run[c] += __popc(b);
          }
        }
      }
      if (p < n) J.perm[(size_t)a * n + q] = (uint16_t)p;
      if (p < n && !blocks && slim) {
        items.put_good((size_t)(ibase + (long long)a * n + q), S.leaf[2][p] & ~sample_bit);
      } else if (p < n && !blocks) {
        RSS s;
        s.pos[0] = S.leaf[0][p];
        s.pos[1] = 0u;
        s.good = S.leaf[2][p];
        s.sampled = S.leaf[3][p];
        s.scen = S.leaf[4][p];
        if (same_step) {
          // a move (or a terminal leaf) leaves the rocks as they were
          s.pos[0] = rep_next.pos[0];
          s.sampled = rep_next.sampled;
        } else if (aa < 5) {
          uint64_t k;
          M.step(s, aa, depth, k);
        }
        const int z = code % 3;
        const uint32_t pm = z == 1 ? pm_z[1] : (z == 2 ? pm_z[2] : pm_z[0]);
        const size_t it = (size_t)(ibase + (long long)a * n + q);
        items.put(it, s, pm, ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(mycid, cap - 1)), (uint32_t)j);
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Phase A for one robot when a job holds more scenarios than shared memory
// takes (kMaxScen < n <= kMaxScenLarge): the gather writes the leaf's states
// to the job's leaf-state block in global memory (it stays in L2) instead of
// shared memory, and the second pass recomputes each scenario's sensor word,
// step and observation code instead of keeping them. The placement is the
// same as rs1_group_job's, so the result is identical.
__device__ void rs1_group_job_large(RSGroupSmem& S, const RSModel<1>& M, int j, long long ibase, Items<1> items,
                                    DevWork* work, unsigned long long& steps, const LeafBlocks& lb,
                                    const Slices& sl) {
  constexpr int kC = 6;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const dsp_leaf_job& J = S.J;
  const int n = J.n_scen, depth = J.depth, A = J.n_actions, cap = J.child_cap;
  uint32_t* const L = J.leaf_states;  // field-major, capacity n (required by the host for n > kMaxScen)
  for (int p = tid; p < n; p += (int)blockDim.x) {
    RSS s = M.load(J.parent, J.parent_cap, J.idx[p]);
    if (J.last_action >= 0) {
      if (!M.terminal(s)) steps += 1;
      uint64_t k;
      M.step(s, J.last_action, depth - 1, k);
    }
    M.store(s, L, n, p);
    if (lb.leaf != nullptr) put_leaf(lb, j, n, p, s.pos[0], s.good, s.sampled);
  }
  if (lb.leaf != nullptr) put_blocks(lb, j, n, A);
  if (tid == 0) {
    uint32_t h[8];
    const uint32_t* hw = reinterpret_cast<const uint32_t*>(J.hist);
#pragma unroll
    for (int k = 0; k < 8; ++k) h[k] = hw[k];
    S.pm_job = positive_mask(h, M.m);
  }
  __syncthreads();
  const uint32_t lt = lanemask_lt();
  const uint32_t pm_job = S.pm_job;
  const int nwarps = (int)(blockDim.x >> 5);
  for (int a = warp; a < A; a += nwarps) {
    const int aa = J.first_action + a;
    int cnt[kC], first[kC], rsum[kC];  // |reward sum| <= 100 * 8192 fits 32 bits
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      cnt[c] = 0;
      first[c] = 0x7FFFFFFF;
      rsum[c] = 0;
    }
    for (int w = 0; w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      int code = kC, rint = 0;
      if (p < n) {
        RSS s = M.load(L, n, p);
        if (!M.terminal(s)) steps += 1;
        uint64_t key;
        const uint32_t sw[2] = {M.sense_word(s.scen, depth, 0), 0u};
        rint = (int)M.step(s, aa, depth, key, sw);
        code = (int)(key & 3u) + 3 * (int)(key >> 62);
      }
      const uint32_t present = __reduce_or_sync(0xFFFFFFFFu, code < kC ? 1u << code : 0u);
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        if (present & (1u << c)) {
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, code == c);
          if (cnt[c] == 0) first[c] = w * 32 + __ffs(b) - 1;
          cnt[c] += __popc(b);
          rsum[c] += __reduce_add_sync(0xFFFFFFFFu, code == c ? rint : 0);
        }
      }
    }
    int cid[kC], off[kC], nch = 0;
#pragma unroll
    for (int c = 0; c < kC; ++c) {
      cid[c] = -1;
      off[c] = 0;
      if (cnt[c] > 0) {
        nch += 1;
        int k = 0, o = 0;
#pragma unroll
        for (int c2 = 0; c2 < kC; ++c2)
          if (cnt[c2] > 0 && first[c2] < first[c]) {
            k += 1;
            o += cnt[c2];
          }
        cid[c] = k;
        off[c] = o;
      }
    }
    if (lane == 0) {
      J.child_count[a] = nch;
      if (nch > cap) report(work, kStatusOverflow);
      if (nch <= cap) J.child_off[(size_t)a * (cap + 1) + nch] = n;
      const uint32_t no_pm[3] = {0u, 0u, 0u};
      put_slices<kC>(sl, ibase, a, n, cnt, off, cid, cap, depth, j, false, 0u, no_pm, 0u, work);
#pragma unroll
      for (int c = 0; c < kC; ++c)
        if (cnt[c] > 0 && cid[c] < cap) {
          const size_t o = (size_t)a * cap + cid[c];
          J.child_off[(size_t)a * (cap + 1) + cid[c]] = off[c];
          J.child_key[o] = (uint64_t)(c % 3) | ((uint64_t)(c / 3) << 62);
          J.rew_sum[o] = (long long)rsum[c] * 4294967296LL;
          J.u_sum[o] = 0;
          J.l_sum[o] = 0;
        }
    }
    uint32_t pm_z[3] = {pm_job, pm_job, pm_job};
    if (aa >= 5) {
      const int i = aa - 5;
      const int c0 = (int)J.hist[i];
      const int cg = min(c0 + 1, 127), cb = max(c0 - 1, -127);
      pm_z[1] = cg > 0 ? (pm_job | (1u << i)) : (pm_job & ~(1u << i));
      pm_z[2] = cb > 0 ? (pm_job | (1u << i)) : (pm_job & ~(1u << i));
    }
    int run[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) run[c] = 0;
    for (int w = 0; w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      int code = kC;
      RSS s;
      if (p < n) {
        s = M.load(L, n, p);
        uint64_t key;
        const uint32_t sw[2] = {M.sense_word(s.scen, depth, 0), 0u};
        M.step(s, aa, depth, key, sw);
        code = (int)(key & 3u) + 3 * (int)(key >> 62);
      }
      int q = 0, mycid = 0;
#pragma unroll
      for (int c = 0; c < kC; ++c) {
        if (cnt[c] > 0) {
          const uint32_t b = __ballot_sync(0xFFFFFFFFu, code == c);
          if (code == c) {
            q = off[c] + run[c] + __popc(b & lt);
            mycid = cid[c];
          }
          run[c] += __popc(b);
        }
      }
      if (p < n) J.perm[(size_t)a * n + q] = (uint16_t)p;
      if (p < n && lb.leaf == nullptr) {
        const int z = code % 3;
        const uint32_t pm = z == 1 ? pm_z[1] : (z == 2 ? pm_z[2] : pm_z[0]);
        const size_t it = (size_t)(ibase + (long long)a * n + q);
        items.put(it, s, pm, ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(mycid, cap - 1)), (uint32_t)j);
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Phase A for two robots, organised like rs1_group_job: each warp expands
// whole actions in two passes over 32-scenario chunks. The codes (z0 * 3 + z1
// and whether the step ended the world, up to 18) are too many for
// registers, so each warp keeps its per-code counts, first positions, reward
// sums, child numbers, offsets and running counts in its own rows of the
// shared tables. Lanes with the same code meet through __match_any_sync and
// their leader updates the code's row; the warp's own __syncwarp orders the
// updates. The result is identical to the general grouping.
__device__ void rs2_group_job(RSGroupSmem& S, const RSModel<2>& M, int j, long long ibase, int a_begin, int a_end,
                              bool first_unit, Items<2> items, DevWork* work, unsigned long long& steps,
                              const Slices& sl) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  gather_update<2>(S, M, first_unit, steps);
  const dsp_leaf_job& J = S.J;
  const int n = J.n_scen, depth = J.depth, cap = J.child_cap;
  // with a slice list: whether the job's scenarios share both robots' cells
  // and the sampled mask (a tree node's do), so that each child's items share
  // their state after the step (the slice holds it; the items their good
  // masks)
  bool same = true;
  if (sl.list != nullptr)
    for (int p = tid; p < n; p += (int)blockDim.x)
      same = same && S.leaf[0][p] == S.leaf[0][0] && S.leaf[1][p] == S.leaf[1][0] && S.leaf[3][p] == S.leaf[3][0];
  const bool slim = sl.list != nullptr && !items.full && __syncthreads_and(same ? 1 : 0) != 0;
  const uint32_t lt = lanemask_lt();
  uint8_t* codes = S.code1[warp];
  int* cnt = S.wcnt[warp];
  int* first = S.wfirst[warp];
  int* run = S.wpre[warp];
  int* off = S.aoff[warp];
  int* cid = S.acid[warp];
  unsigned long long* rsum = S.sr[warp];
  const int nwarps = (int)(blockDim.x >> 5);
  for (int a = a_begin + warp; a < a_end; a += nwarps) {
    const int aa = J.first_action + a;
    const int a0 = aa / M.per, a1 = aa - a0 * M.per;
    if (lane < kCodes) {
      cnt[lane] = 0;
      first[lane] = 0x7FFFFFFF;
      rsum[lane] = 0ull;
    }
    __syncwarp();
    // pass 1: step, record each scenario's code, per-code counts and sums
    for (int w = 0; w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      int code = kCodes, rint = 0;
      if (p < n) {
        RSS s;
        s.pos[0] = S.leaf[0][p];
        s.pos[1] = S.leaf[1][p];
        s.good = S.leaf[2][p];
        s.sampled = S.leaf[3][p];
        s.scen = S.leaf[4][p];
        if (!M.terminal(s)) steps += 1;
        uint64_t key;
        const uint32_t sw[2] = {S.sense[0][p], S.sense[1][p]};
        rint = (int)M.step(s, aa, depth, key, sw);
        code = (int)(key & 0xFu) + 9 * (int)(key >> 62);
        codes[p] = (uint8_t)code;
      }
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, code);
      const int rs = __reduce_add_sync(peers, rint);
      if (p < n && lane == __ffs(peers) - 1) {
        if (cnt[code] == 0) first[code] = p;
        cnt[code] += __popc(peers);
        rsum[code] += (unsigned long long)((long long)rs * 4294967296LL);
      }
      __syncwarp();
    }
    // children in order of first position
    int nch = 0;
    if (lane < kCodes) {
      int k = 0, o = 0;
      const int mine = first[lane];
      if (cnt[lane] > 0)
        for (int c2 = 0; c2 < kCodes; ++c2)
          if (cnt[c2] > 0 && first[c2] < mine) {
            k += 1;
            o += cnt[c2];
          }
      cid[lane] = cnt[lane] > 0 ? k : -1;
      off[lane] = o;
      run[lane] = 0;
    }
    nch = __popc(__ballot_sync(0xFFFFFFFFu, lane < kCodes && cnt[lane] > 0));
    __syncwarp();
    // per-action results: counts, offsets, keys, exact reward sums; u and l start at 0
    if (lane == 0) {
      J.child_count[a] = nch;
      if (nch > cap) report(work, kStatusOverflow);
      if (nch <= cap) J.child_off[(size_t)a * (cap + 1) + nch] = n;
    }
    if (lane < kCodes && cid[lane] >= 0 && cid[lane] < cap) {
      const size_t o = (size_t)a * cap + cid[lane];
      J.child_off[(size_t)a * (cap + 1) + cid[lane]] = off[lane];
      J.child_key[o] = (uint64_t)(lane % 9) | ((uint64_t)(lane / 9) << 62);
      J.rew_sum[o] = (long long)rsum[lane];
      J.u_sum[o] = 0;
      J.l_sum[o] = 0;
    }
    // the child's positive-counter mask depends only on the observation
    // (z0 * 3 + z1 < 9): lane c holds the one of observation c
    uint32_t pm_obs = S.pm_job;
    if (lane < 9) {
      uint32_t h[8];
      const uint32_t* hw = reinterpret_cast<const uint32_t*>(J.hist);
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] = hw[k];
      M.observe(h, pm_obs, aa, (uint64_t)lane);
    }
    // the children's slices: lane c < kCodes takes code c's, after a scan of
    // the codes' slice counts; one atomic per action reserves them. A shared
    // job's state after the step is scenario 0's (both robots' moves and
    // Samples applied; a Sense leaves it as it was); `clear` holds the rocks
    // the step sampled, bad in every scenario afterwards.
    uint32_t clear = 0u;
    if (sl.list != nullptr) {
      RSS nxt;
      nxt.pos[0] = S.leaf[0][0];
      nxt.pos[1] = S.leaf[1][0];
      nxt.good = S.leaf[2][0];
      nxt.sampled = S.leaf[3][0];
      nxt.scen = S.leaf[4][0];
      int zz;
      if (a0 < 5) M.robot_step(nxt, 0, a0, depth, zz);
      if (a1 < 5) M.robot_step(nxt, 1, a1, depth, zz);
      clear = nxt.sampled & ~S.leaf[3][0];
      const int mc = lane < kCodes ? cnt[lane] : 0;
      const int ns = (mc + kSliceItemsTwo - 1) / kSliceItemsTwo;
      int incl = ns;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
      }
      const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      unsigned int base = 0u;
      if (lane == 0 && total > 0) base = atomicAdd(sl.count, (unsigned int)total);
      base = __shfl_sync(0xFFFFFFFFu, base, 0);
      const uint32_t pmc = __shfl_sync(0xFFFFFFFFu, pm_obs, lane % 9);
      if (total > 0 && base + (unsigned int)total > sl.cap) {
        if (lane == 0) report(work, kStatusOverflow);
      } else if (ns > 0) {
        unsigned int k = base + (unsigned int)(incl - ns);
        const uint32_t meta = ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(cid[lane], cap - 1));
        const uint32_t cand = pmc & ~nxt.sampled;
        const long long first_it = ibase + (long long)a * n + off[lane];
        for (int s0 = 0; s0 < mc; s0 += kSliceItemsTwo) {
          const uint32_t count = (uint32_t)min(kSliceItemsTwo, mc - s0) | (slim ? kSliceShared : 0u);
          sl.list[2 * k] = make_uint4((uint32_t)(first_it + s0), count, nxt.pos[0], cand);
          sl.list[2 * k + 1] = make_uint4(meta, (uint32_t)j, nxt.pos[1], 0u);
          ++k;
        }
      }
    }
    // pass 2: grouped positions and rollout items; only Sense draws random
    // numbers and it leaves the state as it was, so each robot's other
    // actions are simply applied again
    for (int w = 0; w * 32 < n; ++w) {
      const int p = w * 32 + lane;
      const int code = p < n ? (int)codes[p] : kCodes;
      const uint32_t peers = __match_any_sync(0xFFFFFFFFu, code);
      int q = 0, mycid = 0;
      if (p < n) {
        q = off[code] + run[code] + __popc(peers & lt);
        mycid = cid[code];
      }
      __syncwarp();
      if (p < n && lane == __ffs(peers) - 1) run[code] += __popc(peers);
      if (slim) {
        // the item's good mask alone (its slice holds the rest)
        if (p < n) {
          J.perm[(size_t)a * n + q] = (uint16_t)p;
          items.put_good((size_t)(ibase + (long long)a * n + q), S.leaf[2][p] & ~clear);
        }
        __syncwarp();
        continue;
      }
      RSS s;
      if (p < n) {
        s.pos[0] = S.leaf[0][p];
        s.pos[1] = S.leaf[1][p];
        s.good = S.leaf[2][p];
        s.sampled = S.leaf[3][p];
        s.scen = S.leaf[4][p];
        int z;
        if (a0 < 5) M.robot_step(s, 0, a0, depth, z);
        if (a1 < 5) M.robot_step(s, 1, a1, depth, z);
        J.perm[(size_t)a * n + q] = (uint16_t)p;
      }
      const uint32_t pm = __shfl_sync(0xFFFFFFFFu, pm_obs, p < n ? code % 9 : 0);
      if (p < n) {
        const size_t it = (size_t)(ibase + (long long)a * n + q);
        items.put(it, s, pm, ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(mycid, cap - 1)), (uint32_t)j);
      }
      __syncwarp();
    }
  }
  __syncthreads();
}

// One unit of phase A: actions [a_begin, a_end) of job j (one robot: always
// the whole job); `first` marks the job's first unit. kLarge: one-robot jobs
// above kMaxScen scenarios may occur (not in the queue, which refuses them).
template <int R, bool kLarge = true>
__device__ __forceinline__ void group_job(RSGroupSmem& S, const RSModel<R>& M, int j, long long ibase, int a_begin,
                                          int a_end, bool first, Items<R> items, DevWork* work,
                                          unsigned long long& steps, const LeafBlocks& lb = LeafBlocks{},
                                          const Slices& sl = Slices{}) {
  if constexpr (R == 1) {
    if (kLarge && S.J.n_scen > kMaxScen)
      rs1_group_job_large(S, M, j, ibase, items, work, steps, lb, sl);
    else
      rs1_group_job(S, M, j, ibase, items, work, steps, lb, sl);
  } else
    rs2_group_job(S, M, j, ibase, a_begin, a_end, first, items, work, steps, sl);
}

// kLarge: one-robot jobs above kMaxScen scenarios may occur (their path is
// compiled in only then, so that the common path keeps its registers)
template <int R, bool kLarge>
__global__ void __launch_bounds__(kBlockA, 2) rs_group_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                             const dsp_leaf_job* __restrict__ jobs,
                                                             const long long* __restrict__ item_base,
                                                             const int* __restrict__ order, int n_jobs,
                                                             unsigned int* head, uint32_t plan_step,
                                                             Items<R> items, int splits, LeafBlocks lb,
                                                             Slices sl) {
  __shared__ RSGroupSmem S;
  load_rs_consts(S.c, gm);
  const RSModel<R> M = make_rs<R>(gm, &S.c, plan_step);
  unsigned long long steps = 0;
  __syncthreads();
  // unit k: part k % splits of job order[k / splits], its actions in runs of
  // a multiple of the CTA's warps
  const int nwarps = (int)(blockDim.x >> 5);
  while (true) {
    if (threadIdx.x == 0) {
      const int k = (int)atomicAdd(head, 1u);
      const int q = k / splits;
      S.job = q < n_jobs ? (order != nullptr ? order[q] : q) : n_jobs;
      S.part = k - q * splits;
      if (S.job < n_jobs) S.J = jobs[S.job];
    }
    __syncthreads();
    const int j = S.job;
    if (j >= n_jobs) break;
    const int A = S.J.n_actions;
    const int run = nwarps * ((A + splits * nwarps - 1) / (splits * nwarps));
    const int a_begin = S.part * run, a_end = min(A, a_begin + run);
    // both ways end at a barrier (group_job's last), so thread 0 may take the
    // next unit (the condition is the same for the whole CTA)
    if (a_begin < a_end)
      group_job<R, kLarge>(S, M, j, item_base != nullptr ? item_base[j] : 0, a_begin, a_end, S.part == 0, items, work,
                   steps, lb, sl);
    else
      __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// Exact sum of an int64 over the full warp from three 32-bit warp reductions:
// x = hi * 2^32 + lo with lo unsigned, and lo split in 16-bit halves, so no
// partial sum of 32 lanes overflows.
__device__ __forceinline__ long long warp_sum64(long long x) {
  const uint32_t lo = (uint32_t)(unsigned long long)x;
  const int hi = (int)(x >> 32);
  const unsigned a = __reduce_add_sync(0xFFFFFFFFu, lo & 0xFFFFu);
  const unsigned b = __reduce_add_sync(0xFFFFFFFFu, lo >> 16);
  const int h = __reduce_add_sync(0xFFFFFFFFu, hi);
  return (long long)h * 4294967296LL + (long long)b * 65536LL + (long long)a;
}

// u0 of a state whose robots stand at p0 (and p1) as upper() computes it,
// split for a warp whose items share the robots' cells: lane i's term of rock
// i (10 G[d], d the distance of its nearest live robot), and the live
// robots' exit terms added in robot order.
template <int R>
__device__ __forceinline__ float upper_term(const RSModel<R>& M, uint32_t p0, uint32_t p1, int i) {
  if (i >= M.m) return 0.0f;
  int bestd = 1 << 30;
  if (!((p0 >> 16) & 1u))
    bestd = min(bestd, (int)M.nkey[i * M.nn + (int)(p0 & 0xFFu) + (int)((p0 >> 8) & 0xFFu) * M.n] >> 7);
  if (R == 2 && !((p1 >> 16) & 1u))
    bestd = min(bestd, (int)M.nkey[i * M.nn + (int)(p1 & 0xFFu) + (int)((p1 >> 8) & 0xFFu) * M.n] >> 7);
  return __fmul_rn(10.0f, M.sh->G[bestd]);
}
template <int R>
__device__ __forceinline__ float upper_exits(const RSModel<R>& M, uint32_t p0, uint32_t p1, float u) {
  if (!((p0 >> 16) & 1u)) u = __fadd_rn(u, __fmul_rn(10.0f, M.sh->G[M.n - 1 - (int)(p0 & 0xFFu)]));
  if (R == 2 && !((p1 >> 16) & 1u)) u = __fadd_rn(u, __fmul_rn(10.0f, M.sh->G[M.n - 1 - (int)(p1 & 0xFFu)]));
  return u;
}
template <int R>
__device__ __forceinline__ bool rs_terminal(uint32_t p0, uint32_t p1) {
  return R == 1 ? ((p0 >> 16) & 1u) != 0u : (((p0 >> 16) & 1u) && ((p1 >> 16) & 1u));
}

// A warp's chunk claims, used by its lane 0 and kept in shared memory (one
// record per warp) so that no register carries them through the rollouts.
// Every warp of the grid draws chunks from one counter; one atomic per
// 32-item chunk came near the rate at which the memory system serves atomics
// on one address, and the warps queued on the claims. So a claim takes
// kBatch chunks, handed out one at a time.
constexpr int kMaxWarpsB = 16;  // rollout-phase CTAs of at most 512 threads
struct ChunkClaims {
  static constexpr unsigned int kBatch = 4;
  unsigned int next, left;
  __device__ __forceinline__ unsigned int take(unsigned int* head) {
    if (left == 0) {
      next = atomicAdd(head, kBatch);
      left = kBatch;
    }
    --left;
    return next++;
  }
};

// Phase B for one 32-item chunk (one whole warp calls it), the lane's compact
// item given (ok: the lane holds an item): u0 and the rollout, then the sums
// into the children. One robot reads the child's sum pointers from the job
// table before the rollout, so their latency hides behind it.
template <int R>
__device__ __forceinline__ void rs_rollout_values(const RSModel<R>& M, const dsp_leaf_job* __restrict__ jobs, bool ok,
                                                  const RSS& s, uint32_t pm, uint32_t meta, uint32_t job,
                                                  unsigned long long& steps) {
  const int lane = threadIdx.x & 31;
  {
    uint32_t slot = 0;
    long long fu = 0, fl = 0;
    int64_t* usum = nullptr;
    int64_t* lsum = nullptr;
    // u0 of a chunk whose items share the robot's cell and the depth (a
    // child's items do, and so do an action's): rock i's term 10 G[d_i] from
    // lane i, each lane adding its good rocks' terms in index order, as
    // upper() does (lane 0 always holds an item)
    float u_shared = 0.0f;
    const uint32_t p0 = __shfl_sync(0xFFFFFFFFu, s.pos[0], 0);
    const uint32_t p1 = R == 2 ? __shfl_sync(0xFFFFFFFFu, s.pos[1], 0) : 0u;
    const uint32_t d0 = __shfl_sync(0xFFFFFFFFu, meta >> 24, 0);
    const bool shared =
        __all_sync(0xFFFFFFFFu, !ok || (s.pos[0] == p0 && (R == 1 || s.pos[1] == p1) && (meta >> 24) == d0)) &&
        !rs_terminal<R>(p0, p1) && (int)d0 + 1 < M.D;
    if (shared) {
      const float w = upper_term<R>(M, p0, p1, lane);
      const uint32_t g = s.good;
      for (int i = 0; i < M.m; ++i) {
        const float wi = __shfl_sync(0xFFFFFFFFu, w, i);
        if ((g >> i) & 1u) u_shared = __fadd_rn(u_shared, wi);
      }
      u_shared = upper_exits<R>(M, p0, p1, u_shared);
    }
    if (!ok) job = 0xFFFFFFFFu;
    if (ok) {
      if (R == 1) {  // one robot: loaded before its short rollout (two robots: after, fewer registers)
        usum = jobs[job].u_sum;
        lsum = jobs[job].l_sum;
      }
      slot = meta & 0xFFFFFFu;
      const int depth = (int)(meta >> 24);
      float u = 0.0f, v = 0.0f;
      if (!M.terminal(s)) {
        u = shared ? u_shared : ((depth + 1 >= M.D) ? M.tail(s) : M.upper(s));
        v = M.rollout(s, pm, depth + 1, steps);
      }
      fu = to_fixed(u);
      fl = to_fixed(v);
      if (R == 2) {
        usum = jobs[job].u_sum;
        lsum = jobs[job].l_sum;
      }
    }
    // runs of lanes with the same (job, slot) are contiguous
    const uint32_t pj = __shfl_up_sync(0xFFFFFFFFu, job, 1);
    const uint32_t ps = __shfl_up_sync(0xFFFFFFFFu, slot, 1);
    const uint32_t starts = __ballot_sync(0xFFFFFFFFu, lane == 0 || pj != job || ps != slot);
    if (starts == 1u) {
      // the whole chunk is one child (lane 0 always holds an item, so every
      // lane does): one warp sum per value
      fu = warp_sum64(fu);
      fl = warp_sum64(fl);
      if (lane == 0 && ok) {
        sum_add(usum + slot, fu);
        sum_add(lsum + slot, fl);
      }
      return;
    }
    // else a segmented scan
    const uint32_t le = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
    const int lo = 31 - __clz(starts & le);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      long long yu = __shfl_up_sync(0xFFFFFFFFu, fu, d);
      long long yl = __shfl_up_sync(0xFFFFFFFFu, fl, d);
      if (lane - d >= lo) {
        fu += yu;
        fl += yl;
      }
    }
    const bool last = lane == 31 || ((starts >> (lane + 1)) & 1u);
    if (ok && last) {
      sum_add(usum + slot, fu);
      sum_add(lsum + slot, fl);
    }
  }
}

// Phase B for one 32-item chunk of the item list read from global memory.
template <int R>
__device__ __forceinline__ void rs_rollout_chunk(const RSModel<R>& M, const dsp_leaf_job* __restrict__ jobs,
                                                 Items<R> items, long long chunk, unsigned long long& steps) {
  const long long it = chunk * 32 + (threadIdx.x & 31);
  const bool ok = it < items.total;
  RSS s;
  uint32_t pm = 0, meta = 0, job = 0;  // compact items: pm is the candidate mask, sampled 0
  if (ok) items.get_compact((size_t)it, s, pm, meta, job);
  rs_rollout_values<R>(M, jobs, ok, s, pm, meta, job, steps);
}

// Per warp, two chunks of compact items in shared memory: the one being
// rolled out and the next, copied in with cp.async meanwhile, so that a
// chunk's item loads do not stall the warp (its rollouts are short now).
template <int R>
__device__ __forceinline__ void stage_chunk_async(uint32_t* buf, const Items<R>& items, long long chunk) {
  constexpr int F = Items<R>::kCompactFields;
  const int lane = threadIdx.x & 31;
  const long long it = chunk * 32 + lane;
  if (it < items.total)
#pragma unroll
    for (int k = 0; k < F; ++k) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(buf + k * 32 + lane);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(items.f(k) + it) : "memory");
    }
}

// One robot's unit of phase B: two consecutive 32-item chunks, staged
// together (one commit group).
constexpr int kUnitChunks = 2;
template <int R>
__device__ __forceinline__ void stage_unit(uint32_t* buf, const Items<R>& items, long long unit) {
  constexpr int F = Items<R>::kCompactFields;
#pragma unroll
  for (int c = 0; c < kUnitChunks; ++c) stage_chunk_async<R>(buf + c * F * 32, items, unit * kUnitChunks + c);
  asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int R>
constexpr size_t rs_stage_bytes(int block) {
  return (size_t)(block / 32) * 2 * kUnitChunks * Items<R>::kCompactFields * 32 * sizeof(uint32_t);
}

// Phase B for a unit whose 64 items all belong to one child: the same
// positions, candidate set and depth, so one trajectory (rollout_one2, or
// rollout_two2 for two robots) gives both of each lane's values; u0's
// per-rock terms come from lane i as in rs_rollout_values, and the child's
// sums take one warp sum each.
template <int R>
__device__ __forceinline__ void rs_rollout_pair(const RSModel<R>& M, const dsp_leaf_job* __restrict__ jobs,
                                                uint32_t p0, uint32_t p1, uint32_t good_a, uint32_t good_b,
                                                uint32_t cand, uint32_t meta, uint32_t job,
                                                unsigned long long& steps) {
  const int lane = threadIdx.x & 31;
  int64_t* usum = jobs[job].u_sum;
  int64_t* lsum = jobs[job].l_sum;
  const uint32_t slot = meta & 0xFFFFFFu;
  const int depth = (int)(meta >> 24);
  float ua = 0.0f, ub = 0.0f, va = 0.0f, vb = 0.0f;
  if (!rs_terminal<R>(p0, p1)) {
    if (depth + 1 >= M.D) {
      RSS s;
      s.pos[0] = p0;
      s.pos[1] = p1;
      ua = ub = M.tail(s);
    } else {
      const float w = upper_term<R>(M, p0, p1, lane);
      for (int i = 0; i < M.m; ++i) {
        const float wi = __shfl_sync(0xFFFFFFFFu, w, i);
        if ((good_a >> i) & 1u) ua = __fadd_rn(ua, wi);
        if ((good_b >> i) & 1u) ub = __fadd_rn(ub, wi);
      }
      ua = upper_exits<R>(M, p0, p1, ua);
      ub = upper_exits<R>(M, p0, p1, ub);
    }
    if constexpr (R == 1)
      M.rollout_one2(p0, good_a, good_b, cand, depth + 1, va, vb, steps);
    else
      M.rollout_two2(p0, p1, good_a, good_b, cand, depth + 1, va, vb, steps);
  }
  const long long fu = warp_sum64(to_fixed(ua) + to_fixed(ub));
  const long long fl = warp_sum64(to_fixed(va) + to_fixed(vb));
  if (lane == 0) {
    sum_add(usum + slot, fu);
    sum_add(lsum + slot, fl);
  }
}
__host__ __device__ constexpr size_t rs_key_bytes_aligned(size_t key_bytes) { return (key_bytes + 15) & ~(size_t)15; }

// 42 registers (three 512-thread CTAs per SM) hold a unit's two items
// without spills (one robot: 0.557 against 0.567 ms per 15x15 expansion at
// 32).
template <int R>
__global__ void __launch_bounds__(512, 3) rs_rollout_items_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                              const dsp_leaf_job* __restrict__ jobs,
                                                              Items<R> items, unsigned int* chunk_head,
                                                              uint32_t plan_step) {
  __shared__ RSShared c;
  extern __shared__ __align__(16) uint16_t rs_keys[];
  load_rs_consts(c, gm);
  load_rs_keys(rs_keys, gm);
  __syncthreads();
  RSModel<R> M = make_rs<R>(gm, &c, plan_step);
  M.nkey = rs_keys;
  constexpr int F = Items<R>::kCompactFields;
  const int lane = threadIdx.x & 31;
  // each warp's two stages of one unit (rs_stage_bytes per CTA)
  uint32_t* stage = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(rs_keys) +
                                                rs_key_bytes_aligned(sizeof(uint16_t) * (size_t)gm->m * gm->n * gm->n)) +
                    (size_t)(threadIdx.x >> 5) * 2 * kUnitChunks * F * 32;
  // chunks of 32 items (fewer than 2^26: the list holds fewer than 2^31)
  const unsigned int nchunks = (unsigned int)((items.total + 31) >> 5);
  unsigned long long steps = 0;
  __shared__ ChunkClaims claims[kMaxWarpsB];
  ChunkClaims& cc = claims[threadIdx.x >> 5];
  if (lane == 0) cc.left = 0;
  if constexpr (R == 2) {
    // Two robots: rollouts are long, so reading a chunk's items straight
    // from global memory costs less than staging them (4.40 against
    // 4.68 ms per 512-job launch of 15x15).
    // Units of two chunks as for one robot: a unit that is one child's walks
    // one joint trajectory for both of each lane's items.
    const unsigned int nunits2 = (nchunks + kUnitChunks - 1) / kUnitChunks;
    while (true) {
      unsigned int un = 0;
      if (lane == 0) un = cc.take(chunk_head);
      un = __shfl_sync(0xFFFFFFFFu, un, 0);
      if (un >= nunits2) break;
      const long long ia = (long long)un * (32 * kUnitChunks) + lane;
      const bool oka = ia < items.total, okb = ia + 32 < items.total;
      RSS sa, sb;
      uint32_t cand_a = 0, meta_a = 0, job_a = 0, cand_b = 0, meta_b = 0, job_b = 0;
      if (oka) items.get_compact((size_t)ia, sa, cand_a, meta_a, job_a);
      if (okb) items.get_compact((size_t)(ia + 32), sb, cand_b, meta_b, job_b);
      const uint32_t q0 = __shfl_sync(0xFFFFFFFFu, sa.pos[0], 0), q1 = __shfl_sync(0xFFFFFFFFu, sa.pos[1], 0);
      const uint32_t c0 = __shfl_sync(0xFFFFFFFFu, cand_a, 0), m0 = __shfl_sync(0xFFFFFFFFu, meta_a, 0);
      const uint32_t j0 = __shfl_sync(0xFFFFFFFFu, job_a, 0);
      const bool one = __all_sync(0xFFFFFFFFu, oka && okb && sa.pos[0] == q0 && sb.pos[0] == q0 && sa.pos[1] == q1 &&
                                                   sb.pos[1] == q1 && cand_a == c0 && cand_b == c0 && meta_a == m0 &&
                                                   meta_b == m0 && job_a == j0 && job_b == j0);
      if (one) {
        rs_rollout_pair<R>(M, jobs, q0, q1, sa.good, sb.good, c0, m0, j0, steps);
        continue;
      }
      rs_rollout_values<R>(M, jobs, oka, sa, cand_a, meta_a, job_a, steps);
      if (__any_sync(0xFFFFFFFFu, okb)) rs_rollout_values<R>(M, jobs, okb, sb, cand_b, meta_b, job_b, steps);
    }
    for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
    if (lane == 0 && steps) atomicAdd(&work->steps, steps);
    return;
  }
  // One robot: units of two chunks (64 items), claimed ChunkClaims::kBatch
  // at a time, and one step ahead of their staging: the claim for the unit
  // after next is made before a unit's rollouts and read after them. A unit
  // whose 64 items are one child's shares one trajectory (rs_rollout_pair);
  // any other takes its two chunks one after the other.
  const unsigned int nunits = (nchunks + kUnitChunks - 1) / kUnitChunks;
  auto claim = [&]() {
    unsigned int ch = 0;
    if (lane == 0) ch = cc.take(chunk_head);
    return __shfl_sync(0xFFFFFFFFu, ch, 0);
  };
  constexpr int kUnitWords = kUnitChunks * F * 32;
  unsigned int cur = claim();
  if (cur < nunits) stage_unit<R>(stage, items, cur);
  unsigned int nxt = cur < nunits ? claim() : nunits;
  if (nxt < nunits) stage_unit<R>(stage + kUnitWords, items, nxt);
  unsigned int pending = 0;  // lane 0: the claim in flight
  if (nxt < nunits && lane == 0) pending = cc.take(chunk_head);
  int b = 0;
  while (cur < nunits) {
    if (nxt < nunits)
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    const uint32_t* w = stage + b * kUnitWords;
    const long long ia = (long long)cur * (32 * kUnitChunks) + lane;
    const bool oka = ia < items.total, okb = ia + 32 < items.total;
    const uint32_t pos_a = w[lane], good_a = w[32 + lane], cand_a = w[64 + lane], meta_a = w[96 + lane],
                   job_a = w[128 + lane];
    const uint32_t pos_b = w[F * 32 + lane], good_b = w[F * 32 + 32 + lane], cand_b = w[F * 32 + 64 + lane],
                   meta_b = w[F * 32 + 96 + lane], job_b = w[F * 32 + 128 + lane];
    __syncwarp();  // the buffer is read: the unit after next may go there
    cur = nxt;
    b ^= 1;
    if (cur < nunits) {
      // cur < nunits: the claim issued one unit ago names the unit to stage now
      nxt = __shfl_sync(0xFFFFFFFFu, pending, 0);
      if (nxt < nunits) {
        stage_unit<R>(stage + (b ^ 1) * kUnitWords, items, nxt);
        if (lane == 0) pending = cc.take(chunk_head);
      }
    }
    // one child for all 64 items (lane 0 always holds an item)
    const uint32_t p0 = __shfl_sync(0xFFFFFFFFu, pos_a, 0), c0 = __shfl_sync(0xFFFFFFFFu, cand_a, 0);
    const uint32_t m0 = __shfl_sync(0xFFFFFFFFu, meta_a, 0), j0 = __shfl_sync(0xFFFFFFFFu, job_a, 0);
    const bool one = __all_sync(0xFFFFFFFFu, oka && okb && pos_a == p0 && pos_b == p0 && cand_a == c0 &&
                                                 cand_b == c0 && meta_a == m0 && meta_b == m0 && job_a == j0 &&
                                                 job_b == j0);
    if constexpr (R == 1) {
      if (one) {
        rs_rollout_pair<1>(M, jobs, p0, 0u, good_a, good_b, c0, m0, j0, steps);
        continue;
      }
    }
    RSS s;
    s.pos[0] = pos_a;
    s.pos[1] = 0u;
    s.good = good_a;
    s.sampled = 0u;
    s.scen = 0u;
    rs_rollout_values<R>(M, jobs, oka, s, cand_a, meta_a, job_a, steps);
    if (__any_sync(0xFFFFFFFFu, okb)) {
      s.pos[0] = pos_b;
      s.good = good_b;
      rs_rollout_values<R>(M, jobs, okb, s, cand_b, meta_b, job_b, steps);
    }
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if (lane == 0 && steps) atomicAdd(&work->steps, steps);
}

// Phase B over slices (heuristic default policy): a warp takes one slice at
// a time (claims in batches as for chunks), lane l its items l, l + 32,
// l + 64 and l + 96. A slice is one child's: the same
// slot and job, and in a job whose scenarios share the robots' cells (a tree
// node's) the same positions and candidate set, which the slice then
// carries (its items hold only their good masks). Then one trajectory
// (rollout_oneK, or rollout_twoK's joint one) gives all of a lane's values,
// u0's per-rock terms come from lane i as in rs_rollout_values, and the
// child's sums take one warp sum each. A slice whose items differ in
// position or candidate set takes rs_rollout_values 32 items at a time. 64
// registers (two 512-thread CTAs per SM) hold a lane's items.
template <int R>
constexpr int kSliceLen = R == 1 ? kSliceItems : kSliceItemsTwo;
template <int R>
__global__ void __launch_bounds__(512, 2) rs_rollout_slices_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                   const dsp_leaf_job* __restrict__ jobs,
                                                                   Items<R> items, Slices sl,
                                                                   unsigned int* slice_head, uint32_t plan_step) {
  constexpr int kSliceLanes = kSliceLen<R> / 32;
  constexpr int kGood = R == 2 ? 2 : 1;  // the good field of a compact item
  __shared__ RSShared c;
  extern __shared__ __align__(16) uint16_t rs_keys[];
  load_rs_consts(c, gm);
  load_rs_keys(rs_keys, gm);
  __syncthreads();
  RSModel<R> M = make_rs<R>(gm, &c, plan_step);
  M.nkey = rs_keys;
  const int lane = threadIdx.x & 31;
  const unsigned int ns = min(*sl.count, sl.cap);
  unsigned long long steps = 0;
  __shared__ ChunkClaims claims[kMaxWarpsB];
  ChunkClaims& cc = claims[threadIdx.x >> 5];
  if (lane == 0) cc.left = 0;
  while (true) {
    unsigned int si = 0;
    if (lane == 0) si = cc.take(slice_head);
    si = __shfl_sync(0xFFFFFFFFu, si, 0);
    if (si >= ns) break;
    const uint4 d0 = sl.list[2 * si], d1 = sl.list[2 * si + 1];
    const long long st = (long long)d0.x;
    const int cnt = (int)(d0.y & 0xFFFFu);
    const bool shared = (d0.y & kSliceShared) != 0u;
    // (a slice list that overflowed its capacity has flagged the status word;
    // no entry outside the item list is read)
    if (cnt < 1 || cnt > kSliceLen<R> || st + cnt > items.total) continue;
    bool ok[kSliceLanes];
    uint32_t pos[kSliceLanes], pos1[kSliceLanes], good[kSliceLanes], cand[kSliceLanes], meta[kSliceLanes],
        job[kSliceLanes];
    uint32_t p0 = d0.z, q1 = d1.z, c0 = d0.w, m0 = d1.x, j0 = d1.y;
    if (shared) {
      // the child's state is the slice's; the items hold their good masks
#pragma unroll
      for (int k = 0; k < kSliceLanes; ++k) {
        ok[k] = lane + 32 * k < cnt;
        good[k] = ok[k] ? items.f(kGood)[st + lane + 32 * k] : 0u;
        pos[k] = p0;
        pos1[k] = q1;
        cand[k] = c0;
        meta[k] = m0;
        job[k] = j0;
      }
    } else {
#pragma unroll
      for (int k = 0; k < kSliceLanes; ++k) {
        ok[k] = lane + 32 * k < cnt;
        RSS s;
        s.pos[0] = s.pos[1] = 0u;
        s.good = 0u;
        cand[k] = meta[k] = job[k] = 0u;
        if (ok[k]) items.get_compact((size_t)(st + lane + 32 * k), s, cand[k], meta[k], job[k]);
        pos[k] = s.pos[0];
        pos1[k] = s.pos[1];
        good[k] = s.good;
      }
      p0 = __shfl_sync(0xFFFFFFFFu, pos[0], 0);
      q1 = __shfl_sync(0xFFFFFFFFu, pos1[0], 0);
      c0 = __shfl_sync(0xFFFFFFFFu, cand[0], 0);
      m0 = __shfl_sync(0xFFFFFFFFu, meta[0], 0);
      j0 = __shfl_sync(0xFFFFFFFFu, job[0], 0);
    }
    bool same = true;
#pragma unroll
    for (int k = 0; k < kSliceLanes; ++k)
      same = same && (!ok[k] || (pos[k] == p0 && pos1[k] == q1 && cand[k] == c0 && meta[k] == m0 && job[k] == j0));
    if (shared || __all_sync(0xFFFFFFFFu, same)) {
      int64_t* usum = jobs[j0].u_sum;
      int64_t* lsum = jobs[j0].l_sum;
      const uint32_t slot = m0 & 0xFFFFFFu;
      const int depth = (int)(m0 >> 24);
      float u[kSliceLanes], v[kSliceLanes];
#pragma unroll
      for (int k = 0; k < kSliceLanes; ++k) u[k] = v[k] = 0.0f;
      if (!rs_terminal<R>(p0, q1)) {
        if (depth + 1 >= M.D) {
          RSS s;
          s.pos[0] = p0;
          s.pos[1] = q1;
          const float tl = M.tail(s);
#pragma unroll
          for (int k = 0; k < kSliceLanes; ++k) u[k] = tl;
        } else {
          const float w = upper_term<R>(M, p0, q1, lane);
          for (int i = 0; i < M.m; ++i) {
            const float wi = __shfl_sync(0xFFFFFFFFu, w, i);
#pragma unroll
            for (int k = 0; k < kSliceLanes; ++k)
              if ((good[k] >> i) & 1u) u[k] = __fadd_rn(u[k], wi);
          }
#pragma unroll
          for (int k = 0; k < kSliceLanes; ++k) u[k] = upper_exits<R>(M, p0, q1, u[k]);
        }
        int live = 0;
#pragma unroll
        for (int k = 0; k < kSliceLanes; ++k) live += ok[k] ? 1 : 0;
        if constexpr (R == 1)
          M.template rollout_oneK<kSliceLanes>(p0, good, c0, depth + 1, v, (unsigned long long)live, steps);
        else
          M.template rollout_twoK<kSliceLanes>(p0, q1, good, c0, depth + 1, v, (unsigned long long)live, steps);
      }
      long long fu = 0, fl = 0;
#pragma unroll
      for (int k = 0; k < kSliceLanes; ++k)
        if (ok[k]) {
          fu += to_fixed(u[k]);
          fl += to_fixed(v[k]);
        }
      fu = warp_sum64(fu);
      fl = warp_sum64(fl);
      if (lane == 0) {
        sum_add(usum + slot, fu);
        sum_add(lsum + slot, fl);
      }
      continue;
    }
#pragma unroll
    for (int k = 0; k < kSliceLanes; ++k) {
      if (32 * k >= cnt) break;
      RSS s;
      s.pos[0] = pos[k];
      s.pos[1] = pos1[k];
      s.good = good[k];
      s.sampled = 0u;
      s.scen = 0u;
      rs_rollout_values<R>(M, jobs, ok[k], s, cand[k], meta[k], job[k], steps);
    }
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if (lane == 0 && steps) atomicAdd(&work->steps, steps);
}

// Phase B in block form for one chunk u (one robot, heuristic default
// policy): the 32 grouped positions [32 b, 32 b + 32) of action a of job j =
// chunk_job[u], where u - unit_base[j] = a * ceil(n / 32) + b. Each lane
// rebuilds the item phase A would have written for its grouped position q:
// the scenario p = perm[a][q] and its leaf state; the child whose offset
// range holds q, and that child's observation z; the child's
// positive-counter mask (the leaf's, with a Sense reading's +-1 on its
// rock's counter); and the state after a move or Sample (a Sense leaves it as
// it was). Then u0, the rollout and the sums as for a stored item.
__device__ __forceinline__ void rs_block_values(const RSModel<1>& M, const dsp_leaf_job* __restrict__ jobs,
                                                const LeafBlocks& lb, unsigned int u, int j,
                                                unsigned long long& steps) {
  const int lane = threadIdx.x & 31;
  const dsp_leaf_job* J = jobs + j;
  const int n = J->n_scen, cap = J->child_cap, depth = J->depth;
  const int nb = (n + 31) >> 5;
  const int local = (int)((long long)u - lb.unit_base[j]);
  const int a = local / nb;
  const int q = (local - a * nb) * 32 + lane;
  const int aa = J->first_action + a;
  const bool ok = q < n;
  // the child of grouped position q: the last whose offset is <= q (at most
  // six children, in lanes 0..nc-1)
  const int nc = min(J->child_count[a], cap);
  const int myoff = lane < nc ? J->child_off[(size_t)a * (cap + 1) + lane] : 0;
  const uint32_t myz = lane < nc ? (uint32_t)(J->child_key[(size_t)a * cap + lane] & 3u) : 0u;
  int ci = 0;
  for (int k = 1; k < nc; ++k) ci += q >= __shfl_sync(0xFFFFFFFFu, myoff, k) ? 1 : 0;
  const int z = (int)__shfl_sync(0xFFFFFFFFu, myz, ci);
  // the leaf's positive-counter mask, rock i's counter in lane i
  const int hv = lane < M.m ? (int)J->hist[lane] : 0;
  uint32_t pm = __ballot_sync(0xFFFFFFFFu, hv > 0);
  if (aa >= 5) {  // Sense rock i: a good reading adds one, a bad one takes one (clamped to +-127)
    const int i = aa - 5;
    const int c0 = __shfl_sync(0xFFFFFFFFu, hv, i);
    const int c = z == 1 ? min(c0 + 1, 127) : (z == 2 ? max(c0 - 1, -127) : c0);
    pm = c > 0 ? (pm | (1u << i)) : (pm & ~(1u << i));
  }
  RSS s;
  s.pos[0] = 0u;
  s.pos[1] = 0u;
  s.good = 0u;
  s.sampled = 0u;
  s.scen = 0u;
  if (ok) {
    const int p = J->perm[(size_t)a * n + q];
    const uint32_t* L = lb.leaf + 3 * lb.scen_base[j];
    s.pos[0] = L[p];
    s.good = L[n + p];
    s.sampled = L[2 * n + p];
    if (aa < 5) {
      uint64_t k;
      M.step(s, aa, depth, k);
    }
  }
  const uint32_t cand = pm & ~s.sampled;
  s.sampled = 0u;
  const uint32_t meta = ((uint32_t)depth << 24) | (uint32_t)(a * cap + min(ci, cap - 1));
  rs_rollout_values<1>(M, jobs, ok, s, cand, meta, (uint32_t)j, steps);
}

// Phase B in block form: warps claim chunks as rs_rollout_items_kernel does
// and read each chunk's job one chunk ahead.
__global__ void __launch_bounds__(512, 3) rs_rollout_blocks_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                   const dsp_leaf_job* __restrict__ jobs,
                                                                   int n_jobs, LeafBlocks lb, unsigned int nchunks,
                                                                   unsigned int* chunk_head, uint32_t plan_step) {
  __shared__ RSShared c;
  extern __shared__ __align__(16) uint16_t rs_keys[];
  load_rs_consts(c, gm);
  load_rs_keys(rs_keys, gm);
  __syncthreads();
  RSModel<1> M = make_rs<1>(gm, &c, plan_step);
  M.nkey = rs_keys;
  const int lane = threadIdx.x & 31;
  unsigned long long steps = 0;
  __shared__ ChunkClaims claims[kMaxWarpsB];
  ChunkClaims& cc = claims[threadIdx.x >> 5];
  if (lane == 0) cc.left = 0;
  unsigned int pending = 0;  // lane 0: the claim in flight
  if (lane == 0) pending = cc.take(chunk_head);
  unsigned int cur = __shfl_sync(0xFFFFFFFFu, pending, 0);
  int jcur = cur < nchunks ? lb.chunk_job[cur] : 0;
  if (lane == 0 && cur < nchunks) pending = cc.take(chunk_head);
  while (cur < nchunks) {
    // the claim made one chunk ago; its job is loaded now and read next time
    const unsigned int nxt = __shfl_sync(0xFFFFFFFFu, pending, 0);
    int jnxt = 0;
    if (nxt < nchunks) {
      jnxt = lb.chunk_job[nxt];
      if (lane == 0) pending = cc.take(chunk_head);
    }
    if ((unsigned)jcur < (unsigned)n_jobs)  // the grouping phase wrote every block's job
      rs_block_values(M, jobs, lb, cur, jcur, steps);
    else if (lane == 0)
      report(work, kStatusBadJob);
    cur = nxt;
    jcur = jnxt;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if (lane == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_step: one g call per scenario.
template <int R>
__global__ void rs_step_kernel(const DevModel* __restrict__ gm, const uint32_t* in, int in_cap, int count,
                               const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                               float* rewards, uint32_t plan_step) {
  __shared__ RSShared c;
  load_rs_consts(c, gm);
  __syncthreads();
  const RSModel<R> M = make_rs<R>(gm, &c, plan_step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    RSS s = M.load(in, in_cap, i);
    uint64_t key;
    float r = 0.0f;
    if (M.terminal(s))
      key = kTermBit;
    else
      r = M.step(s, actions[i], depth, key);
    M.store(s, out, out_cap, i);
    keys[i] = key;
    rewards[i] = r;
  }
}

// dsp_rollout: Eq. lb per scenario.
template <int R>
__global__ void rs_rollout_kernel(const DevModel* __restrict__ gm, DevWork* work, const uint32_t* block, int cap,
                                  int count, const int8_t* hist, int start_depth, float* value,
                                  uint32_t plan_step) {
  __shared__ RSShared c;
  load_rs_consts(c, gm);
  __syncthreads();
  const RSModel<R> M = make_rs<R>(gm, &c, plan_step);
  unsigned long long steps = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    RSS s = M.load(block, cap, i);
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      h[k] = hist ? *reinterpret_cast<const uint32_t*>(hist + 32 * (size_t)i + 4 * k) : 0u;
    value[i] = M.rollout(s, positive_mask(h, M.m), start_depth, steps);
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// CTAs per SM of a kernel at a CTA size and dynamic shared memory, asked of
// the runtime once per (kernel, size, memory, device) and kept: the answer
// never changes, and the query costs host time on every launch otherwise.
template <class K>
int occupancy_cached(K kernel, int block, size_t smem) {
  struct Entry {
    const void* k;
    int block, dev;
    size_t smem;
    int per_sm;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const void* key = reinterpret_cast<const void*>(kernel);
  {
    std::lock_guard<std::mutex> lock(mu);
    for (const Entry& e : cache)
      if (e.k == key && e.block == block && e.smem == smem && e.dev == dev) return e.per_sm;
  }
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem);
  std::lock_guard<std::mutex> lock(mu);
  cache.push_back({key, block, dev, smem, n});
  return n;
}

template <int R>
cudaError_t launch_two_phase(const DevModel* gm, int num_actions, int key_words, DevWork* work, const dsp_leaf_job* jobs,
                             const long long* item_base, const int* order, int n_jobs, long long total_items, uint32_t* item_buf, unsigned int* counters,
                             uint32_t plan_step, int num_sms, int block_b, const void* policy, cudaStream_t st,
                             int warps_a, int ctas_b, LeafBlocks lb, Slices sl, bool large_jobs) {
  // block form (lb.leaf set; one robot, heuristic policy): no item list,
  // total_items counts the 32-position blocks
  const bool blocks = lb.leaf != nullptr;
  Items<R> items{blocks ? nullptr : item_buf, blocks ? 0 : total_items, policy != nullptr && R == 1};
  // slices: one robot's heuristic rollouts over the item list; phase A counts
  // them in counters[2]
  if (blocks || policy != nullptr) sl = Slices{};
  if (sl.list != nullptr) sl.count = counters + 2;
  // Each warp expands whole actions: as many warps as give every warp the
  // same number of a job's actions (20 actions: 10 warps of 2; 400: 16 of
  // 25). One robot with at least two jobs per CTA slot: at most five warps
  // (20 actions: 5 of 4), so that six CTAs fit per SM and a CTA waiting at a
  // job's barriers leaves others running (4096 jobs of 15x15: 0.280 against
  // 0.295 ms). With fewer jobs the wider CTA finishes the largest job sooner
  // (512 jobs: 55 against 72 us).
  // warps_a (the launch shape's grouping-phase warps, 1..16) replaces the rule.
  int block_a = kBlockA;
  if (warps_a > 0) {
    block_a = 32 * std::min(warps_a, kWarpsA);
  } else {
    const int na = std::max(1, num_actions);
    const bool narrow = R == 1 && n_jobs >= 12 * num_sms;
    const int per_warp = narrow ? (na + 4) / 5 : (na + kWarpsA - 1) / kWarpsA;
    block_a = 32 * ((na + per_warp - 1) / per_warp);
  }
  // (two robots have no large-job path)
  constexpr bool kMayBeLarge = R == 1;
  const bool large = kMayBeLarge && large_jobs;
  int per_sm_a = large ? occupancy_cached(rs_group_kernel<R, kMayBeLarge>, block_a, 0)
                       : occupancy_cached(rs_group_kernel<R, false>, block_a, 0);
  int grid_a = std::max(1, std::min(n_jobs, std::max(1, per_sm_a) * num_sms));
  // two robots: a job's hundreds of actions split over several CTAs (runs of
  // about 80), so that the largest jobs do not leave a tail
  const int splits = R == 2 ? std::max(1, num_actions / 80) : 1;
  grid_a = std::max(1, std::min(n_jobs * splits, std::max(1, per_sm_a) * num_sms));
  if (large)
    rs_group_kernel<R, kMayBeLarge><<<grid_a, block_a, 0, st>>>(gm, work, jobs, blocks ? nullptr : item_base, order,
                                                                n_jobs, counters, plan_step, items, splits, lb, sl);
  else
    rs_group_kernel<R, false><<<grid_a, block_a, 0, st>>>(gm, work, jobs, blocks ? nullptr : item_base, order,
                                                          n_jobs, counters, plan_step, items, splits, lb, sl);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (policy != nullptr && R == 1)
    return launch_rs_rollout_mlp_items(gm, work, jobs, item_buf, total_items, counters + 1, policy, plan_step,
                                       num_sms, st);
  if constexpr (R == 1) {
    if (blocks) {
      const size_t kb = rs_key_bytes_aligned(sizeof(uint16_t) * (size_t)key_words);
      int per_sm = occupancy_cached(rs_rollout_blocks_kernel, block_b, kb);
      if (ctas_b > 0) per_sm = std::min(per_sm, ctas_b);
      const long long want = (total_items + block_b / 32 - 1) / (block_b / 32);
      const int grid = (int)std::max(1LL, std::min<long long>(want, (long long)std::max(1, per_sm) * num_sms));
      rs_rollout_blocks_kernel<<<grid, block_b, kb, st>>>(gm, work, jobs, n_jobs, lb, (unsigned int)total_items,
                                                           counters + 1, plan_step);
      return cudaGetLastError();
    }
  }
  if (sl.list != nullptr) {
    const size_t kb = rs_key_bytes_aligned(sizeof(uint16_t) * (size_t)key_words);
    int per_sm = occupancy_cached(rs_rollout_slices_kernel<R>, block_b, kb);
    if (ctas_b > 0) per_sm = std::min(per_sm, ctas_b);
    const long long want = ((long long)sl.cap + block_b / 32 - 1) / (block_b / 32);
    const int grid = (int)std::max(1LL, std::min<long long>(want, (long long)std::max(1, per_sm) * num_sms));
    rs_rollout_slices_kernel<R><<<grid, block_b, kb, st>>>(gm, work, jobs, items, sl, counters + 1, plan_step);
    return cudaGetLastError();
  }
  // phase B keeps the policy-key table in shared memory (limit set by rs_set_key_smem)
  const size_t key_bytes =
      rs_key_bytes_aligned(sizeof(uint16_t) * (size_t)key_words) + (R == 1 ? rs_stage_bytes<R>(block_b) : 0);
  int per_sm_b = occupancy_cached(rs_rollout_items_kernel<R>, block_b, key_bytes);
  if (ctas_b > 0) per_sm_b = std::min(per_sm_b, ctas_b);
  long long chunks = (total_items + 31) / 32;
  long long want = (chunks + block_b / 32 - 1) / (block_b / 32);
  int grid_b = (int)std::max(1LL, std::min<long long>(want, (long long)std::max(1, per_sm_b) * num_sms));
  rs_rollout_items_kernel<R><<<grid_b, block_b, key_bytes, st>>>(gm, work, jobs, items, counters + 1, plan_step);
  return cudaGetLastError();
}

// ------------------------------------------------------------ job queue ---
// Persistent expansion fed by host threads through a ring in mapped pinned
// host memory. Ticket t lives in slot t % cap:
//  - seq = t + 1 once its job is published, seq = t + cap once the slot may
//    take ticket t + cap;
//  - done = t + 1 once its results are written.
// A CTA claims the next ticket only after its job is published, so no ticket
// is ever held without a job.
//
// Work is shared across the whole grid:
//  - The CTA that claims a job runs phase A into the slot's item list and
//    publishes the job's rollout chunks in the slot's claim word: the ticket's
//    low 32 bits, and the next chunk.
//  - Any warp of any CTA takes chunks of any published job by compare-and-swap
//    on that word, which succeeds only while the job it read is still the
//    slot's.
//  - The warp that finishes a job's last chunk closes the word (chunk field
//    all ones), writes done and frees the slot.
// No CTA waits on another. A CTA that finds neither a job nor a chunk for
// idle_ns (or finds the ring closed) exits, and the host relaunches the
// kernel when more jobs arrive.

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Claim word of a ring slot: the ticket's low 16 bits << 48 | the job's chunk
// count << 24 | the next chunk (count 0: closed). Warps claim chunks with
// atomicAdd, which always succeeds, so claims never retry on a busy word: the
// returned word names the slot's current job (its data were written before it
// was published) and whether chunks were left. A warp adds only after reading
// that chunks remain, so the next-chunk field passes the count by at most the
// number of warps times the grain and never reaches the count's bits.
__device__ __forceinline__ unsigned long long claim_word(unsigned long long ticket, unsigned int nchunks) {
  return ((ticket & 0xFFFFull) << 48) | ((unsigned long long)nchunks << 24);
}
__device__ __forceinline__ unsigned int claim_next(unsigned long long w) { return (unsigned int)(w & 0xFFFFFFu); }
__device__ __forceinline__ unsigned int claim_count(unsigned long long w) {
  return (unsigned int)((w >> 24) & 0xFFFFFFu);
}

// The job in `slot` is finished: close its claim word, publish done, free the slot.
__device__ __forceinline__ void queue_complete(const QueueRing& ring, int slot, unsigned long long ticket) {
  atomicExch(&ring.share[slot].claim, claim_word(ticket, 0u));
  atomicAdd(ring.finished, 1ull);
  __threadfence_system();
  st_release_sys(ring.done + slot, ticket + 1);
  st_release_sys(ring.seq + slot, ticket + (unsigned long long)ring.cap);
}

// One warp looks for rollout chunks of any published job and claims up to the
// job's grain of them (consecutive). Returns the slot (or -1), the first chunk
// and the count, the same in every lane.
__device__ __forceinline__ int queue_claim_chunk(const QueueRing& ring, unsigned int& chunk, unsigned int& count) {
  const int lane = threadIdx.x & 31;
  const int start = (int)((blockIdx.x * 7 + (threadIdx.x >> 5)) % (unsigned)ring.cap);
  for (int base = 0; base < ring.cap; base += 32) {
    for (int attempt = 0; attempt < 4; ++attempt) {
      const int s = (start + base + lane) % ring.cap;
      bool can = false;
      if (base + lane < ring.cap) {
        const unsigned long long c = ld_acquire_gpu(&ring.share[s].claim);
        can = claim_next(c) < claim_count(c);
      }
      const unsigned int ready = __ballot_sync(0xFFFFFFFFu, can);
      if (ready == 0u) break;
      // lanes with a claimable slot spread the warp over them
      const int pick = __fns(ready, 0, 1 + (int)(((blockIdx.x >> 1) + (threadIdx.x >> 5)) % __popc(ready)));
      const int leader = pick >= 0 ? pick : __ffs(ready) - 1;
      unsigned int got = 0, first = 0;
      if (lane == leader) {
        const unsigned int g = max(1u, *(volatile unsigned int*)&ring.share[s].grain);
        const unsigned long long old = atomicAdd(&ring.share[s].claim, (unsigned long long)g);
        first = claim_next(old);
        const unsigned int n = claim_count(old);
        got = first < n ? min(g, n - first) : 0u;
        if (got) __threadfence();  // the job's data, published before its claim word
      }
      __syncwarp();
      got = __shfl_sync(0xFFFFFFFFu, got, leader);
      if (got) {
        count = got;
        chunk = __shfl_sync(0xFFFFFFFFu, first, leader);
        return __shfl_sync(0xFFFFFFFFu, s, leader);
      }
    }
  }
  return -1;
}

template <int R>
__global__ void __launch_bounds__(kBlockA, 2) rs_queue_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                             QueueRing ring, unsigned long long* head,
                                                             uint32_t* scratch, size_t slot_words,
                                                             dsp_leaf_job* jcopy, unsigned long long idle_ns) {
  __shared__ RSGroupSmem S;
  __shared__ long long s_ticket;
  __shared__ unsigned int s_plan_step;
  __shared__ int s_work, s_exit;
  extern __shared__ uint16_t rs_keys[];
  load_rs_consts(S.c, gm);
  load_rs_keys(rs_keys, gm);
  RSModel<R> M = make_rs<R>(gm, &S.c, 0u);  // each job carries its own plan step
  M.nkey = rs_keys;
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned long long steps = 0, last_work = global_ns();
  unsigned int backoff = 256;  // idle sleep, doubled while nothing comes (ns)
  __syncthreads();
  while (true) {
    // a new job from the ring, if one is published (no waiting); warp 0 reads
    // the descriptor from host memory with all lanes at once
    if (tid < 32) {
      long long ticket = -1;
      if (lane == 0) {
        const unsigned long long h = *(volatile unsigned long long*)head;
        if (ld_acquire_sys(ring.seq + (h % ring.cap)) == h + 1 && atomicCAS(head, h, h + 1) == h)
          ticket = (long long)h;
      }
      __syncwarp();
      ticket = __shfl_sync(0xFFFFFFFFu, ticket, 0);
      if (ticket >= 0) {
        constexpr int kWords = (int)(sizeof(dsp_leaf_job) / 4);
        const int slot = (int)(ticket % ring.cap);
        const volatile uint32_t* src = (const volatile uint32_t*)(ring.jobs + slot);
        uint32_t* dst = (uint32_t*)&S.J;
        uint32_t* dcopy = (uint32_t*)(jcopy + slot);
        for (int w = lane; w < kWords; w += 32) {
          const uint32_t x = src[w];
          dst[w] = x;
          dcopy[w] = x;
        }
        if (lane == 0) s_plan_step = *(volatile unsigned int*)(ring.plan_step + slot);
      }
      if (lane == 0) {
        s_ticket = ticket;
        s_work = 0;
      }
    }
    __syncthreads();
    const long long ticket = s_ticket;
    if (ticket >= 0) {
      const int slot = (int)(ticket % ring.cap);
      const int n = S.J.n_scen;
      long long nchunks = 0;
      M.plan_step = s_plan_step;
      if (n > 0) {  // a job with no scenarios is a placeholder: nothing to do
        Items<R> items{scratch + (size_t)slot * slot_words, (long long)n * S.J.n_actions, false};
        group_job<R, false>(S, M, 0, 0, 0, S.J.n_actions, true, items, work, steps);
        nchunks = (items.total + 31) >> 5;
      }
      __threadfence();  // every thread's phase-A results, before the job is published
      __syncthreads();
      if (tid == 0) {
        if (nchunks == 0) {
          queue_complete(ring, slot, (unsigned long long)ticket);
        } else {
          QueueShare& sh = ring.share[slot];
          sh.ticket = (unsigned long long)ticket;
          sh.nchunks = (unsigned int)nchunks;
          sh.remaining = (unsigned int)nchunks;
          // large jobs hand out several chunks per claim, so claims do not
          // queue up on the claim word; small ones one chunk at a time
          sh.grain = (unsigned int)max(1LL, min(16LL, nchunks / 256));
          sh.plan_step = s_plan_step;
          __threadfence();
          atomicExch(&sh.claim, claim_word((unsigned long long)ticket, (unsigned int)nchunks));
        }
      }
    }
    // rollout chunks of any published job, warp by warp, until none is left
    bool did = false;
    while (true) {
      unsigned int chunk = 0, count = 0;
      const int slot = queue_claim_chunk(ring, chunk, count);
      if (slot < 0) break;
      const dsp_leaf_job* J = jcopy + slot;
      Items<R> items{scratch + (size_t)slot * slot_words, (long long)J->n_scen * J->n_actions, false};
      M.plan_step = *(volatile unsigned int*)&ring.share[slot].plan_step;
      for (unsigned int k = 0; k < count; ++k) rs_rollout_chunk<R>(M, J, items, chunk + k, steps);
      __threadfence();  // every lane's sums, before the chunks count as done
      __syncwarp();
      if (lane == 0) {
        if (atomicSub(&ring.share[slot].remaining, count) == count)
          queue_complete(ring, slot, *(volatile unsigned long long*)&ring.share[slot].ticket);
      }
      did = true;
    }
    if (did && lane == 0) s_work = 1;
    __syncthreads();
    if (tid == 0) {
      const unsigned long long now = global_ns();
      const bool busy = ticket >= 0 || s_work != 0;
      if (busy) last_work = now;
      // a CTA stays while any claimed job is unfinished (its chunks may still
      // be published), up to a hard second of idling
      const bool drained =
          *(volatile unsigned long long*)ring.finished == *(volatile unsigned long long*)head;
      const unsigned long long idle = now - last_work;
      s_exit = !busy && (*(volatile unsigned int*)ring.close != 0u || idle > idle_ns) &&
               (drained || idle > 1000000000ull);
      if (busy) backoff = 256;
      if (!busy && !s_exit) {
        // idle CTAs back off, so their polling leaves the working CTAs'
        // issue slots and the shared claim words alone
        __nanosleep(backoff);
        backoff = min(backoff * 2u, 16384u);
      }
    }
    __syncthreads();
    if (s_exit) break;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if (lane == 0 && steps) atomicAdd(&work->steps, steps);
}

}  // namespace

int rs_item_fields(int robots, bool full) {
  if (full) return robots == 2 ? Items<2>::kFields : Items<1>::kFields;
  return robots == 2 ? Items<2>::kCompactFields : Items<1>::kCompactFields;
}

size_t rs_queue_slot_words(int robots, int num_actions) {
  return (size_t)rs_item_fields(robots, false) * (size_t)kMaxScen * (size_t)num_actions;
}

// The persistent kernel keeps the policy-key table in dynamic shared memory.
// The queue sets the kernel's shared-memory limit when it is created, before
// any capture (rs_queue_blocks_per_sm).
template <int R>
static cudaError_t rs_queue_smem(int key_words, size_t& bytes) {
  bytes = sizeof(uint16_t) * (size_t)key_words;
  if (bytes + sizeof(RSGroupSmem) > 48 * 1024)
    return cudaFuncSetAttribute(rs_queue_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

int rs_queue_blocks_per_sm(int robots, int key_words) {
  int n = 0;
  size_t bytes = 0;
  if (robots == 1) {
    if (rs_queue_smem<1>(key_words, bytes) == cudaSuccess)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rs_queue_kernel<1>, kBlockA, bytes);
  } else {
    if (rs_queue_smem<2>(key_words, bytes) == cudaSuccess)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rs_queue_kernel<2>, kBlockA, bytes);
  }
  return n > 0 ? n : 1;
}

cudaError_t launch_rs_queue(const DevModel* gm, int robots, int key_words, DevWork* work, QueueRing ring,
                            unsigned long long* head, uint32_t* scratch, size_t slot_words, dsp_leaf_job* jcopy,
                            unsigned long long idle_ns, int grid, cudaStream_t st) {
  const size_t bytes = sizeof(uint16_t) * (size_t)key_words;
  if (robots == 1)
    rs_queue_kernel<1><<<grid, kBlockA, bytes, st>>>(gm, work, ring, head, scratch, slot_words, jcopy, idle_ns);
  else
    rs_queue_kernel<2><<<grid, kBlockA, bytes, st>>>(gm, work, ring, head, scratch, slot_words, jcopy, idle_ns);
  return cudaGetLastError();
}

cudaError_t rs_set_key_smem(int robots, int key_words) {
  // the key table and the item staging of the largest CTA (512 threads)
  const size_t keys = rs_key_bytes_aligned(sizeof(uint16_t) * (size_t)key_words);
  if (robots == 1) {
    cudaError_t e = cudaFuncSetAttribute(rs_rollout_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)keys);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rs_rollout_slices_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)keys);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(rs_rollout_items_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(keys + rs_stage_bytes<1>(512)));
  }
  cudaError_t e2 =
      cudaFuncSetAttribute(rs_rollout_slices_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)keys);
  if (e2 != cudaSuccess) return e2;
  return cudaFuncSetAttribute(rs_rollout_items_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)keys);
}

cudaError_t launch_rs_expand(const DevModel* gm, int robots, int num_actions, int key_words, DevWork* work,
                             const dsp_leaf_job* jobs, const long long* item_base, const int* order, int n_jobs,
                             long long total_items, uint32_t* item_buf, unsigned int* counters, uint32_t plan_step,
                             int num_sms, int block_b, const void* policy, cudaStream_t st, int warps_a, int ctas_b,
                             const LeafBlocks* blocks, const Slices* slices, bool large_jobs) {
  const LeafBlocks lb = (blocks != nullptr && robots == 1 && policy == nullptr) ? *blocks : LeafBlocks{};
  if (blocks != nullptr && lb.leaf == nullptr) return cudaErrorInvalidValue;  // block form: one robot, heuristic
  const Slices sl = slices != nullptr ? *slices : Slices{};
  if (robots == 1)
    return launch_two_phase<1>(gm, num_actions, key_words, work, jobs, item_base, order, n_jobs, total_items,
                               item_buf, counters, plan_step, num_sms, block_b, policy, st, warps_a, ctas_b, lb, sl,
                               large_jobs);
  return launch_two_phase<2>(gm, num_actions, key_words, work, jobs, item_base, order, n_jobs, total_items, item_buf,
                             counters, plan_step, num_sms, block_b, nullptr, st, warps_a, ctas_b, lb, sl, false);
}

cudaError_t launch_rs_step(const DevModel* gm, int robots, const uint32_t* in, int in_cap, int count,
                           const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                           float* rewards, uint32_t plan_step, cudaStream_t st) {
  int block = 256, grid = (count + block - 1) / block;
  if (grid > 4096) grid = 4096;
  if (robots == 1)
    rs_step_kernel<1><<<grid, block, 0, st>>>(gm, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                                              plan_step);
  else
    rs_step_kernel<2><<<grid, block, 0, st>>>(gm, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                                              plan_step);
  return cudaGetLastError();
}

cudaError_t launch_rs_rollout(const DevModel* gm, int robots, DevWork* work, const uint32_t* block, int cap,
                              int count, const int8_t* hist, int start_depth, float* value, uint32_t plan_step,
                              cudaStream_t st) {
  int b = 256, grid = (count + b - 1) / b;
  if (grid > 4096) grid = 4096;
  if (robots == 1)
    rs_rollout_kernel<1><<<grid, b, 0, st>>>(gm, work, block, cap, count, hist, start_depth, value, plan_step);
  else
    rs_rollout_kernel<2><<<grid, b, 0, st>>>(gm, work, block, cap, count, hist, start_depth, value, plan_step);
  return cudaGetLastError();
}

}  // namespace dsp

// ---------------------------------------------------------------------------
// Leaf expansion without device allocation (dsp_expand_leaves_noalloc).
//
// dsp_expand_leaves takes its job table, item offsets, counters and the
// rollout-item list from the model's memory pool on every call. Callers that cannot
// allocate device memory during planning use this variant instead: the same
// two kernels run on a fixed scratch array that the library keeps in device
// memory for the life of the process. Its size caps one call at
// kNoAllocJobs jobs and kNoAllocItems (action, scenario) items.
//
// The job table, the jobs' item offsets and their phase-A order reach the
// device in one copy from a static host array, page-locked once per process
// (cudaHostRegister pins the array; it allocates nothing), so a call does not
// wait for the work queued before it on its stream. The array is reused once
// the previous call's copy has run; a call made before then waits for that copy.
#include <cstring>
#include <mutex>

#include "model.hpp"

namespace dsp {
namespace {

constexpr int kNoAllocJobs = 8192;
constexpr long long kNoAllocItems = 1LL << 20;
constexpr size_t kNoAllocJobBytes = ((sizeof(dsp_leaf_job) * kNoAllocJobs + 255) / 256) * 256;
constexpr size_t kNoAllocBaseBytes = sizeof(long long) * kNoAllocJobs;
constexpr size_t kNoAllocOrderBytes = sizeof(int) * kNoAllocJobs;
constexpr size_t kNoAllocTableBytes = kNoAllocJobBytes + kNoAllocBaseBytes + kNoAllocOrderBytes;
constexpr size_t kNoAllocCounterBytes = 256;
constexpr size_t kNoAllocItemBytes = sizeof(uint32_t) * 8 * (size_t)kNoAllocItems;  // 8 = most item fields
constexpr size_t kNoAllocBytes = kNoAllocTableBytes + kNoAllocCounterBytes + kNoAllocItemBytes;
constexpr size_t kNoAllocHostBytes = (kNoAllocTableBytes + 4095) / 4096 * 4096;

// One copy per GPU that loads the library, held until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host side of the copies: laid out like the front of the device array.
alignas(4096) static unsigned char g_noalloc_host[kNoAllocHostBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};
cudaEvent_t g_noalloc_copied[256] = {};  // per device: the last table copy from g_noalloc_host
cudaEvent_t g_noalloc_last = nullptr;    // the event of the most recent copy on any device
bool g_noalloc_host_tried = false;

// Device address of the scratch array on `device`, looked up once per device
// with that device current (the array's name in host code is only a stand-in),
// and that device's copy event. Called with g_noalloc_mu held.
dsp_status noalloc_setup(int device, unsigned char** out) {
  if (device < 0 || device >= 256) return fail(DSP_E_UNSUPPORTED, "device %d out of range", device);
  if (!g_noalloc_host_tried) {
    // pinned for every context; if pinning is refused the copies stay correct
    // but come from pageable memory, which may make the host wait
    g_noalloc_host_tried = true;
    if (cudaHostRegister(g_noalloc_host, kNoAllocHostBytes, cudaHostRegisterPortable) != cudaSuccess)
      cudaGetLastError();
  }
  if (g_noalloc_addr[device] == nullptr) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves_noalloc: cudaGetDevice");
    if (cur != device) {
      e = cudaSetDevice(device);
      if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves_noalloc: cudaSetDevice");
    }
    void* p = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaError_t e2 = cur != device ? cudaSetDevice(cur) : cudaSuccess;
    if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves_noalloc: set-up on the device");
    if (e2 != cudaSuccess) return cuda_fail(e2, "dsp_expand_leaves_noalloc: restoring the device");
    g_noalloc_addr[device] = p;
    g_noalloc_copied[device] = ev;
  }
  *out = (unsigned char*)g_noalloc_addr[device];
  return DSP_OK;
}

}  // namespace
}  // namespace dsp

extern "C" dsp_status dsp_expand_leaves_noalloc(dsp_model* m, const dsp_leaf_job* jobs, int32_t n_jobs,
                                                void* stream) {
  using namespace dsp;
  if (!m) return fail(DSP_E_INVALID, "dsp_expand_leaves_noalloc: model is NULL");
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(DSP_E_INVALID, "dsp_expand_leaves_noalloc: bad job array");
  if (m->host->kind != DSP_MODEL_GRID && m->host->kind != DSP_MODEL_MULTIGRID)
    return fail(DSP_E_UNSUPPORTED, "dsp_expand_leaves_noalloc: Rock Sample models only");
  if (m->timing)
    return fail(DSP_E_UNSUPPORTED,
                "dsp_expand_leaves_noalloc: kernel timing is on (its events are created per call); turn it off");
  if (n_jobs == 0) return DSP_OK;
  if (n_jobs > kNoAllocJobs)
    return fail(DSP_E_UNSUPPORTED, "dsp_expand_leaves_noalloc: %d jobs, the fixed scratch holds at most %d", n_jobs,
                kNoAllocJobs);
  ExpandPlan plan;
  dsp_status vs = plan_units(m, jobs, n_jobs, plan);
  if (vs != DSP_OK) return vs;
  if (plan.total_items > kNoAllocItems)
    return fail(DSP_E_UNSUPPORTED,
                "dsp_expand_leaves_noalloc: %lld (action, scenario) items, the fixed scratch holds at most %lld",
                plan.total_items, kNoAllocItems);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  unsigned char* base = nullptr;
  vs = noalloc_setup(m->device, &base);
  if (vs != DSP_OK) return vs;
  cudaStream_t st = (cudaStream_t)stream;
  // table layout of this call: jobs, then (256-byte aligned) item offsets and order
  const size_t jb = ((sizeof(dsp_leaf_job) * (size_t)n_jobs + 255) / 256) * 256;
  const size_t span = jb + (sizeof(long long) + sizeof(int)) * (size_t)n_jobs;
  dsp_leaf_job* djobs = (dsp_leaf_job*)base;
  long long* dbase = (long long*)(base + jb);
  int* dorder = (int*)(dbase + n_jobs);
  unsigned int* counters = (unsigned int*)(base + kNoAllocTableBytes);
  uint32_t* items = (uint32_t*)(base + kNoAllocTableBytes + kNoAllocCounterBytes);
  // the host array is free once the previous call's copy has run
  cudaError_t e = g_noalloc_last ? cudaEventSynchronize(g_noalloc_last) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves_noalloc: waiting for the previous copy");
  std::memcpy(g_noalloc_host, jobs, sizeof(dsp_leaf_job) * (size_t)n_jobs);
  std::memcpy(g_noalloc_host + jb, plan.item_base.data(), sizeof(long long) * (size_t)n_jobs);
  std::memcpy(g_noalloc_host + jb + sizeof(long long) * (size_t)n_jobs, plan.order.data(),
              sizeof(int) * (size_t)n_jobs);
  e = cudaMemcpyAsync(base, g_noalloc_host, span, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventRecord(g_noalloc_copied[m->device], st);
  if (e == cudaSuccess) g_noalloc_last = g_noalloc_copied[m->device];
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, kNoAllocCounterBytes, st);
  if (e == cudaSuccess) {
    int block_b = m->tune_block > 0 ? m->tune_block : 256;
    bool large = false;
    for (int k = 0; k < n_jobs && !large; ++k) large = jobs[k].n_scen > kMaxScen;
    e = launch_rs_expand(m->dmodel, m->host->robots, m->host->num_actions, rs_key_words(m->host), m->dwork, djobs,
                         dbase, dorder, n_jobs, plan.total_items, items, counters, m->plan_step, m->num_sms,
                         block_b, m->policy_on ? m->policy : nullptr, st, m->tune_warps_a, m->tune_ctas_b, nullptr,
                         nullptr, large);
  }
  if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves_noalloc launch");
  return DSP_OK;
}
