// Pieces of the Rock Sample expansion shared by its kernels: constant loading,
// model set-up and the rollout-item list that links the grouping phase to the
// rollout phase.
#pragma once
#include "common.cuh"
#include "rs_model.cuh"

namespace dsp {

__device__ __forceinline__ void load_rs_consts(RSShared& c, const DevModel* gm) {
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) c.G[k] = gm->G[k];
  for (int k = threadIdx.x; k < kMaxRocks; k += blockDim.x) c.rock_xy[k] = gm->rock_xy[k];
  for (int k = threadIdx.x; k < kMaxSide * kMaxSide; k += blockDim.x) c.cell_rock[k] = gm->cell_rock[k];
}

// Copies the policy-key table into shared memory (no barrier).
__device__ __forceinline__ void load_rs_keys(uint16_t* dst, const DevModel* gm) {
  const int total = gm->m * gm->n * gm->n;
  for (int k = threadIdx.x; k < total; k += blockDim.x) dst[k] = gm->nkey[k];
}

template <int R>
__device__ __forceinline__ RSModel<R> make_rs(const DevModel* gm, const RSShared* c, uint32_t plan_step) {
  RSModel<R> M;
  M.sh = c;
  M.thresh = gm->thresh;
  M.n = gm->n;
  M.nn = gm->n * gm->n;
  M.nkey = gm->nkey;
  M.m = gm->m;
  M.per = gm->per_robot;
  M.D = gm->D;
  M.seed = gm->seed;
  M.plan_step = plan_step;
  return M;
}

// Item list (field-major, `total` items). The full layout, read by the
// learned-policy rollouts (their policy senses, so they need the scenario's
// random streams and the whole history): robot 0 [, robot 1], good, sampled,
// scenario, positive-counter mask of the child's history, depth<<24 | slot
// (slot = action * child_cap + child in the job's result arrays), job. The
// compact layout, read by the heuristic rollouts (they never sense and only
// need the believed-good unsampled rocks): robot 0 [, robot 1], good, the
// candidate mask (positive counter and not sampled), depth<<24 | slot, job.
template <int R>
struct Items {
  static constexpr int kFields = R == 2 ? 8 : 7;
  static constexpr int kCompactFields = R == 2 ? 6 : 5;
  uint32_t* base;
  long long total;
  bool full;
  __device__ __forceinline__ uint32_t* f(int k) const { return base + (size_t)k * total; }
  // the item of a stepped scenario s with its child's positive-counter mask
  __device__ __forceinline__ void put(size_t it, const RSS& s, uint32_t pm, uint32_t meta, uint32_t job) const {
    int k = 0;
    f(k++)[it] = s.pos[0];
    if (R == 2) f(k++)[it] = s.pos[1];
    f(k++)[it] = s.good;
    if (full) {
      f(k++)[it] = s.sampled;
      f(k++)[it] = s.scen;
      f(k++)[it] = pm;
    } else {
      f(k++)[it] = pm & ~s.sampled;
    }
    f(k++)[it] = meta;
    f(k)[it] = job;
  }
  // a compact item's good mask alone (a child whose other fields its slice holds)
  __device__ __forceinline__ void put_good(size_t it, uint32_t good) const { f(R == 2 ? 2 : 1)[it] = good; }
  // a compact item: the state for the heuristic rollout (sampled rocks are
  // out of the candidate mask, which takes the positive-counter mask's place)
  __device__ __forceinline__ void get_compact(size_t it, RSS& s, uint32_t& cand, uint32_t& meta, uint32_t& job) const {
    int k = 0;
    s.pos[0] = f(k++)[it];
    s.pos[1] = R == 2 ? f(k++)[it] : 0u;
    s.good = f(k++)[it];
    s.sampled = 0u;
    s.scen = 0u;
    cand = f(k++)[it];
    meta = f(k++)[it];
    job = f(k)[it];
  }
};

}  // namespace dsp
