// Autotuner of the expansion's launch shape. The paper fixes the mapping of
// work to the GPU (actions to thread blocks, scenarios to threads, factored
// elements to warps; Sec. III-D); here the mapping is a parameter: the CTA
// size and CTAs per SM of the rollout phase, the grouping phase's warps per
// CTA (actions per warp), the lanes that share one car scenario
// (element-level parallelism), the car kernel's CTAs per SM and, for one
// robot, whether the rollout phase reads items or rebuilds them. Each
// candidate is timed with CUDA events on the caller's jobs and the fastest
// is kept in the model.
#include <cuda_runtime.h>

#include <vector>

#include "model.hpp"

extern "C" dsp_status dsp_autotune(dsp_model* m, const dsp_leaf_job* jobs, int32_t n_jobs, int32_t reps,
                                   void* stream, int32_t* best_block, int32_t* best_tps, float* best_ms) {
  using namespace dsp;
  if (!m || !jobs || n_jobs < 1 || reps < 1 || !best_block || !best_tps || !best_ms)
    return fail(DSP_E_INVALID, "dsp_autotune: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<std::pair<int, int>> cands;
  if (m->host->kind == DSP_MODEL_CAR)
    cands = {{0, 4}, {0, 8}, {0, 16}, {0, 32}};
  else if (m->host->kind == DSP_MODEL_NAV)
    cands = {{0, 0}};  // one launch shape
  else
    cands = {{128, 0}, {256, 0}, {512, 0}};
  const int keep_block = m->tune_block, keep_tps = m->tune_tps;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(DSP_E_CUDA, "dsp_autotune: events");
  float best = -1.0f;
  int bb = keep_block, bt = keep_tps;
  dsp_status s = DSP_OK;
  for (auto& c : cands) {
    m->tune_block = c.first;
    m->tune_tps = c.second;
    s = dsp_expand_leaves(m, jobs, n_jobs, st);  // warm-up
    if (s != DSP_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps && s == DSP_OK; ++r) s = dsp_expand_leaves(m, jobs, n_jobs, st);
    cudaEventRecord(e1, st);
    if (s != DSP_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "dsp_autotune: timing");
      break;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best < 0 || ms < best) {
      best = ms;
      bb = c.first;
      bt = c.second;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != DSP_OK) {
    m->tune_block = keep_block;
    m->tune_tps = keep_tps;
    return s;
  }
  m->tune_block = bb;
  m->tune_tps = bt;
  *best_block = bb > 0 ? bb : 256;
  *best_tps = bt > 0 ? bt : (m->host->kind == DSP_MODEL_CAR ? car_default_tps(m->host->P) : 32);  // car only
  *best_ms = best;
  return DSP_OK;
}

namespace {

// Mean ms per dsp_expand_leaves call under the model's current shape, after
// one warm-up call.
dsp_status time_shape(dsp_model* m, const dsp_leaf_job* jobs, int n_jobs, int reps, cudaStream_t st, cudaEvent_t e0,
                      cudaEvent_t e1, float* ms) {
  dsp_status s = dsp_expand_leaves(m, jobs, n_jobs, st);
  if (s != DSP_OK) return s;
  cudaEventRecord(e0, st);
  for (int r = 0; r < reps && s == DSP_OK; ++r) s = dsp_expand_leaves(m, jobs, n_jobs, st);
  cudaEventRecord(e1, st);
  if (s != DSP_OK) return s;
  cudaError_t e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return dsp::cuda_fail(e, "dsp_autotune_shape: timing");
  cudaEventElapsedTime(ms, e0, e1);
  *ms /= (float)reps;
  return DSP_OK;
}

}  // namespace

extern "C" dsp_status dsp_autotune_shape(dsp_model* m, const dsp_leaf_job* jobs, int32_t n_jobs, int32_t reps,
                                         void* stream, dsp_launch_shape* best, float* best_ms, float* default_ms,
                                         int32_t* tried) {
  using namespace dsp;
  if (!m || !jobs || n_jobs < 1 || reps < 1) return fail(DSP_E_INVALID, "dsp_autotune_shape: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<dsp_launch_shape> cands;
  const int kind = m->host->kind;
  if (kind == DSP_MODEL_CAR) {
    for (int tps : {4, 8, 16, 32})
      for (int c : {0, 3, 2}) cands.push_back({0, 0, 0, tps, c, 0});
  } else if (kind == DSP_MODEL_NAV) {
    for (int c : {0, 6, 4, 2}) cands.push_back({0, c, 0, 0, 0, 0});
  } else {
    const bool two = m->host->robots == 2;
    // the rollout phase's two forms (one robot, heuristic policy)
    std::vector<int> forms = {0};
    if (!two && !m->policy_on) forms = {1, 2};
    for (int f : forms)
      for (int b : {128, 256, 512})
        for (int c : {0, 6, 4})
          for (int w : {0, two ? 8 : 5, two ? 16 : 10}) cands.push_back({b, c, w, 0, 0, f});
  }
  dsp_launch_shape keep;
  dsp_get_launch_shape(m, &keep);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(DSP_E_CUDA, "dsp_autotune_shape: events");
  const dsp_launch_shape dflt = {0, 0, 0, 0, 0, 0};
  dsp_set_launch_shape(m, &dflt);
  float dms = 0.0f;
  dsp_status s = time_shape(m, jobs, n_jobs, reps, st, e0, e1, &dms);
  dsp_launch_shape pick = dflt;
  float pms = dms;
  int n_tried = 1;
  for (size_t k = 0; k < cands.size() && s == DSP_OK; ++k) {
    s = dsp_set_launch_shape(m, &cands[k]);
    if (s != DSP_OK) break;
    float ms = 0.0f;
    s = time_shape(m, jobs, n_jobs, reps, st, e0, e1, &ms);
    n_tried += 1;
    if (s == DSP_OK && ms < pms) {
      pms = ms;
      pick = cands[k];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != DSP_OK) {
    dsp_set_launch_shape(m, &keep);
    return s;
  }
  dsp_set_launch_shape(m, &pick);
  if (best) *best = pick;
  if (best_ms) *best_ms = pms;
  if (default_ms) *default_ms = dms;
  if (tried) *tried = n_tried;
  return DSP_OK;
}
