// C ABI of the leaf-expansion library (include/dsp.h): model creation with its
// constant tables, argument validation, work-unit scheduling and launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "model.hpp"

namespace dsp {

static thread_local std::string g_last_error;

dsp_status fail(dsp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

dsp_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? DSP_E_OOM : DSP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Sensor thresholds: floor((0.5 + 0.5 * 2^(-d/20)) * 2^32) per squared distance.
static void build_thresholds(uint64_t* t, int max_d2) {
  for (int d2 = 0; d2 <= max_d2; ++d2) {
    double p = 0.5 + 0.5 * std::exp2(-std::sqrt((double)d2) / 20.0);
    t[d2] = (uint64_t)std::floor(p * 4294967296.0);
  }
}

// Quantile of N(0,1) by Newton's method on Phi(x) - p from x = 0. Phi is
// convex left of 0 and concave right of it, so the iterates approach the root
// monotonically from the side of 0.
static double normal_quantile(double p) {
  const double inv_sqrt2pi = 0.39894228040143267794;
  double x = 0.0;
  for (int it = 0; it < 200; ++it) {
    double f = 0.5 * std::erfc(-x * 0.70710678118654752440) - p;
    double d = inv_sqrt2pi * std::exp(-0.5 * x * x);
    double nx = x - f / d;
    if (nx == x) break;
    if (std::fabs(nx - x) <= 1e-17 * std::max(1.0, std::fabs(x))) {
      x = nx;
      break;
    }
    x = nx;
  }
  return x;
}

}  // namespace dsp

using namespace dsp;

extern "C" {

const char* dsp_last_error(void) { return g_last_error.c_str(); }

dsp_status dsp_create_model(const dsp_model_desc* d, dsp_model** out) {
  if (!out) return fail(DSP_E_INVALID, "dsp_create_model: out is NULL");
  *out = nullptr;
  if (!d) return fail(DSP_E_INVALID, "dsp_create_model: desc is NULL");
  if (d->kind < 0 || d->kind > 3) return fail(DSP_E_INVALID, "unknown model kind %d", d->kind);
  const int max_k = d->kind == DSP_MODEL_GRID ? kMaxScenLarge : kMaxScen;
  if (d->K < 1 || d->K > max_k) return fail(DSP_E_INVALID, "K=%d outside 1..%d", d->K, max_k);
  if (d->D < 1 || d->D > kGammaLen - 6) return fail(DSP_E_INVALID, "D=%d outside 1..%d", d->D, kGammaLen - 6);
  if (!(d->gamma > 0.0f && d->gamma <= 1.0f)) return fail(DSP_E_INVALID, "gamma must be in (0, 1]");
  DevModel* h = new DevModel();
  std::memset(h, 0, sizeof(DevModel));
  h->kind = d->kind;
  h->K = d->K;
  h->D = d->D;
  h->seed = d->seed;
  h->gamma = d->gamma;
  if (d->kind == DSP_MODEL_GRID || d->kind == DSP_MODEL_MULTIGRID) {
    if (d->n < 2 || d->n > kMaxSide) {
      delete h;
      return fail(DSP_E_INVALID, "map side n=%d outside 2..%d", d->n, kMaxSide);
    }
    if (d->m < 1 || d->m > kMaxRocks || !d->rock_cells) {
      delete h;
      return fail(DSP_E_INVALID, "rocks m=%d outside 1..%d (or rock_cells NULL)", d->m, kMaxRocks);
    }
    h->n = d->n;
    h->m = d->m;
    h->robots = d->kind == DSP_MODEL_GRID ? 1 : 2;
    h->per_robot = 5 + d->m;
    h->num_actions = h->robots == 1 ? h->per_robot : h->per_robot * h->per_robot;
    h->words = 5;
    std::memset(h->cell_rock, 0xFF, sizeof(h->cell_rock));
    for (int i = 0; i < d->m; ++i) {
      int x = d->rock_cells[i] & 0xFF, y = (d->rock_cells[i] >> 8) & 0xFF;
      if (x >= d->n || y >= d->n || h->cell_rock[y * d->n + x] != 0xFF) {
        delete h;
        return fail(DSP_E_INVALID, "rock %d at (%d,%d) outside the map or on another rock", i, x, y);
      }
      h->rock_xy[i] = x | (y << 8);
      h->cell_rock[y * d->n + x] = (uint8_t)i;
    }
    build_thresholds(h->thresh, 2 * (d->n - 1) * (d->n - 1));
    const int nn = d->n * d->n;
    for (int i = 0; i < d->m; ++i) {
      const int rx = h->rock_xy[i] & 0xFF, ry = h->rock_xy[i] >> 8;
      for (int y = 0; y < d->n; ++y)
        for (int x = 0; x < d->n; ++x) {
          const int dist = std::abs(x - rx) + std::abs(y - ry);
          const int mv = rx > x ? 1 : rx < x ? 3 : ry > y ? 0 : 2;
          h->nkey[i * nn + y * d->n + x] = (uint16_t)((dist << 7) | (i << 2) | (dist == 0 ? 0 : mv));
        }
    }
  } else if (d->kind == DSP_MODEL_NAV) {
    if (d->n < 5 || d->n > 16) {
      delete h;
      return fail(DSP_E_INVALID, "navigation map side n=%d outside 5..16", d->n);
    }
    if (!(d->fail_p >= 0.0 && d->fail_p <= 1.0) || !(d->sense_p >= 0.0 && d->sense_p <= 1.0)) {
      delete h;
      return fail(DSP_E_INVALID, "navigation probabilities outside [0, 1]");
    }
    h->n = d->n;
    h->num_actions = 9;
    h->words = 2 + (d->n * d->n + 31) / 32;
    h->fail_thresh = (uint64_t)std::floor(d->fail_p * 4294967296.0);
    h->sense_thresh = (uint64_t)std::floor(d->sense_p * 4294967296.0);
  } else {
    if (d->P < 1 || d->P > kMaxPeds) {
      delete h;
      return fail(DSP_E_INVALID, "pedestrians P=%d outside 1..%d", d->P, kMaxPeds);
    }
    h->P = d->P;
    h->num_actions = 3;
    h->words = 4 + 2 * d->P + (d->P + 3) / 4;
    h->path_len = d->path_len;
    h->dt = d->dt;
    h->ped_speed = d->ped_speed;
    h->sigma = d->sigma;
    h->stride = d->ped_speed * d->dt;
    h->fail_thresh = (uint64_t)std::floor(d->fail_p * 4294967296.0);
    for (int i = 0; i < kGaussLen; ++i) h->gauss[i] = (float)normal_quantile((i + 0.5) / (double)kGaussLen);
  }
  for (int k = 0; k < kGammaLen; ++k) h->G[k] = (float)std::pow((double)d->gamma, (double)k);

  dsp_model* m = new dsp_model();
  m->desc = *d;
  m->desc.rock_cells = nullptr;
  m->host = h;
  m->plan_step = d->plan_step;
  cudaError_t e = cudaGetDevice(&m->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device);
  if (e == cudaSuccess) {
    // The work buffers of each call come from this pool. Its release threshold
    // keeps freed memory mapped, so a call after a synchronisation does not
    // map its buffers again (the default pool returns them at every sync).
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = m->device;
    e = cudaMemPoolCreate(&m->pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      e = cudaMemPoolSetAttribute(m->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&m->dmodel, sizeof(DevModel));
  if (e == cudaSuccess) e = cudaMalloc(&m->dwork, sizeof(DevWork));
  if (e == cudaSuccess) e = cudaMemcpy(m->dmodel, h, sizeof(DevModel), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->dwork, 0, sizeof(DevWork));
  if (e == cudaSuccess && h->robots > 0) e = rs_set_key_smem(h->robots, rs_key_words(h));
  if (e != cudaSuccess) {
    dsp_status st = cuda_fail(e, "dsp_create_model");
    dsp_destroy_model(m);
    return st;
  }
  *out = m;
  return DSP_OK;
}

void dsp_destroy_model(dsp_model* m) {
  if (!m) return;
  if (m->dmodel) cudaFree(m->dmodel);
  if (m->dwork) cudaFree(m->dwork);
  if (m->policy) cudaFree(m->policy);
  for (cudaEvent_t ev : m->timing_events) cudaEventDestroy(ev);
  for (cudaEvent_t ev : m->timing_pool) cudaEventDestroy(ev);
  for (dsp_staging_slot* sl : m->staging) {
    cudaEventSynchronize(sl->done);
    cudaEventDestroy(sl->done);
    cudaFreeHost(sl->host);
    delete sl;
  }
  if (m->queue) dsp_queue_destroy(m->queue);
  if (m->pool) cudaMemPoolDestroy(m->pool);
  delete m->host;
  delete m;
}

int32_t dsp_state_words(const dsp_model* m) { return m ? m->host->words : 0; }
int32_t dsp_num_actions(const dsp_model* m) { return m ? m->host->num_actions : 0; }
int32_t dsp_max_children(const dsp_model* m, int32_t n_scen) {
  if (!m) return 0;
  const int kind = m->host->kind;
  int z = kind == DSP_MODEL_GRID ? 4 : (kind == DSP_MODEL_MULTIGRID ? 10 : (kind == DSP_MODEL_NAV ? 257 : n_scen));
  return std::min(z, n_scen);
}

dsp_status dsp_set_plan_step(dsp_model* m, uint32_t plan_step) {
  if (!m) return fail(DSP_E_INVALID, "dsp_set_plan_step: model is NULL");
  m->plan_step = plan_step;
  return DSP_OK;
}

dsp_status dsp_get_table(const dsp_model* m, int32_t which, void* out, int32_t* count) {
  if (!m || !out || !count) return fail(DSP_E_INVALID, "dsp_get_table: NULL argument");
  const DevModel* h = m->host;
  if (which == 0) {
    int n = (h->kind == DSP_MODEL_CAR || h->kind == DSP_MODEL_NAV) ? 0 : 2 * (h->n - 1) * (h->n - 1) + 1;
    std::memcpy(out, h->thresh, n * sizeof(uint64_t));
    *count = n;
  } else if (which == 1) {
    std::memcpy(out, h->G, sizeof(h->G));
    *count = kGammaLen;
  } else if (which == 2) {
    std::memcpy(out, h->gauss, sizeof(h->gauss));
    *count = kGaussLen;
  } else {
    return fail(DSP_E_INVALID, "dsp_get_table: unknown table %d", which);
  }
  return DSP_OK;
}

dsp_status dsp_step(const dsp_model* m, const uint32_t* in, int32_t in_cap, int32_t count, const int32_t* actions,
                    int32_t depth, uint32_t* out, int32_t out_cap, uint64_t* keys, float* rewards, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_step: model is NULL");
  if (count < 0 || in_cap < count || out_cap < count) return fail(DSP_E_INVALID, "dsp_step: bad count/capacity");
  if (count == 0) return DSP_OK;
  if (!in || !out || !actions || !keys || !rewards) return fail(DSP_E_INVALID, "dsp_step: NULL buffer");
  if (depth < 0) return fail(DSP_E_INVALID, "dsp_step: negative depth");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (m->host->kind == DSP_MODEL_CAR)
    e = launch_car_step(m->dmodel, m->host->P, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                        m->plan_step, st);
  else if (m->host->kind == DSP_MODEL_NAV)
    e = launch_nav_step(m->dmodel, in, in_cap, count, actions, depth, out, out_cap, keys, rewards, m->plan_step, st);
  else
    e = launch_rs_step(m->dmodel, m->host->robots, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                       m->plan_step, st);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_step launch");
}

dsp_status dsp_rollout(const dsp_model* m, const uint32_t* block, int32_t cap, int32_t count, const int8_t* hist,
                       int32_t start_depth, float* value, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_rollout: model is NULL");
  if (count < 0 || cap < count) return fail(DSP_E_INVALID, "dsp_rollout: bad count/capacity");
  if (count == 0) return DSP_OK;
  if (!block || !value) return fail(DSP_E_INVALID, "dsp_rollout: NULL buffer");
  if (start_depth < 0 || start_depth > m->host->D)
    return fail(DSP_E_INVALID, "dsp_rollout: start depth %d outside 0..D", start_depth);
  if (m->policy_on) return dsp_rollout_logged(m, block, cap, count, hist, start_depth, value, nullptr, nullptr, stream);
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (m->host->kind == DSP_MODEL_CAR)
    e = launch_car_rollout(m->dmodel, m->host->P, m->dwork, block, cap, count, start_depth, value, m->plan_step,
                           st);
  else if (m->host->kind == DSP_MODEL_NAV)
    e = launch_nav_rollout(m->dmodel, m->dwork, block, cap, count, hist, start_depth, value, m->plan_step, st);
  else
    e = launch_rs_rollout(m->dmodel, m->host->robots, m->dwork, block, cap, count, hist, start_depth, value,
                          m->plan_step, st);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_rollout launch");
}

dsp_status dsp_expand_leaves(dsp_model* m, const dsp_leaf_job* jobs, int32_t n_jobs, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_expand_leaves: model is NULL");
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(DSP_E_INVALID, "dsp_expand_leaves: bad job array");
  if (n_jobs == 0) return DSP_OK;
  ExpandPlan plan;
  dsp_status vs = plan_units(m, jobs, n_jobs, plan, true);
  if (vs != DSP_OK) return vs;
  return launch_expand(m, jobs, n_jobs, plan, (cudaStream_t)stream);
}

dsp_status dsp_read_counters(dsp_model* m, uint64_t* steps, uint32_t* status) {
  if (!m) return fail(DSP_E_INVALID, "dsp_read_counters: model is NULL");
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "dsp_read_counters sync");
  DevWork w;
  e = cudaMemcpy(&w, m->dwork, sizeof(DevWork), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_read_counters copy");
  if (steps) *steps = w.steps;
  if (status) *status = w.status;
  return DSP_OK;
}

dsp_status dsp_set_tuning(dsp_model* m, int32_t block, int32_t tps) {
  if (!m) return fail(DSP_E_INVALID, "dsp_set_tuning: model is NULL");
  if (!(block == 0 || block == 128 || block == 256 || block == 512))
    return fail(DSP_E_INVALID, "dsp_set_tuning: block %d not in {0,128,256,512}", block);
  if (m->host->kind == DSP_MODEL_CAR && block != 0 && block != 256)
    return fail(DSP_E_INVALID, "dsp_set_tuning: the car kernel runs 256-thread CTAs");
  if (!(tps == 0 || tps == 4 || tps == 8 || tps == 16 || tps == 32))
    return fail(DSP_E_INVALID, "dsp_set_tuning: tps %d not in {0,4,8,16,32}", tps);
  m->tune_block = block;
  m->tune_tps = tps;
  return DSP_OK;
}

dsp_status dsp_get_tuning(const dsp_model* m, int32_t* block, int32_t* tps) {
  if (!m || !block || !tps) return fail(DSP_E_INVALID, "dsp_get_tuning: NULL argument");
  *block = m->tune_block > 0 ? m->tune_block : 256;
  *tps = m->tune_tps > 0 ? m->tune_tps : (m->host->kind == DSP_MODEL_CAR ? car_default_tps(m->host->P) : 32);
  return DSP_OK;
}

dsp_status dsp_set_launch_shape(dsp_model* m, const dsp_launch_shape* s) {
  if (!m || !s) return fail(DSP_E_INVALID, "dsp_set_launch_shape: NULL argument");
  if (!(s->block_b == 0 || s->block_b == 128 || s->block_b == 256 || s->block_b == 512))
    return fail(DSP_E_INVALID, "dsp_set_launch_shape: block_b %d not in {0,128,256,512}", s->block_b);
  if (!(s->tps == 0 || s->tps == 4 || s->tps == 8 || s->tps == 16 || s->tps == 32))
    return fail(DSP_E_INVALID, "dsp_set_launch_shape: tps %d not in {0,4,8,16,32}", s->tps);
  if (s->ctas_b < 0 || s->ctas_b > 32 || s->ctas_car < 0 || s->ctas_car > 32)
    return fail(DSP_E_INVALID, "dsp_set_launch_shape: CTAs per SM outside 0..32");
  if (s->warps_a < 0 || s->warps_a > 16)
    return fail(DSP_E_INVALID, "dsp_set_launch_shape: warps_a %d outside 0..16", s->warps_a);
  if (s->rs_form < 0 || s->rs_form > 2)
    return fail(DSP_E_INVALID, "dsp_set_launch_shape: rs_form %d outside 0..2", s->rs_form);
  m->tune_block = s->block_b;
  m->tune_ctas_b = s->ctas_b;
  m->tune_warps_a = s->warps_a;
  m->tune_tps = s->tps;
  m->tune_ctas_car = s->ctas_car;
  m->tune_rs_form = s->rs_form;
  return DSP_OK;
}

dsp_status dsp_get_launch_shape(const dsp_model* m, dsp_launch_shape* s) {
  if (!m || !s) return fail(DSP_E_INVALID, "dsp_get_launch_shape: NULL argument");
  s->block_b = m->tune_block;
  s->ctas_b = m->tune_ctas_b;
  s->warps_a = m->tune_warps_a;
  s->tps = m->tune_tps;
  s->ctas_car = m->tune_ctas_car;
  s->rs_form = m->tune_rs_form;
  return DSP_OK;
}

dsp_status dsp_kernel_timing(dsp_model* m, int32_t enable, double* total_ms, int32_t* calls) {
  if (!m) return fail(DSP_E_INVALID, "dsp_kernel_timing: model is NULL");
  std::lock_guard<std::mutex> lock(m->timing_mu);
  double tot = 0;
  int n = 0;
  for (size_t i = 0; i + 1 < m->timing_events.size(); i += 2) {
    cudaError_t e = cudaEventSynchronize(m->timing_events[i + 1]);
    if (e != cudaSuccess) return cuda_fail(e, "dsp_kernel_timing");
    float ms = 0;
    cudaEventElapsedTime(&ms, m->timing_events[i], m->timing_events[i + 1]);
    tot += ms;
    n += 1;
  }
  for (cudaEvent_t ev : m->timing_events) m->timing_pool.push_back(ev);
  m->timing_events.clear();
  m->timing = enable != 0;
  if (total_ms) *total_ms = tot;
  if (calls) *calls = n;
  return DSP_OK;
}

dsp_status dsp_reset_counters(dsp_model* m, void* stream) {
  if (!m) return fail(DSP_E_INVALID, "dsp_reset_counters: model is NULL");
  cudaError_t e = cudaMemsetAsync(m->dwork, 0, sizeof(DevWork), (cudaStream_t)stream);
  return e == cudaSuccess ? DSP_OK : cuda_fail(e, "dsp_reset_counters");
}

}  // extern "C"

namespace dsp {

// Validates the jobs and plans the launch: car and navigation units are (job,
// action), each with the first index of its rollout items; Rock Sample jobs
// get the first index of theirs (n_scen * n_actions each, in job order).
dsp_status plan_units(const dsp_model* m, const dsp_leaf_job* jobs, int n_jobs, ExpandPlan& plan, bool allow_blocks) {
  const DevModel* h = m->host;
  plan.units.clear();
  plan.item_base.clear();
  plan.unit_base.clear();
  plan.scen_base.clear();
  plan.total_items = plan.total_blocks = plan.total_scen = plan.slice_cap = 0;
  plan.large_jobs = false;
  plan.blocks = allow_blocks && h->kind != DSP_MODEL_CAR && h->kind != DSP_MODEL_NAV && h->robots == 1 &&
                !m->policy_on && m->tune_rs_form == 1;
  plan.slices = allow_blocks && (h->kind == DSP_MODEL_GRID || h->kind == DSP_MODEL_MULTIGRID) && !m->policy_on &&
                !plan.blocks;
  for (int j = 0; j < n_jobs; ++j) {
    const dsp_leaf_job& J = jobs[j];
    const int max_n = h->kind == DSP_MODEL_GRID ? kMaxScenLarge : kMaxScen;
    if (J.n_scen < 1 || J.n_scen > max_n)
      return fail(DSP_E_UNSUPPORTED, "job %d: n_scen=%d outside 1..%d", j, J.n_scen, max_n);
    if (J.n_scen > kMaxScen && J.leaf_states == nullptr)
      return fail(DSP_E_UNSUPPORTED, "job %d: more than %d scenarios need leaf_states", j, kMaxScen);
    if (J.n_scen > kMaxScen) plan.large_jobs = true;
    if (J.n_actions < 1 || J.first_action < 0 || J.first_action + J.n_actions > h->num_actions)
      return fail(DSP_E_INVALID, "job %d: actions [%d,%d) outside 0..%d", j, J.first_action,
                  J.first_action + J.n_actions, h->num_actions);
    if (J.depth < 0 || J.depth >= h->D) return fail(DSP_E_INVALID, "job %d: depth %d outside 0..D-1", j, J.depth);
    if (J.last_action >= h->num_actions || J.last_action < -1)
      return fail(DSP_E_INVALID, "job %d: last action %d", j, J.last_action);
    if (J.last_action >= 0 && J.depth == 0) return fail(DSP_E_INVALID, "job %d: update step at depth 0", j);
    if (!J.parent || !J.idx || J.parent_cap < 1) return fail(DSP_E_INVALID, "job %d: parent block missing", j);
    if (J.child_cap < 1 || !J.child_count || !J.child_off || !J.child_key || !J.rew_sum || !J.u_sum || !J.l_sum ||
        !J.perm)
      return fail(DSP_E_INVALID, "job %d: result buffer missing", j);
    if ((long long)J.n_actions * J.child_cap >= (1LL << 24))
      return fail(DSP_E_UNSUPPORTED, "job %d: n_actions * child_cap >= 2^24", j);
    if (h->kind == DSP_MODEL_CAR || h->kind == DSP_MODEL_NAV) {
      for (int a = 0; a < J.n_actions; ++a) plan.units.push_back(make_int4(j, a, 1, 0));
    } else if (plan.blocks) {
      plan.unit_base.push_back(plan.total_blocks);
      plan.scen_base.push_back(plan.total_scen);
      plan.total_blocks += (long long)J.n_actions * ((J.n_scen + 31) / 32);
      plan.total_scen += J.n_scen;
      plan.total_items += (long long)J.n_scen * J.n_actions;
    } else {
      plan.item_base.push_back(plan.total_items);
      plan.total_items += (long long)J.n_scen * J.n_actions;
      // an action's children (at most 6 observation codes) in runs of at
      // most kSliceItems
      if (plan.slices) {
        // one robot: at most 6 observation codes an action; two robots: 18
        const int len = h->robots == 1 ? kSliceItems : kSliceItemsTwo, codes = h->robots == 1 ? 6 : 18;
        plan.slice_cap += (long long)J.n_actions * ((J.n_scen + len - 1) / len + codes);
      }
    }
  }
  if (plan.slice_cap >= (1LL << 31)) plan.slices = false;
  if (plan.total_items >= (1LL << 31)) return fail(DSP_E_UNSUPPORTED, "more than 2^31 (action, scenario) items");
  // Largest work first (units and jobs are independent, so the order changes
  // no result): persistent CTAs that pull work in this order end together
  // instead of waiting on one large unit drawn last.
  if (h->kind == DSP_MODEL_CAR || h->kind == DSP_MODEL_NAV) {
    std::stable_sort(plan.units.begin(), plan.units.end(), [&](const int4& x, const int4& y) {
      return jobs[x.x].n_scen > jobs[y.x].n_scen;
    });
    // first rollout item of each unit (navigation's phase B, the car's learned rollouts)
    for (int4& u : plan.units) {
      u.z = (int)plan.total_items;
      plan.total_items += jobs[u.x].n_scen;
      if (plan.total_items >= (1LL << 31)) return fail(DSP_E_UNSUPPORTED, "more than 2^31 (action, scenario) items");
    }
  } else {
    // sorted on a contiguous (work, index) array: the order of a stable sort
    // by decreasing work, without touching the job table again
    std::vector<std::pair<long long, int>> key(n_jobs);
    for (int j = 0; j < n_jobs; ++j) key[j] = {-(long long)jobs[j].n_scen * jobs[j].n_actions, j};
    std::sort(key.begin(), key.end());
    plan.order.resize(n_jobs);
    for (int j = 0; j < n_jobs; ++j) plan.order[j] = key[j].second;
  }
  return DSP_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// A pinned staging slot of at least `bytes` whose last copy has run, or a new
// one; null if pinned memory cannot be had (the caller then copies from its
// own pageable buffers). Pinned sources keep cudaMemcpyAsync asynchronous, so
// a call returns without waiting for the work queued before it.
static dsp_staging_slot* take_staging(dsp_model* m, size_t bytes) {
  std::lock_guard<std::mutex> lock(m->staging_mu);
  for (dsp_staging_slot* sl : m->staging)
    if (!sl->busy && sl->cap >= bytes && cudaEventQuery(sl->done) == cudaSuccess) {
      sl->busy = true;
      return sl;
    }
  dsp_staging_slot* sl = new dsp_staging_slot();
  sl->cap = std::max<size_t>((bytes + 0xFFFFF) & ~(size_t)0xFFFFF, 1 << 20);
  if (cudaHostAlloc(&sl->host, sl->cap, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    delete sl;
    return nullptr;
  }
  if (cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(sl->host);
    delete sl;
    return nullptr;
  }
  sl->busy = true;
  m->staging.push_back(sl);
  return sl;
}

// Marks the slot's copy (already enqueued on st) and frees the slot for reuse
// once that copy has run.
static cudaError_t release_staging(dsp_model* m, dsp_staging_slot* sl, cudaStream_t st) {
  cudaError_t e = cudaEventRecord(sl->done, st);
  std::lock_guard<std::mutex> lock(m->staging_mu);
  sl->busy = false;
  return e;
}

// Two timing events from the model's pool (created once, returned to the pool
// when dsp_kernel_timing has read them).
static void take_timing_events(dsp_model* m, cudaEvent_t (&ev)[2]) {
  std::lock_guard<std::mutex> lock(m->timing_mu);
  for (int k = 0; k < 2; ++k) {
    if (!m->timing_pool.empty()) {
      ev[k] = m->timing_pool.back();
      m->timing_pool.pop_back();
    } else {
      cudaEventCreate(&ev[k]);
    }
  }
}

// Copies the job table (and the unit table, or Rock Sample's item offsets) to
// stream-ordered device memory, takes the rollout-item list from the same
// allocation and launches the expansion kernels.
dsp_status launch_expand(dsp_model* m, const dsp_leaf_job* jobs, int n_jobs, const ExpandPlan& plan,
                         cudaStream_t st) {
  const DevModel* h = m->host;
  const bool car = h->kind == DSP_MODEL_CAR, nav = h->kind == DSP_MODEL_NAV;
  const bool by_unit = car || nav;  // (job, action) units instead of Rock Sample's item list
  size_t jb = sizeof(dsp_leaf_job) * (size_t)n_jobs;
  // Rock Sample: per-job offsets (item list: first item; block form: first
  // block and first leaf scenario), then the phase-A order
  const size_t nb = plan.blocks ? 2 * plan.unit_base.size() : plan.item_base.size();
  size_t ub = by_unit ? sizeof(int4) * plan.units.size() : sizeof(long long) * nb + sizeof(int) * plan.order.size();
  const bool car_items = car && m->policy_on;
  // block form: the leaves' states (3 words a scenario), then each block's job
  size_t ib = car   ? (car_items ? sizeof(uint32_t) * (size_t)(h->words + 2) * (size_t)plan.total_items : 0)
              : nav ? sizeof(uint32_t) * (size_t)nav_item_fields(h->n) * (size_t)plan.total_items
              : plan.blocks
                  ? align256(sizeof(uint32_t) * 3 * (size_t)plan.total_scen) + sizeof(int) * (size_t)plan.total_blocks
                  : sizeof(uint32_t) * (size_t)rs_item_fields(h->robots, m->policy_on) * (size_t)plan.total_items;
  const bool slices = !by_unit && plan.slices;
  const size_t sb = slices ? 2 * sizeof(uint4) * (size_t)plan.slice_cap : 0;
  size_t total = align256(jb) + align256(ub) + 256 + align256(ib) + sb;
  unsigned char* buf = nullptr;
  cudaError_t e = cudaMallocFromPoolAsync((void**)&buf, total, m->pool, st);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves: work buffers");
  dsp_leaf_job* djobs = (dsp_leaf_job*)buf;
  void* dunits = buf + align256(jb);
  unsigned int* counters = (unsigned int*)(buf + align256(jb) + align256(ub));
  uint32_t* items = (uint32_t*)(buf + align256(jb) + align256(ub) + 256);
  const int* dorder = by_unit ? nullptr : (const int*)((const long long*)dunits + nb);
  // the job table and the unit table (or item offsets and order) in one copy
  // from pinned staging laid out like the device buffer
  const size_t hb = align256(jb) + ub;
  dsp_staging_slot* sl = take_staging(m, hb);
  if (sl != nullptr) {
    unsigned char* hs = (unsigned char*)sl->host;
    std::memcpy(hs, jobs, jb);
    if (by_unit) {
      std::memcpy(hs + align256(jb), plan.units.data(), ub);
    } else if (plan.blocks) {
      const size_t n = plan.unit_base.size();
      std::memcpy(hs + align256(jb), plan.unit_base.data(), sizeof(long long) * n);
      std::memcpy(hs + align256(jb) + sizeof(long long) * n, plan.scen_base.data(), sizeof(long long) * n);
      std::memcpy(hs + align256(jb) + sizeof(long long) * nb, plan.order.data(), sizeof(int) * plan.order.size());
    } else {
      std::memcpy(hs + align256(jb), plan.item_base.data(), sizeof(long long) * plan.item_base.size());
      std::memcpy(hs + align256(jb) + sizeof(long long) * plan.item_base.size(), plan.order.data(),
                  sizeof(int) * plan.order.size());
    }
    e = cudaMemcpyAsync(buf, hs, hb, cudaMemcpyHostToDevice, st);
    cudaError_t er = release_staging(m, sl, st);
    if (e == cudaSuccess) e = er;
  } else {
    e = cudaMemcpyAsync(djobs, jobs, jb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && by_unit)
      e = cudaMemcpyAsync(dunits, plan.units.data(), ub, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !by_unit && plan.blocks) {
      const size_t n = plan.unit_base.size();
      e = cudaMemcpyAsync(dunits, plan.unit_base.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((long long*)dunits + n, plan.scen_base.data(), sizeof(long long) * n,
                            cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)dorder, plan.order.data(), sizeof(int) * plan.order.size(),
                            cudaMemcpyHostToDevice, st);
    } else if (e == cudaSuccess && !by_unit) {
      e = cudaMemcpyAsync(dunits, plan.item_base.data(), sizeof(long long) * plan.item_base.size(),
                          cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync((void*)dorder, plan.order.data(), sizeof(int) * plan.order.size(),
                            cudaMemcpyHostToDevice, st);
    }
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, 256, st);
  if (e == cudaSuccess) {
    cudaEvent_t ev[2] = {nullptr, nullptr};
    if (m->timing) {
      take_timing_events(m, ev);
      cudaEventRecord(ev[0], st);
    }
    if (car) {
      CarItems ci{car_items ? items : nullptr, plan.total_items, h->words};
      e = launch_car_expand(m, djobs, (const int4*)dunits, (int)plan.units.size(), counters, ci, st);
      if (e == cudaSuccess && car_items) e = launch_car_rollout_mlp_items(m, djobs, ci, counters + 1, st);
    } else if (nav) {
      e = launch_nav_expand(m, djobs, (const int4*)dunits, (int)plan.units.size(), counters, items,
                            plan.total_items, st);
    } else {
      int block_b = m->tune_block > 0 ? m->tune_block : 256;
      LeafBlocks lb;
      if (plan.blocks) {
        const size_t n = plan.unit_base.size();
        lb.leaf = items;
        lb.unit_base = (const long long*)dunits;
        lb.scen_base = (const long long*)dunits + n;
        lb.chunk_job = (int*)((unsigned char*)items + align256(sizeof(uint32_t) * 3 * (size_t)plan.total_scen));
      }
      Slices sl;
      if (slices) {
        sl.list = (uint4*)((unsigned char*)items + align256(ib));
        sl.cap = (unsigned int)plan.slice_cap;
      }
      e = launch_rs_expand(m->dmodel, h->robots, h->num_actions, rs_key_words(h), m->dwork, djobs,
                           (const long long*)dunits, dorder, n_jobs,
                           plan.blocks ? plan.total_blocks : plan.total_items, items, counters, m->plan_step,
                           m->num_sms, block_b, m->policy_on ? m->policy : nullptr, st, m->tune_warps_a,
                           m->tune_ctas_b, plan.blocks ? &lb : nullptr, slices ? &sl : nullptr, plan.large_jobs);
    }
    if (m->timing) {
      cudaEventRecord(ev[1], st);
      std::lock_guard<std::mutex> lock(m->timing_mu);
      m->timing_events.push_back(ev[0]);
      m->timing_events.push_back(ev[1]);
    }
  }
  cudaError_t e2 = cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_expand_leaves launch");
  if (e2 != cudaSuccess) return cuda_fail(e2, "dsp_expand_leaves free");
  return DSP_OK;
}

}  // namespace dsp
