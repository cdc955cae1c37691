// Host-side model object behind the opaque dsp_model handle.
#pragma once
#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "common.cuh"

// Pinned host staging for one call's job table: reused once the copy that
// last read it has run (its event).
struct dsp_staging_slot {
  void* host = nullptr;
  size_t cap = 0;
  cudaEvent_t done = nullptr;
  bool busy = false;
};

struct dsp_model {
  dsp_model_desc desc;
  dsp::DevModel* host = nullptr;     // host copy of the constant block
  dsp::DevModel* dmodel = nullptr;   // device copy
  dsp::DevWork* dwork = nullptr;     // counters and status word
  uint32_t plan_step = 0;
  int device = 0;
  int num_sms = 0;
  cudaMemPool_t pool = nullptr;      // stream-ordered work buffers; keeps its peak size until destroy
  dsp_queue* queue = nullptr;        // device job queue of the tree search, kept across planning steps
  int queue_cap = 0;
  // launch shape (dsp_set_launch_shape / the autotuner); 0 = default
  int tune_block = 0;                // rollout phase CTA size (Rock Sample)
  int tune_tps = 0;                  // car: threads per scenario
  int tune_ctas_b = 0;               // rollout phase CTAs per SM (Rock Sample, navigation)
  int tune_warps_a = 0;              // Rock Sample grouping phase: warps per CTA
  int tune_ctas_car = 0;             // car kernel CTAs per SM
  int tune_rs_form = 0;              // one-robot Rock Sample rollout phase: 1 blocks, 2 items (0: items)
  void* policy = nullptr;            // learned pi0 for rollouts (device, transposed BF16 weights)
  bool policy_on = false;
  bool timing = false;               // record events around the expansion kernels
  std::mutex timing_mu;
  std::vector<cudaEvent_t> timing_events;  // start, end per dsp_expand_leaves call
  std::vector<cudaEvent_t> timing_pool;    // events read back, for reuse
  std::mutex staging_mu;
  std::vector<dsp_staging_slot*> staging;  // pinned copies of the calls' job tables
};

namespace dsp {

// The history update a node's child takes from its observation key (the
// default policies' input): Rock Sample belief counters (+-1 per Sense
// reading, clamped to +-127), the navigation's last reading in counter 0, and
// nothing for the car.
inline void host_observe(int kind, int per_robot, int8_t* h, int a, uint64_t key) {
  if (kind == DSP_MODEL_CAR) return;
  if (kind == DSP_MODEL_NAV) {
    if (!(key & (1ull << 62))) h[0] = (int8_t)(uint8_t)(key & 0xFFu);
    return;
  }
  const int z = (int)(key & ~(1ull << 62));
  int acts[2], zs[2];
  const int robots = kind == DSP_MODEL_GRID ? 1 : 2;
  if (robots == 1) {
    acts[0] = a;
    zs[0] = z;
  } else {
    acts[0] = a / per_robot;
    acts[1] = a % per_robot;
    zs[0] = z / 3;
    zs[1] = z % 3;
  }
  for (int r = 0; r < robots; ++r) {
    if (acts[r] >= 5 && zs[r] != 0) {
      const int i = acts[r] - 5;
      const int v = (int)h[i] + (zs[r] == 1 ? 1 : -1);
      h[i] = (int8_t)(v > 127 ? 127 : (v < -127 ? -127 : v));
    }
  }
}

dsp_status fail(dsp_status st, const char* fmt, ...);
dsp_status cuda_fail(cudaError_t e, const char* what);

struct ExpandPlan {
  std::vector<int4> units;            // car: (job, action, 1, 0)
  std::vector<long long> item_base;   // Rock Sample: first rollout item of each job
  std::vector<int> order;             // Rock Sample: jobs by decreasing n_scen * n_actions (phase-A order)
  long long total_items = 0;
  // Rock Sample, block form of the rollout phase (one robot, heuristic
  // policy): first 32-position block and first leaf scenario of each job
  bool blocks = false;
  std::vector<long long> unit_base, scen_base;
  long long total_blocks = 0, total_scen = 0;
  // Rock Sample, one robot, heuristic policy, item list: the rollout phase
  // takes each child's items in slices; at most slice_cap of them
  bool slices = false;
  long long slice_cap = 0;
  bool large_jobs = false;  // a job holds more than kMaxScen scenarios
};
// allow_blocks: the block form or slices may be planned (dsp_expand_leaves,
// which allocates their buffers); the no-allocation entry point and the
// queue's validation plan items in chunks.
dsp_status plan_units(const dsp_model* m, const dsp_leaf_job* jobs, int n_jobs, ExpandPlan& plan,
                      bool allow_blocks = false);
dsp_status launch_expand(dsp_model* m, const dsp_leaf_job* jobs, int n_jobs, const ExpandPlan& plan,
                         cudaStream_t st);

// Navigation expansion: phase A groups each (job, action) unit and writes one
// rollout item per scenario (nav_item_fields(n) words each, field-major);
// phase B rolls the items out. counters[0] and counters[1] start at 0.
int nav_item_fields(int n);
cudaError_t launch_nav_expand(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units,
                              unsigned int* counters, uint32_t* items, long long total_items, cudaStream_t st);
cudaError_t launch_nav_step(const DevModel* gm, const uint32_t* in, int in_cap, int count, const int32_t* actions,
                            int depth, uint32_t* out, int out_cap, uint64_t* keys, float* rewards, uint32_t plan_step,
                            cudaStream_t st);
cudaError_t launch_nav_rollout(const DevModel* gm, DevWork* work, const uint32_t* block, int cap, int count,
                               const int8_t* hist, int start_depth, float* value, uint32_t plan_step,
                               cudaStream_t st);
struct QueueRing;  // kernels.cuh
// Persistent queue kernels of the navigation and car models (queue.cu):
// set-up (shared-memory limit, CTAs per SM), scratch sizes and the launch.
// Navigation: per ring slot, one job's rollout items (slot_words each);
// car: per CTA, one observation scratch.
cudaError_t nav_queue_setup(int* per_sm);
size_t nav_queue_slot_words(const dsp_model* m);
cudaError_t launch_nav_queue(dsp_model* m, QueueRing ring, unsigned long long* head, uint32_t* scratch,
                             size_t slot_words, dsp_leaf_job* jcopy, unsigned long long idle_ns, int grid,
                             cudaStream_t st);
cudaError_t car_queue_setup(const dsp_model* m, int* per_sm);
size_t car_queue_scratch_words(int grid);
cudaError_t launch_car_queue(dsp_model* m, QueueRing ring, unsigned long long* head, uint32_t* scratch,
                             dsp_leaf_job* jcopy, unsigned long long idle_ns, int grid, cudaStream_t st);
// Lanes per car scenario when untuned: enough for one pedestrian pair per
// lane (4 to 32).
int car_default_tps(int P);
cudaError_t launch_car_expand(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units,
                              unsigned int* head, CarItems items, cudaStream_t st);
// Learned-policy rollouts of the car expansion's items; counter: a device
// uint, zero on entry.
cudaError_t launch_car_rollout_mlp_items(dsp_model* m, const dsp_leaf_job* jobs, CarItems items, unsigned int* counter,
                                         cudaStream_t st);
// Learned-policy rollouts of single car scenarios (dsp_rollout_logged).
cudaError_t launch_car_rollout_logged(const dsp_model* m, const uint32_t* block, int cap, int count, int start_depth,
                                      float* value, int32_t* actions, float* logits, unsigned int* counter,
                                      cudaStream_t st);
// Default policies per state (dsp_default_policy).
cudaError_t launch_car_policy(const dsp_model* m, const uint32_t* block, int cap, int count, int32_t* actions,
                              cudaStream_t st);
cudaError_t launch_nav_policy(const DevModel* gm, const int8_t* hist, int count, int32_t* actions, cudaStream_t st);
// Learned-policy features of car states (dsp_features).
cudaError_t launch_car_features(const dsp_model* m, const uint32_t* block, int cap, int count, float* out,
                                cudaStream_t st);
cudaError_t launch_car_step(const DevModel* gm, int P, const uint32_t* in, int in_cap, int count,
                            const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                            float* rewards, uint32_t plan_step, cudaStream_t st);
cudaError_t launch_car_rollout(const DevModel* gm, int P, DevWork* work, const uint32_t* block, int cap, int count,
                               int start_depth, float* value, uint32_t plan_step, cudaStream_t st);

}  // namespace dsp
