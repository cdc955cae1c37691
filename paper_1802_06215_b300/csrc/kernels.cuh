// Host-side launchers of the device kernels (one per .cu file).
#pragma once
#include <cuda_runtime.h>

#include "common.cuh"

namespace dsp {

// Phase A's output for the block form of phase B (one robot, heuristic
// default policy), in place of the rollout-item list: job j's leaf states
// (position, good, sampled; field-major, n_scen each) at 3 * scen_base[j]
// words of `leaf`, and chunk_job[u] = j for each of the job's 32-position
// blocks u in [unit_base[j], unit_base[j] + n_actions * ceil(n_scen / 32)).
// Phase B rebuilds each (action, scenario)'s item from these, the grouped
// positions and the children's offsets and keys. leaf == nullptr: items.
struct LeafBlocks {
  uint32_t* leaf = nullptr;
  const long long* scen_base = nullptr;
  const long long* unit_base = nullptr;
  int* chunk_job = nullptr;
};

// Rock Sample (one or two robots), heuristic default policy, item list:
// phase A lists each child's items as slices of at most kSliceItems
// (kSliceItemsTwo) consecutive items at list[2 i], list[2 i + 1] for
// i < *count, and phase B takes slices instead of fixed chunks, so that the
// items it rolls out together always belong to one child (one trajectory for
// all of them). A slice is (first item, count | kSliceShared, robot 0's
// position, candidate mask) (depth << 24 | slot, job, robot 1's position, 0).
// With kSliceShared (a job whose scenarios share the robots' cells and the
// sampled mask) the child's items hold only their good masks and the slice
// holds the rest; else the items hold every field and the slice's position
// and candidate words are unused. list == nullptr: chunks.
struct Slices {
  uint4* list = nullptr;
  unsigned int* count = nullptr;
  unsigned int cap = 0;
};
constexpr int kSliceItems = 128;     // one robot: four items a lane
constexpr int kSliceItemsTwo = 128;  // two robots: four items a lane as well (no spills at 56 registers)
constexpr uint32_t kSliceShared = 1u << 31;

// Rock Sample: words per rollout item of the two-phase expansion.
int rs_item_fields(int robots, bool full);  // words per rollout item (full: learned-policy layout)
// Rock Sample two-phase expansion: phase A over n_jobs jobs (item_base[j] =
// first item of job j, total_items in all), phase B over the item list.
// counters: two device uints, zero on entry (job head, chunk head).
// policy: learned pi0 for the rollout phase (one robot), or null for the
// heuristic policy.
// order: phase A takes jobs in this order (null: index order).
// large_jobs: some one-robot job may hold more than kMaxScen scenarios.
// blocks: the block form (one robot, heuristic policy only): item_base and
// item_buf are unused and total_items is the number of 32-position blocks.
// Raises the rollout phase's dynamic shared-memory limit to hold the model's
// policy-key table (m * n * n keys); called once when the model is created.
cudaError_t rs_set_key_smem(int robots, int key_words);
// key_words: entries of the model's policy-key table, m * n * n.
cudaError_t launch_rs_expand(const DevModel* gm, int robots, int num_actions, int key_words, DevWork* work,
                             const dsp_leaf_job* jobs, const long long* item_base, const int* order, int n_jobs,
                             long long total_items, uint32_t* item_buf,
                             unsigned int* counters, uint32_t plan_step, int num_sms, int block_b,
                             const void* policy, cudaStream_t st, int warps_a = 0, int ctas_b = 0,
                             const LeafBlocks* blocks = nullptr, const Slices* slices = nullptr,
                             bool large_jobs = true);
// Learned-policy rollout phase over the item list (one robot).
cudaError_t launch_rs_rollout_mlp_items(const DevModel* gm, DevWork* work, const dsp_leaf_job* jobs,
                                        uint32_t* item_buf, long long total_items, unsigned int* counter,
                                        const void* policy, uint32_t plan_step, int num_sms, cudaStream_t st);
// Device view of the job ring (device addresses of mapped pinned host memory).
// Work sharing of one ring slot's job across the grid (device memory).
struct QueueShare {
  unsigned long long claim;   // (ticket & 0xFFFF) << 48 | chunk count << 24 | next chunk; count 0: closed
  unsigned long long ticket;  // full ticket of the published job
  unsigned int nchunks;       // rollout chunks of 32 items
  unsigned int remaining;     // chunks not yet finished
  unsigned int grain;         // chunks a warp takes per claim
  unsigned int plan_step;     // plan step of the published job
};
struct QueueRing {
  unsigned long long* seq;   // [cap] t + 1: ticket t published; t + cap: slot free for ticket t + cap
  dsp_leaf_job* jobs;        // [cap]
  unsigned long long* done;  // [cap] last finished ticket + 1
  unsigned int* close;       // nonzero: exit once no job is ready
  unsigned int* plan_step;   // [cap] plan step (fourth Philox counter word) of the slot's job
  QueueShare* share;         // [cap] device memory
  unsigned long long* finished;  // device: jobs completed (consumed tickets - finished = jobs in flight)
  int cap;
};
size_t rs_queue_slot_words(int robots, int num_actions);
int rs_queue_blocks_per_sm(int robots, int key_words);
cudaError_t launch_rs_queue(const DevModel* gm, int robots, int key_words, DevWork* work, QueueRing ring,
                            unsigned long long* head, uint32_t* scratch, size_t slot_words, dsp_leaf_job* jcopy,
                            unsigned long long idle_ns, int grid, cudaStream_t st);

cudaError_t launch_rs_step(const DevModel* gm, int robots, const uint32_t* in, int in_cap, int count,
                           const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                           float* rewards, uint32_t plan_step, cudaStream_t st);
cudaError_t launch_rs_rollout(const DevModel* gm, int robots, DevWork* work, const uint32_t* block, int cap,
                              int count, const int8_t* hist, int start_depth, float* value, uint32_t plan_step,
                              cudaStream_t st);

}  // namespace dsp
