// Leaf expansion for navigation in a partially known map (Sec. III-D on the
// task of Sec. IV-A), in two launches.
//
// Phase A (nav_group_kernel): one (job, action) unit per CTA pass, largest
// jobs first; one thread per scenario: gather + update by the action into the
// leaf, the expansion step g with its 8-bit observation and u0. The unit's
// scenarios are grouped by observation with the shared-memory hash of
// group.cuh (the key is the observation itself, so no further comparison is
// needed); the children's reward and u sums are exact int64 fixed-point
// atomics, and each scenario's state after the step goes to a rollout item.
//
// Phase B (nav_rollout_items_kernel): the default-policy rollouts (Eq. lb) of
// all items without a barrier. Each scenario carries its own map, so rollouts
// differ in length; a lane whose rollout ends takes the next item of its
// warp's chunk (and the warp the next chunk) before the next step, so the
// lanes stay busy, and adds its value to the child's int64 l sum with one
// atomic (exact in any order).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "group.cuh"
#include "model.hpp"
#include "nav_model.cuh"
#include "queue_ring.cuh"

namespace dsp {

namespace {

struct NavUnitSmem {
  NavTables T;
  uint64_t key[kMaxScen];
  float rew[kMaxScen], uval[kMaxScen];
  GroupSmem grp;
  unsigned long long sr[kMaxScen], su[kMaxScen];
  int unit;
  dsp_leaf_job job;
};

// Rollout items, field-major with stride `total`, the state as phase B
// holds it in registers: word 0 = x | y << 4 | terminal << 8 | neighbours
// << 9 | last reading << 17, then the kNavRowWords row words of the map, the
// scenario id, depth << 24 | result slot (action offset * child_cap + child),
// job.
constexpr int kNavItemWords = kNavRowWords + 4;
struct NavItems {
  uint32_t* base;
  long long total;
  __device__ __forceinline__ uint32_t* f(int k) const { return base + (size_t)k * (size_t)total; }
};

// One (job, action) unit of phase A by the whole CTA, the job's descriptor
// in S.job: gather + update into the leaf, the step with its 8-bit reading,
// u0 and one rollout item per scenario at item_base (job index job_index in
// the items), then the grouping by reading, the exact reward and u sums and
// the results of action offset `ao` (l sums start at zero; phase B adds the
// rollouts). Ends with a barrier.
__device__ __forceinline__ void nav_unit(NavUnitSmem& S, const NavModel& M, int ao, long long item_base, int job_index,
                                         const NavItems& items, DevWork* work, unsigned long long& steps) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const dsp_leaf_job& job = S.job;
  const int n = job.n_scen, depth = job.depth;
  const int a = job.first_action + ao;
  const bool first_unit = ao == 0;
  const uint32_t last0 = (uint32_t)(uint8_t)job.hist[0];
  const long long ibase = item_base;
  for (int p = tid; p < n; p += nthr) {
    NavS s = M.load(job.parent, job.parent_cap, job.idx[p]);
    if (job.last_action >= 0) {  // update by the action into this leaf
      if (!s.term && first_unit) steps += 1;
      uint64_t k0;
      M.step(s, job.last_action, depth - 1, k0);
    }
    const int src = job.idx[p];
    if (first_unit && job.leaf_states != nullptr) {
      M.store_pos(s, job.leaf_states, n, p);
      M.copy_map(job.parent, job.parent_cap, src, job.leaf_states, n, p);
    }
    // Eq. expand with the observation key
    if (!s.term) steps += 1;
    uint64_t key;
    const float r = M.step(s, a, depth, key);
    // Eq. ub (the tail heuristic is zero at depth D); Eq. lb starts from the
    // child's history, whose last reading is the one just taken
    const float uv = (depth + 1 >= M.D) ? 0.0f : M.upper(s);
    const uint32_t last = (key & kTermBit) ? last0 : (uint32_t)(key & 0xFFu);
    const long long it = ibase + p;
    items.f(0)[it] = (uint32_t)s.x | ((uint32_t)s.y << 4) | ((uint32_t)s.term << 8) | (s.nb << 9) | (last << 17);
#pragma unroll
    for (int k = 0; k < kNavRowWords; ++k) items.f(1 + k)[it] = s.R[k];
    items.f(1 + kNavRowWords)[it] = s.scen;
    S.key[p] = key;
    S.rew[p] = r;
    S.uval[p] = uv;
  }
  for (int c = tid; c < n; c += nthr) {
    S.sr[c] = 0;
    S.su[c] = 0;
  }
  __syncthreads();
  group_by_key(S.grp, S.key, n);
  const int nchild = S.grp.nchild;
  for (int q = tid; q < n; q += nthr) {
    const int c = S.grp.gcid[q];
    atomicAdd(&S.sr[c], (unsigned long long)to_fixed(S.rew[q]));
    atomicAdd(&S.su[c], (unsigned long long)to_fixed(S.uval[q]));
  }
  __syncthreads();
  const int cap = job.child_cap;
  if (tid == 0) {
    job.child_count[ao] = nchild;
    if (nchild > cap) report(work, kStatusOverflow);
  }
  const int ncw = min(nchild, cap);
  for (int c = tid; c <= ncw; c += nthr) job.child_off[(size_t)ao * (cap + 1) + c] = c < nchild ? S.grp.coff[c] : n;
  for (int c = tid; c < ncw; c += nthr) {
    const size_t o = (size_t)ao * cap + c;
    job.child_key[o] = S.key[S.grp.cfirst[c]];
    job.rew_sum[o] = (long long)S.sr[c];
    job.u_sum[o] = (long long)S.su[c];
    job.l_sum[o] = 0;  // phase B adds the rollouts
  }
  for (int q = tid; q < n; q += nthr) {
    const int c = S.grp.gcid[q];
    job.perm[(size_t)ao * n + S.grp.coff[c] + S.grp.rank[q]] = (uint16_t)q;
    const long long it = ibase + q;
    items.f(2 + kNavRowWords)[it] = ((uint32_t)depth << 24) | (uint32_t)(ao * cap + min(c, cap - 1));
    items.f(3 + kNavRowWords)[it] = (uint32_t)job_index;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256, 4) nav_group_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                        const dsp_leaf_job* __restrict__ jobs,
                                                        const int4* __restrict__ units, int n_units,
                                                        unsigned int* head, NavItems items, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NavUnitSmem& S = *reinterpret_cast<NavUnitSmem*>(smem_raw);
  load_nav_tables(S.T, gm);
  const NavModel M = make_nav(gm, &S.T, plan_step);
  const int tid = threadIdx.x;
  unsigned long long steps = 0;
  __syncthreads();
  while (true) {
    if (tid == 0) S.unit = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int u = S.unit;
    __syncthreads();
    if (u >= n_units) break;
    const int4 un = units[u];
    if (tid == 0) S.job = jobs[un.x];
    __syncthreads();
    nav_unit(S, M, un.y, un.z, un.x, items, work, steps);
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

constexpr int kWarpsB = 8;  // phase-B CTA: 256 threads

// Per warp, two 32-item chunks of the item list in shared memory: the one the
// lanes take items from and the next, copied in with cp.async while the
// current one is rolled out, so that a lane that takes an item reads shared
// memory instead of waiting on global memory.
struct NavStage {
  uint32_t w[2][kNavItemWords][32];
};

__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
}

// Claims the next chunk for the warp and starts copying it into buffer b;
// returns the chunk's item count (0: none left).
__device__ __forceinline__ int stage_chunk(NavStage& st, int b, const NavItems& items, unsigned int* chunk_head,
                                           long long nchunks, int lane) {
  long long ch = 0;
  if (lane == 0) ch = (long long)atomicAdd(chunk_head, 1u);
  ch = __shfl_sync(0xFFFFFFFFu, ch, 0);
  if (ch >= nchunks) return 0;
  const long long it = ch * 32 + lane;
  if (it < items.total)
#pragma unroll
    for (int k = 0; k < kNavItemWords; ++k) cp_async4(&st.w[b][k][lane], items.f(k) + it);
  asm volatile("cp.async.commit_group;" ::: "memory");
  return (int)min(32LL, items.total - ch * 32);
}

// Phase B for one warp: takes 32-item chunks of the item list from
// chunk_head (staged in st), rolls each item out with lane refill, and adds
// each value to its child's l sum in jobs[job].
__device__ __forceinline__ void nav_rollout_warp(const NavModel& M, const NavTables& T, NavStage& st,
                                                 const NavItems& items, unsigned int* chunk_head,
                                                 const dsp_leaf_job* jobs, unsigned long long& steps) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = lanemask_lt();
  const long long nchunks = (items.total + 31) >> 5;
  // warp-uniform: buffer in use, items handed out of it, its size, the next's size
  int cur = 0, off = 0;
  int cur_n = stage_chunk(st, 0, items, chunk_head, nchunks, lane);
  int next_n = cur_n ? stage_chunk(st, 1, items, chunk_head, nchunks, lane) : 0;
  if (next_n)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  bool have = false;  // this lane holds an item
  NavS s{};
  uint32_t last = 0, slot = 0, job = 0;
  int t = 0, t0 = 0;
  float v = 0.0f;
  while (true) {
    // idle lanes take the next items, in lane order
    uint32_t idle = __ballot_sync(0xFFFFFFFFu, !have);
    while (idle != 0u && (off < cur_n || next_n > 0)) {
      if (off >= cur_n) {  // switch to the next chunk, start copying the one after
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        cur ^= 1;
        cur_n = next_n;
        off = 0;
        next_n = stage_chunk(st, cur ^ 1, items, chunk_head, nchunks, lane);
      }
      const int give = min(__popc(idle), cur_n - off);
      const int rank = __popc(idle & lt);
      if (!have && rank < give) {
        const int i = off + rank;
        const uint32_t w0 = st.w[cur][0][i];
        s.x = (int)(w0 & 0xFu);
        s.y = (int)((w0 >> 4) & 0xFu);
        s.term = (w0 >> 8) & 1u;
        s.nb = (w0 >> 9) & 0xFFu;
        last = (w0 >> 17) & 0xFFu;
#pragma unroll
        for (int k = 0; k < kNavRowWords; ++k) s.R[k] = st.w[cur][1 + k][i];
        s.scen = st.w[cur][1 + kNavRowWords][i];
        const uint32_t meta = st.w[cur][2 + kNavRowWords][i];
        job = st.w[cur][3 + kNavRowWords][i];
        slot = meta & 0xFFFFFFu;
        t0 = (int)(meta >> 24) + 1;
        t = t0;
        v = 0.0f;
        have = true;
      }
      off += give;
      idle = __ballot_sync(0xFFFFFFFFu, !have);
    }
    if (__ballot_sync(0xFFFFFFFFu, have) == 0u) break;
    // one step of the default policy (the body of NavModel::rollout)
    if (have && t < M.D && !s.term) {
      uint64_t key;
      const float r = M.step(s, M.policy(last), t, key);
      steps += 1;
      if (!(key & kTermBit)) last = (uint32_t)(key & 0xFFu);
      v = __fadd_rn(v, __fmul_rn(T.G[t - t0], r));
      t += 1;
    }
    if (have && (t >= M.D || s.term)) {
      const long long fl = to_fixed(v);
      if (fl != 0) sum_add(jobs[job].l_sum + slot, fl);
      have = false;
    }
  }
}

__global__ void __launch_bounds__(256, 4) nav_rollout_items_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                                const dsp_leaf_job* __restrict__ jobs,
                                                                NavItems items, unsigned int* chunk_head,
                                                                uint32_t plan_step) {
  __shared__ NavTables T;
  __shared__ NavStage stage[kWarpsB];
  load_nav_tables(T, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, &T, plan_step);
  const int lane = threadIdx.x & 31;
  unsigned long long steps = 0;
  nav_rollout_warp(M, T, stage[threadIdx.x >> 5], items, chunk_head, jobs, steps);
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if (lane == 0 && steps) atomicAdd(&work->steps, steps);
}

// Persistent queue kernel of navigation: a CTA claims a published job, runs
// phase A for each of its actions (nav_unit) into the slot's item list, then
// its warps roll the job's items out (nav_rollout_warp, chunks taken from a
// shared counter), and it publishes the job done. Idle CTAs back off and exit
// after idle_ns without a job; the host relaunches the kernel when jobs come.
struct NavQueueSmem {
  NavUnitSmem u;
  NavStage stage[kWarpsB];
  unsigned int chunk_head;
  long long ticket;
  unsigned int plan_step;
  int exit;
};

__global__ void __launch_bounds__(256, 2) nav_queue_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                          QueueRing ring, unsigned long long* head,
                                                          uint32_t* scratch, size_t slot_words, dsp_leaf_job* jcopy,
                                                          unsigned long long idle_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NavQueueSmem& Q = *reinterpret_cast<NavQueueSmem*>(smem_raw);
  NavUnitSmem& S = Q.u;
  load_nav_tables(S.T, gm);
  NavModel M = make_nav(gm, &S.T, 0u);
  const int tid = threadIdx.x;
  unsigned long long steps = 0, last_work = qring::now_ns();
  unsigned int backoff = 256;
  __syncthreads();
  while (true) {
    if (tid < 32) {
      const long long t = qring::take_job(ring, head, &S.job, jcopy, &Q.plan_step);
      if (tid == 0) {
        Q.ticket = t;
        Q.chunk_head = 0;
      }
    }
    __syncthreads();
    const long long ticket = Q.ticket;
    if (ticket >= 0) {
      const int slot = (int)(ticket % ring.cap);
      M.plan_step = Q.plan_step;
      const NavItems items{scratch + (size_t)slot * slot_words, (long long)S.job.n_scen * S.job.n_actions};
      for (int ao = 0; ao < S.job.n_actions; ++ao)
        nav_unit(S, M, ao, (long long)ao * S.job.n_scen, 0, items, work, steps);
      nav_rollout_warp(M, S.T, Q.stage[tid >> 5], items, &Q.chunk_head, jcopy + slot, steps);
      __threadfence();  // every thread's sums, before the job is published done
      __syncthreads();
      if (tid == 0) qring::finish_job(ring, (unsigned long long)ticket);
    }
    if (tid == 0) Q.exit = qring::idle_exit(ring, ticket >= 0, last_work, backoff, idle_ns);
    __syncthreads();
    if (Q.exit) break;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_step: one g call per scenario.
__global__ void __launch_bounds__(256, 4) nav_step_kernel(const DevModel* __restrict__ gm, const uint32_t* in,
                                                       int in_cap, int count, const int32_t* actions, int depth,
                                                       uint32_t* out, int out_cap, uint64_t* keys, float* rewards,
                                                       uint32_t plan_step) {
  __shared__ NavTables T;
  load_nav_tables(T, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, &T, plan_step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    NavS s = M.load(in, in_cap, i);
    uint64_t key;
    const float r = M.step(s, actions[i], depth, key);
    M.store_pos(s, out, out_cap, i);
    M.copy_map(in, in_cap, i, out, out_cap, i);
    keys[i] = key;
    rewards[i] = r;
  }
}

// dsp_rollout: Eq. lb per scenario from start_depth; the last reading is byte 0
// of the scenario's 32-byte history (0 without a history).
__global__ void __launch_bounds__(256, 4) nav_rollout_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                          const uint32_t* block, int cap, int count,
                                                          const int8_t* hist, int start_depth, float* value,
                                                          uint32_t plan_step) {
  __shared__ NavTables T;
  load_nav_tables(T, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, &T, plan_step);
  unsigned long long steps = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    NavS s = M.load(block, cap, i);
    const uint32_t last = hist != nullptr ? (uint32_t)(uint8_t)hist[(size_t)32 * i] : 0u;
    value[i] = M.rollout(s, last, start_depth, steps);
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

}  // namespace

int nav_item_fields(int) { return kNavItemWords; }

cudaError_t launch_nav_expand(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units,
                              unsigned int* counters, uint32_t* items, long long total_items, cudaStream_t st) {
  const size_t smem = sizeof(NavUnitSmem);
  cudaError_t e = cudaFuncSetAttribute(nav_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nav_group_kernel, 256, smem);
  const int grid = std::max(1, std::min(n_units, std::max(1, per_sm) * m->num_sms));
  const NavItems it{items, total_items};
  nav_group_kernel<<<grid, 256, smem, st>>>(m->dmodel, m->dwork, djobs, dunits, n_units, counters, it, m->plan_step);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int per_sm_b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, nav_rollout_items_kernel, 32 * kWarpsB, 0);
  if (m->tune_ctas_b > 0) per_sm_b = std::min(per_sm_b, m->tune_ctas_b);
  const long long warps = (total_items + 31) / 32;
  const int grid_b = (int)std::max(
      1LL, std::min((warps + kWarpsB - 1) / kWarpsB, (long long)std::max(1, per_sm_b) * m->num_sms));
  nav_rollout_items_kernel<<<grid_b, 32 * kWarpsB, 0, st>>>(m->dmodel, m->dwork, djobs, it, counters + 1, m->plan_step);
  return cudaGetLastError();
}

cudaError_t nav_queue_setup(int* per_sm) {
  const size_t smem = sizeof(NavQueueSmem);
  cudaError_t e = cudaFuncSetAttribute(nav_queue_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, nav_queue_kernel, 256, smem);
  return e;
}

size_t nav_queue_slot_words(const dsp_model* m) {
  return (size_t)kNavItemWords * (size_t)kMaxScen * (size_t)m->host->num_actions;
}

cudaError_t launch_nav_queue(dsp_model* m, QueueRing ring, unsigned long long* head, uint32_t* scratch,
                             size_t slot_words, dsp_leaf_job* jcopy, unsigned long long idle_ns, int grid,
                             cudaStream_t st) {
  nav_queue_kernel<<<grid, 256, sizeof(NavQueueSmem), st>>>(m->dmodel, m->dwork, ring, head, scratch, slot_words,
                                                            jcopy, idle_ns);
  return cudaGetLastError();
}

// The navigation default policy per state: it reads only the last reading,
// kept in counter 0 of the history.
__global__ void nav_policy_kernel(const DevModel* __restrict__ gm, const int8_t* __restrict__ hist, int count,
                                  int32_t* __restrict__ actions) {
  __shared__ NavTables T;
  load_nav_tables(T, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, &T, 0u);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) actions[i] = M.policy((uint32_t)(uint8_t)hist[32 * (size_t)i]);
}

cudaError_t launch_nav_policy(const DevModel* gm, const int8_t* hist, int count, int32_t* actions, cudaStream_t st) {
  nav_policy_kernel<<<(count + 255) / 256, 256, 0, st>>>(gm, hist, count, actions);
  return cudaGetLastError();
}

cudaError_t launch_nav_step(const DevModel* gm, const uint32_t* in, int in_cap, int count, const int32_t* actions,
                            int depth, uint32_t* out, int out_cap, uint64_t* keys, float* rewards, uint32_t plan_step,
                            cudaStream_t st) {
  const int grid = std::min(4096, (count + 255) / 256);
  nav_step_kernel<<<grid, 256, 0, st>>>(gm, in, in_cap, count, actions, depth, out, out_cap, keys, rewards,
                                        plan_step);
  return cudaGetLastError();
}

cudaError_t launch_nav_rollout(const DevModel* gm, DevWork* work, const uint32_t* block, int cap, int count,
                               const int8_t* hist, int start_depth, float* value, uint32_t plan_step,
                               cudaStream_t st) {
  const int grid = std::min(4096, (count + 255) / 256);
  nav_rollout_kernel<<<grid, 256, 0, st>>>(gm, work, block, cap, count, hist, start_depth, value, plan_step);
  return cudaGetLastError();
}

}  // namespace dsp
