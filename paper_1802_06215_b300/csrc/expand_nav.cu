// Leaf expansion for navigation in a partially known map (Sec. III-D on the
// task of Sec. IV-A). One (job, action) unit per CTA pass, largest jobs
// first; one thread per scenario: gather + update by the action into the
// leaf, the expansion step g with its 8-bit observation, u0, and the
// default-policy rollout to depth D in registers. The unit's scenarios are
// grouped by observation with the shared-memory hash of group.cuh (the key is
// the observation itself, so no further comparison is needed), and the
// children's reward, u and l sums are exact int64 fixed-point atomics.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "group.cuh"
#include "model.hpp"
#include "nav_model.cuh"

namespace dsp {

namespace {

struct NavUnitSmem {
  float G[kGammaLen];
  uint64_t key[kMaxScen];
  float rew[kMaxScen], uval[kMaxScen], lval[kMaxScen];
  GroupSmem grp;
  unsigned long long sr[kMaxScen], su[kMaxScen], sl[kMaxScen];
  int unit;
  dsp_leaf_job job;
};

__device__ __forceinline__ void load_gamma(float* G, const DevModel* gm) {
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) G[k] = gm->G[k];
}

__global__ void __launch_bounds__(256, 4) nav_expand_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                         const dsp_leaf_job* __restrict__ jobs,
                                                         const int4* __restrict__ units, int n_units,
                                                         unsigned int* head, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NavUnitSmem& S = *reinterpret_cast<NavUnitSmem*>(smem_raw);
  load_gamma(S.G, gm);
  const NavModel M = make_nav(gm, S.G, plan_step);
  const int tid = threadIdx.x, nthr = blockDim.x;
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
    const dsp_leaf_job& job = S.job;
    const int n = job.n_scen, depth = job.depth;
    const int a = job.first_action + un.y;
    const bool first_unit = un.y == 0;
    const uint32_t last0 = (uint32_t)(uint8_t)job.hist[0];
    for (int p = tid; p < n; p += nthr) {
      NavS s = M.load(job.parent, job.parent_cap, job.idx[p]);
      if (job.last_action >= 0) {  // update by the action into this leaf
        if (!s.term && first_unit) steps += 1;
        uint64_t k0;
        M.step(s, job.last_action, depth - 1, k0);
      }
      if (first_unit && job.leaf_states != nullptr) M.store(s, job.leaf_states, n, p);
      // Eq. expand with the observation key
      if (!s.term) steps += 1;
      uint64_t key;
      const float r = M.step(s, a, depth, key);
      // Eq. ub (the tail heuristic is zero at depth D) and Eq. lb from the
      // child's history: the reading just taken
      const float uv = (depth + 1 >= M.D) ? 0.0f : M.upper(s);
      const uint32_t last = (key & kTermBit) ? last0 : (uint32_t)(key & 0xFFu);
      const float lv = s.term ? 0.0f : M.rollout(s, last, depth + 1, steps);
      S.key[p] = key;
      S.rew[p] = r;
      S.uval[p] = uv;
      S.lval[p] = lv;
    }
    for (int c = tid; c < n; c += nthr) {
      S.sr[c] = 0;
      S.su[c] = 0;
      S.sl[c] = 0;
    }
    __syncthreads();
    group_by_key(S.grp, S.key, n);
    const int nchild = S.grp.nchild;
    for (int q = tid; q < n; q += nthr) {
      const int c = S.grp.gcid[q];
      atomicAdd(&S.sr[c], (unsigned long long)to_fixed(S.rew[q]));
      atomicAdd(&S.su[c], (unsigned long long)to_fixed(S.uval[q]));
      atomicAdd(&S.sl[c], (unsigned long long)to_fixed(S.lval[q]));
    }
    __syncthreads();
    const int cap = job.child_cap;
    const int ao = un.y;
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
      job.l_sum[o] = (long long)S.sl[c];
    }
    for (int q = tid; q < n; q += nthr) {
      const int c = S.grp.gcid[q];
      job.perm[(size_t)ao * n + S.grp.coff[c] + S.grp.rank[q]] = (uint16_t)q;
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((tid & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_step: one g call per scenario.
__global__ void __launch_bounds__(256) nav_step_kernel(const DevModel* __restrict__ gm, const uint32_t* in,
                                                       int in_cap, int count, const int32_t* actions, int depth,
                                                       uint32_t* out, int out_cap, uint64_t* keys, float* rewards,
                                                       uint32_t plan_step) {
  __shared__ float G[kGammaLen];
  load_gamma(G, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, G, plan_step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    NavS s = M.load(in, in_cap, i);
    uint64_t key;
    const float r = M.step(s, actions[i], depth, key);
    M.store(s, out, out_cap, i);
    keys[i] = key;
    rewards[i] = r;
  }
}

// dsp_rollout: Eq. lb per scenario from start_depth; the last reading is byte 0
// of the scenario's 32-byte history (0 without a history).
__global__ void __launch_bounds__(256) nav_rollout_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                          const uint32_t* block, int cap, int count,
                                                          const int8_t* hist, int start_depth, float* value,
                                                          uint32_t plan_step) {
  __shared__ float G[kGammaLen];
  load_gamma(G, gm);
  __syncthreads();
  const NavModel M = make_nav(gm, G, plan_step);
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

cudaError_t launch_nav_expand(dsp_model* m, const dsp_leaf_job* djobs, const int4* dunits, int n_units,
                              unsigned int* head, cudaStream_t st) {
  const size_t smem = sizeof(NavUnitSmem);
  cudaError_t e = cudaFuncSetAttribute(nav_expand_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nav_expand_kernel, 256, smem);
  const int grid = std::max(1, std::min(n_units, std::max(1, per_sm) * m->num_sms));
  nav_expand_kernel<<<grid, 256, smem, st>>>(m->dmodel, m->dwork, djobs, dunits, n_units, head, m->plan_step);
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
