// Leaf expansion for Rock Sample models (one or two robots): the fused
// gather -> update -> expansion -> grouping -> bounds -> reduction path of
// Sec. III-D as one persistent kernel.
//
// Work is cut into units (job, run of actions) whose items (action, scenario)
// fit one CTA (<= kItems). A CTA pulls units from a device counter until none
// is left, so leaves of uneven |Phi_b| and action counts balance across SMs.
// Per unit:
//   1. gather the leaf's scenarios from the parent list and apply the last
//      action (update), keeping the leaf's states in shared memory;
//   2. step every item with g (Eq. expand);
//   3. group each action's items by observation (shared-memory hash of
//      (action, key), first-occurrence leaders, warp ballots for child
//      numbering, warp __match_any_sync for stable ranks) (Eq. newnodes);
//   4. in child-grouped order (so a warp's lanes follow the same child and
//      branch alike) compute u (Eq. ub) and the default-policy rollout
//      (Eq. lb) in registers;
//   5. sum rewards, u and l per child in int64 fixed point (shared atomics,
//      exact in any order) and write the results.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.cuh"
#include "rs_model.cuh"

namespace dsp {

namespace {

constexpr int kItems = 512;      // items (action, scenario) per unit
constexpr int kTable = 1024;     // hash slots (>= 2 * kItems)
constexpr uint64_t kEmpty = ~0ull;

struct RSUnitSmem {
  RSShared c;
  uint32_t leaf[5][kMaxScen];      // the leaf's states, field-major
  uint32_t next[5][kItems];        // stepped state of each item
  uint64_t key[kItems];
  float rew[kItems];
  uint16_t slot[kItems];
  uint16_t gcid[kItems];
  uint16_t rank[kItems];
  uint16_t permitem[kItems];       // item at each grouped position
  uint64_t tkey[kTable];
  uint32_t tfirst[kTable];
  uint16_t tcid[kTable];
  int32_t cfirst[kItems];          // first item of each child
  int32_t ccount[kItems];
  int32_t coff[kItems];
  int32_t abase[kItems + 1];       // first child of each action of the unit
  unsigned long long sr[kItems], su[kItems], sl[kItems];
  int nchild;
  int unit;
  dsp_leaf_job job;
};

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

__device__ __forceinline__ uint32_t hash_slot(uint64_t ident) {
  uint64_t z = ident * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(z >> 40) & (kTable - 1);
}

template <int R>
__device__ void rs_unit(RSUnitSmem& S, const RSModel<R>& M, const dsp_leaf_job& job, int a_begin, int a_count,
                        DevWork* work, unsigned long long& steps) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int n = job.n_scen;
  const int items = a_count * n;
  const int depth = job.depth;
  const int a_first = job.first_action + a_begin;

  // 1. gather + update
  for (int p = tid; p < n; p += nthr) {
    RSS s = M.load(job.parent, job.parent_cap, job.idx[p]);
    if (job.last_action >= 0) {
      if (!M.terminal(s) && a_begin == 0) steps += 1;
      uint64_t k;
      M.step(s, job.last_action, depth - 1, k);
    }
    S.leaf[0][p] = s.pos[0];
    S.leaf[1][p] = s.pos[1];
    S.leaf[2][p] = s.good;
    S.leaf[3][p] = s.sampled;
    S.leaf[4][p] = s.scen;
    if (a_begin == 0 && job.leaf_states != nullptr) M.store(s, job.leaf_states, n, p);
  }
  for (int t = tid; t < kTable; t += nthr) {
    S.tkey[t] = kEmpty;
    S.tfirst[t] = 0xFFFFFFFFu;
  }
  for (int g = tid; g < items; g += nthr) {
    S.sr[g] = 0;
    S.su[g] = 0;
    S.sl[g] = 0;
  }
  __syncthreads();

  // 2. expansion step of every item, 3a. hash insert of (action, key)
  for (int i = tid; i < items; i += nthr) {
    int al = i / n, p = i - al * n;
    RSS s;
    s.pos[0] = S.leaf[0][p];
    s.pos[1] = S.leaf[1][p];
    s.good = S.leaf[2][p];
    s.sampled = S.leaf[3][p];
    s.scen = S.leaf[4][p];
    if (!M.terminal(s)) steps += 1;
    uint64_t key;
    float r = M.step(s, a_first + al, depth, key);
    S.next[0][i] = s.pos[0];
    S.next[1][i] = s.pos[1];
    S.next[2][i] = s.good;
    S.next[3][i] = s.sampled;
    S.next[4][i] = s.scen;
    S.key[i] = key;
    S.rew[i] = r;
    uint64_t ident = ((uint64_t)al << 32) | (key & 0xFFFFull) | ((key >> 62) << 31);
    uint32_t h = hash_slot(ident);
    while (true) {
      unsigned long long prev = atomicCAS((unsigned long long*)&S.tkey[h], (unsigned long long)kEmpty,
                                          (unsigned long long)ident);
      if (prev == kEmpty || prev == ident) break;
      h = (h + 1) & (kTable - 1);
    }
    atomicMin(&S.tfirst[h], (uint32_t)i);
    S.slot[i] = (uint16_t)h;
  }
  __syncthreads();

  // 3b. number children in item order (first occurrence), 3c. stable ranks
  if (warp == 0) {
    int base = 0;
    for (int c0 = 0; c0 < items; c0 += 32) {
      int i = c0 + lane;
      bool lead = i < items && S.tfirst[S.slot[i]] == (uint32_t)i;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, lead);
      if (lead) {
        int g = base + __popc(bal & lanemask_lt());
        S.tcid[S.slot[i]] = (uint16_t)g;
        S.cfirst[g] = i;
        S.ccount[g] = 0;
      }
      base += __popc(bal);
    }
    if (lane == 0) S.nchild = base;
    __syncwarp();
    for (int c0 = 0; c0 < items; c0 += 32) {
      int i = c0 + lane;
      bool ok = i < items;
      int g = ok ? S.tcid[S.slot[i]] : -1 - lane;
      uint32_t peers = __match_any_sync(0xFFFFFFFFu, g);
      int base_g = ok ? S.ccount[g] : 0;
      __syncwarp();
      if (ok) {
        S.gcid[i] = (uint16_t)g;
        S.rank[i] = (uint16_t)(base_g + __popc(peers & lanemask_lt()));
        if ((peers >> lane) == 1u) S.ccount[g] = base_g + __popc(peers);
      }
      __syncwarp();
    }
  }
  __syncthreads();

  // 3d. first child of each action; offsets within the action. Children are
  // numbered in item order and every action has exactly n items, so the
  // children of earlier actions hold al * n items in total.
  const int nchild = S.nchild;
  for (int g = tid; g < nchild; g += nthr) {
    int al = S.cfirst[g] / n;
    if (g == 0 || S.cfirst[g - 1] / n != al) S.abase[al] = g;
  }
  if (tid == 0) S.abase[a_count] = nchild;
  if (warp == 0) {
    int carry = 0;
    for (int c0 = 0; c0 < nchild; c0 += 32) {
      int g = c0 + lane;
      int cnt = g < nchild ? S.ccount[g] : 0;
      int v = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= d) v += o;
      }
      if (g < nchild) S.coff[g] = carry + v - cnt - (S.cfirst[g] / n) * n;
      carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
  __syncthreads();
  for (int i = tid; i < items; i += nthr) {
    int al = i / n;
    int g = S.gcid[i];
    S.permitem[al * n + S.coff[g] + S.rank[i]] = (uint16_t)i;
  }
  __syncthreads();

  // 4. bounds in child-grouped order, 5. fixed-point sums per child
  const uint32_t* hw = reinterpret_cast<const uint32_t*>(job.hist);
  for (int q = tid; q < items; q += nthr) {
    int i = S.permitem[q];
    int al = i / n;
    int a = a_first + al;
    int g = S.gcid[i];
    RSS s;
    s.pos[0] = S.next[0][i];
    s.pos[1] = S.next[1][i];
    s.good = S.next[2][i];
    s.sampled = S.next[3][i];
    s.scen = S.next[4][i];
    uint64_t key = S.key[i];
    float u = (depth + 1 >= M.D) ? M.tail(s) : M.upper(s);
    float v = 0.0f;
    if (M.terminal(s)) {
      u = 0.0f;
    } else {
      uint32_t h[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) h[k] = hw[k];
      uint32_t pm = positive_mask(h, M.m);
      M.observe(h, pm, a, key);
      v = M.rollout(s, h, pm, depth + 1, steps);
    }
    atomicAdd(&S.sr[g], (unsigned long long)to_fixed(S.rew[i]));
    atomicAdd(&S.su[g], (unsigned long long)to_fixed(u));
    atomicAdd(&S.sl[g], (unsigned long long)to_fixed(v));
  }
  __syncthreads();

  // results
  const int cap = job.child_cap;
  for (int al = warp; al < a_count; al += nthr / 32) {
    int g0 = S.abase[al], nc = S.abase[al + 1] - g0;
    int ao = a_begin + al;
    if (lane == 0) {
      job.child_count[ao] = nc;
      if (nc > cap) report(work, kStatusOverflow);
    }
    int ncw = nc < cap ? nc : cap;
    for (int c = lane; c <= ncw; c += 32) {
      size_t o = (size_t)ao * (cap + 1) + c;
      job.child_off[o] = c < nc ? S.coff[g0 + c] : n;
    }
    for (int c = lane; c < ncw; c += 32) {
      size_t o = (size_t)ao * cap + c;
      int g = g0 + c;
      job.child_key[o] = S.key[S.cfirst[g]];
      job.rew_sum[o] = (long long)S.sr[g];
      job.u_sum[o] = (long long)S.su[g];
      job.l_sum[o] = (long long)S.sl[g];
    }
  }
  for (int q = tid; q < items; q += nthr) {
    int al = q / n;
    int i = S.permitem[q];
    job.perm[(size_t)(a_begin + al) * n + (q - al * n)] = (uint16_t)(i - al * n);
  }
  __syncthreads();
}

template <int R>
__global__ void __launch_bounds__(256) rs_expand_kernel(const DevModel* __restrict__ gm, DevWork* work,
                                                        const dsp_leaf_job* __restrict__ jobs,
                                                        const int4* __restrict__ units, int n_units,
                                                        unsigned int* head, uint32_t plan_step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RSUnitSmem& S = *reinterpret_cast<RSUnitSmem*>(smem_raw);
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) S.c.G[k] = gm->G[k];
  for (int k = threadIdx.x; k < kMaxRocks; k += blockDim.x) S.c.rock_xy[k] = gm->rock_xy[k];
  for (int k = threadIdx.x; k < kMaxSide * kMaxSide; k += blockDim.x) S.c.cell_rock[k] = gm->cell_rock[k];
  RSModel<R> M;
  M.sh = &S.c;
  M.thresh = gm->thresh;
  M.n = gm->n;
  M.m = gm->m;
  M.per = gm->per_robot;
  M.D = gm->D;
  M.seed = gm->seed;
  M.plan_step = plan_step;
  unsigned long long steps = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) S.unit = (int)atomicAdd(head, 1u);
    __syncthreads();
    int u = S.unit;
    __syncthreads();
    if (u >= n_units) break;
    int4 un = units[u];
    if (threadIdx.x == 0) S.job = jobs[un.x];
    __syncthreads();
    rs_unit<R>(S, M, S.job, un.y, un.z, work, steps);
  }
  // block-wide sum of the scenario-step counter
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

// dsp_step: one g call per scenario.
template <int R>
__global__ void rs_step_kernel(const DevModel* __restrict__ gm, const uint32_t* in, int in_cap, int count,
                               const int32_t* actions, int depth, uint32_t* out, int out_cap, uint64_t* keys,
                               float* rewards, uint32_t plan_step) {
  __shared__ RSShared c;
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) c.G[k] = gm->G[k];
  for (int k = threadIdx.x; k < kMaxRocks; k += blockDim.x) c.rock_xy[k] = gm->rock_xy[k];
  for (int k = threadIdx.x; k < kMaxSide * kMaxSide; k += blockDim.x) c.cell_rock[k] = gm->cell_rock[k];
  __syncthreads();
  RSModel<R> M{&c, gm->thresh, gm->n, gm->m, gm->per_robot, gm->D, gm->seed, plan_step};
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
  for (int k = threadIdx.x; k < kGammaLen; k += blockDim.x) c.G[k] = gm->G[k];
  for (int k = threadIdx.x; k < kMaxRocks; k += blockDim.x) c.rock_xy[k] = gm->rock_xy[k];
  for (int k = threadIdx.x; k < kMaxSide * kMaxSide; k += blockDim.x) c.cell_rock[k] = gm->cell_rock[k];
  __syncthreads();
  RSModel<R> M{&c, gm->thresh, gm->n, gm->m, gm->per_robot, gm->D, gm->seed, plan_step};
  unsigned long long steps = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    RSS s = M.load(block, cap, i);
    uint32_t h[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      h[k] = hist ? *reinterpret_cast<const uint32_t*>(hist + 32 * (size_t)i + 4 * k) : 0u;
    uint32_t pm = positive_mask(h, M.m);
    value[i] = M.rollout(s, h, pm, start_depth, steps);
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_down_sync(0xFFFFFFFFu, steps, o);
  if ((threadIdx.x & 31) == 0 && steps) atomicAdd(&work->steps, steps);
}

}  // namespace

size_t rs_expand_smem() { return sizeof(RSUnitSmem); }

int rs_expand_blocks_per_sm(int robots, int block) {
  int n = 0;
  size_t smem = sizeof(RSUnitSmem);
  if (robots == 1) {
    cudaFuncSetAttribute(rs_expand_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rs_expand_kernel<1>, block, smem);
  } else {
    cudaFuncSetAttribute(rs_expand_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rs_expand_kernel<2>, block, smem);
  }
  return n > 0 ? n : 1;
}
int rs_items_per_unit() { return kItems; }

cudaError_t launch_rs_expand(const DevModel* gm, int robots, DevWork* work, const dsp_leaf_job* jobs,
                             const int4* units, int n_units, unsigned int* head, uint32_t plan_step, int grid,
                             int block, cudaStream_t st) {
  size_t smem = sizeof(RSUnitSmem);
  if (robots == 1) {
    cudaFuncSetAttribute(rs_expand_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rs_expand_kernel<1><<<grid, block, smem, st>>>(gm, work, jobs, units, n_units, head, plan_step);
  } else {
    cudaFuncSetAttribute(rs_expand_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    rs_expand_kernel<2><<<grid, block, smem, st>>>(gm, work, jobs, units, n_units, head, plan_step);
  }
  return cudaGetLastError();
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
