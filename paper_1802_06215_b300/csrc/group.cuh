// Stable grouping of one action's scenarios by observation key inside a CTA
// (Eq. newnodes): children in order of the first position holding their key,
// members in position order. Shared-memory open-addressing hash of the keys
// (atomicCAS insert, atomicMin first position), warp ballots to number the
// first occurrences, __match_any_sync for ranks within a child.
#pragma once
#include "common.cuh"

namespace dsp {

constexpr int kGroupTable = 2 * kMaxScen;
constexpr uint64_t kGroupEmpty = ~0ull;

struct GroupSmem {
  uint64_t tkey[kGroupTable];
  uint32_t tfirst[kGroupTable];
  uint16_t tcid[kGroupTable];
  uint16_t slot[kMaxScen];
  uint16_t gcid[kMaxScen];   // child of each position
  uint16_t rank[kMaxScen];   // rank of each position inside its child
  int32_t cfirst[kMaxScen];  // first position of each child
  int32_t ccount[kMaxScen];
  int32_t coff[kMaxScen];    // offset of each child in the grouped order
  int nchild;
};

__device__ __forceinline__ uint32_t lane_lt_mask() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Groups keys[0..n) (keys never equal kGroupEmpty: bit 63 is always clear).
// All threads of the CTA call it; it ends with a barrier.
__device__ __forceinline__ void group_by_key(GroupSmem& G, const uint64_t* keys, int n) {
  const int tid = threadIdx.x, nthr = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < kGroupTable; t += nthr) {
    G.tkey[t] = kGroupEmpty;
    G.tfirst[t] = 0xFFFFFFFFu;
  }
  __syncthreads();
  for (int p = tid; p < n; p += nthr) {
    uint64_t k = keys[p];
    uint32_t h = (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 40) & (kGroupTable - 1);
    while (true) {
      unsigned long long prev =
          atomicCAS((unsigned long long*)&G.tkey[h], (unsigned long long)kGroupEmpty, (unsigned long long)k);
      if (prev == kGroupEmpty || prev == k) break;
      h = (h + 1) & (kGroupTable - 1);
    }
    atomicMin(&G.tfirst[h], (uint32_t)p);
    G.slot[p] = (uint16_t)h;
  }
  __syncthreads();
  if (warp == 0) {
    int base = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
      int p = c0 + lane;
      bool lead = p < n && G.tfirst[G.slot[p]] == (uint32_t)p;
      uint32_t bal = __ballot_sync(0xFFFFFFFFu, lead);
      if (lead) {
        int g = base + __popc(bal & lane_lt_mask());
        G.tcid[G.slot[p]] = (uint16_t)g;
        G.cfirst[g] = p;
        G.ccount[g] = 0;
      }
      base += __popc(bal);
    }
    if (lane == 0) G.nchild = base;
    __syncwarp();
    for (int c0 = 0; c0 < n; c0 += 32) {
      int p = c0 + lane;
      bool ok = p < n;
      int g = ok ? G.tcid[G.slot[p]] : -1 - lane;
      uint32_t peers = __match_any_sync(0xFFFFFFFFu, g);
      int bg = ok ? G.ccount[g] : 0;
      __syncwarp();
      if (ok) {
        G.gcid[p] = (uint16_t)g;
        G.rank[p] = (uint16_t)(bg + __popc(peers & lane_lt_mask()));
        if ((peers >> lane) == 1u) G.ccount[g] = bg + __popc(peers);
      }
      __syncwarp();
    }
    __syncwarp();
    int carry = 0;
    const int nc = G.nchild;
    for (int c0 = 0; c0 < nc; c0 += 32) {
      int g = c0 + lane;
      int cnt = g < nc ? G.ccount[g] : 0;
      int v = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int o = __shfl_up_sync(0xFFFFFFFFu, v, d);
        if (lane >= d) v += o;
      }
      if (g < nc) G.coff[g] = carry + v - cnt;
      carry += __shfl_sync(0xFFFFFFFFu, v, 31);
    }
  }
  __syncthreads();
}

}  // namespace dsp
