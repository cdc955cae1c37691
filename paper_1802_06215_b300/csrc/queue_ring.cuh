// Device side of the leaf-job ring shared by the persistent queue kernels of
// the car and of navigation (the Rock Sample kernel adds work sharing across
// CTAs on top of the same protocol). Ticket t lives in slot t % cap of a ring
// in mapped pinned host memory: seq = t + 1 once the job is published, seq =
// t + cap once the slot may take ticket t + cap; done = t + 1 once the job's
// results are written. A CTA claims the next ticket only after its job is
// published, so no ticket is ever held without a job.
#pragma once
#include "kernels.cuh"

namespace dsp {
namespace qring {

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Warp 0 of a CTA (all its lanes): claims the next published ticket, if any
// (no waiting), and copies its descriptor from host memory into `dst` (shared
// memory) and the slot's device copy, and its plan step. Returns the ticket
// or -1 in every lane.
__device__ __forceinline__ long long take_job(const QueueRing& ring, unsigned long long* head, dsp_leaf_job* dst,
                                              dsp_leaf_job* jcopy, unsigned int* plan_step) {
  const int lane = threadIdx.x & 31;
  long long ticket = -1;
  if (lane == 0) {
    const unsigned long long h = *(volatile unsigned long long*)head;
    if (ld_acquire_sys(ring.seq + (h % ring.cap)) == h + 1 && atomicCAS(head, h, h + 1) == h) ticket = (long long)h;
  }
  __syncwarp();
  ticket = __shfl_sync(0xFFFFFFFFu, ticket, 0);
  if (ticket >= 0) {
    constexpr int kWords = (int)(sizeof(dsp_leaf_job) / 4);
    const int slot = (int)(ticket % ring.cap);
    const volatile uint32_t* src = (const volatile uint32_t*)(ring.jobs + slot);
    uint32_t* d = (uint32_t*)dst;
    uint32_t* c = (uint32_t*)(jcopy + slot);
    for (int w = lane; w < kWords; w += 32) {
      const uint32_t x = src[w];
      d[w] = x;
      c[w] = x;
    }
    if (lane == 0) *plan_step = *(volatile unsigned int*)(ring.plan_step + slot);
  }
  return ticket;
}

// One thread, after the whole CTA finished the job and fenced its results:
// counts it finished, publishes done and frees the slot for ticket + cap.
__device__ __forceinline__ void finish_job(const QueueRing& ring, unsigned long long ticket) {
  const int slot = (int)(ticket % (unsigned long long)ring.cap);
  atomicAdd(ring.finished, 1ull);
  __threadfence_system();
  st_release_sys(ring.done + slot, ticket + 1);
  st_release_sys(ring.seq + slot, ticket + (unsigned long long)ring.cap);
}

// Idle handling of a CTA without work (thread 0): sleeps with a backoff that
// doubles from 256 ns to 16 us, and decides to exit after idle_ns without a
// job or once the ring is closed. CTAs of these kernels share no work, so one
// may leave while others still run jobs.
__device__ __forceinline__ bool idle_exit(const QueueRing& ring, bool busy, unsigned long long& last_work,
                                          unsigned int& backoff, unsigned long long idle_ns) {
  const unsigned long long t = now_ns();
  if (busy) {
    last_work = t;
    backoff = 256;
    return false;
  }
  if (*(volatile unsigned int*)ring.close != 0u || t - last_work > idle_ns) return true;
  __nanosleep(backoff);
  backoff = min(backoff * 2u, 16384u);
  return false;
}

}  // namespace qring
}  // namespace dsp
