// Device job queue of leaf expansions (host side). Many search threads submit
// leaf jobs of uneven |Phi_b| into a ring in mapped pinned host memory; one
// persistent kernel of the model's kind (rs_queue_kernel, car_queue_kernel,
// nav_queue_kernel), launched from a CUDA graph, pulls them (node-level
// parallelism of Sec. III-D with the per-leaf launches replaced by one
// resident kernel). A monitor thread relaunches the kernel whenever jobs are
// pending and it has exited after idling; every wait, on the host and on the
// device, is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "kernels.cuh"
#include "model.hpp"

struct dsp_queue {
  dsp_model* m = nullptr;
  int cap = 0;
  // mapped pinned host memory: seq[cap], done[cap], jobs[cap], plan_step[cap], close flag
  unsigned char* host = nullptr;
  unsigned long long* seq = nullptr;
  unsigned long long* done = nullptr;
  dsp_leaf_job* jobs = nullptr;
  unsigned int* plan_step = nullptr;
  unsigned int* close = nullptr;
  dsp::QueueRing ring{};
  unsigned long long* d_head = nullptr;  // device: next ticket to consume
  uint32_t* d_scratch = nullptr;         // device: one rollout-item list per ring slot
  dsp_leaf_job* d_jcopy = nullptr;       // device: one job copy per ring slot
  dsp::QueueShare* d_share = nullptr;    // device: work sharing per ring slot
  unsigned long long* d_finished = nullptr;  // device: jobs completed
  size_t slot_words = 0;                 // per-slot rollout items (Rock Sample, navigation)
  size_t scratch_words = 0;              // all of d_scratch
  int grid = 0;
  unsigned long long idle_ns = 0;
  cudaStream_t stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  std::atomic<unsigned long long> tail{0};  // next ticket to hand out
  std::atomic<unsigned long long> launches{0};
  std::atomic<unsigned long long> consumed{0};
  std::mutex mu;
  std::condition_variable cv;
  bool shutdown = false;
  std::atomic<int> monitor_status{DSP_OK};
  std::thread monitor;
};

namespace dsp {
namespace {

dsp_status build_graph(dsp_queue* q) {
  if (q->graph) {
    cudaGraphExecDestroy(q->graph);
    q->graph = nullptr;
  }
  cudaGraph_t g;
  cudaError_t e = cudaStreamBeginCapture(q->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_queue: begin capture");
  cudaError_t el;
  const int kind = q->m->host->kind;
  if (kind == DSP_MODEL_CAR)
    el = launch_car_queue(q->m, q->ring, q->d_head, q->d_scratch, q->d_jcopy, q->idle_ns, q->grid, q->stream);
  else if (kind == DSP_MODEL_NAV)
    el = launch_nav_queue(q->m, q->ring, q->d_head, q->d_scratch, q->slot_words, q->d_jcopy, q->idle_ns, q->grid,
                          q->stream);
  else
    el = launch_rs_queue(q->m->dmodel, q->m->host->robots, rs_key_words(q->m->host), q->m->dwork, q->ring,
                         q->d_head, q->d_scratch, q->slot_words, q->d_jcopy, q->idle_ns, q->grid, q->stream);
  e = cudaStreamEndCapture(q->stream, &g);
  if (el != cudaSuccess) return cuda_fail(el, "dsp_queue: capture launch");
  if (e != cudaSuccess) return cuda_fail(e, "dsp_queue: end capture");
  e = cudaGraphInstantiate(&q->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(e, "dsp_queue: instantiate");
  return DSP_OK;
}

// Launches the persistent kernel while jobs are pending; the kernel exits by
// itself after idle_ns without a job.
void monitor_loop(dsp_queue* q) {
  cudaSetDevice(q->m->device);
  while (true) {
    {
      std::unique_lock<std::mutex> lock(q->mu);
      q->cv.wait(lock, [&] { return q->shutdown || q->tail.load() > q->consumed.load(); });
      if (q->shutdown && q->tail.load() <= q->consumed.load()) break;
    }
    dsp_status s = DSP_OK;
    if (q->graph == nullptr) s = build_graph(q);
    cudaError_t e = cudaSuccess;
    if (s == DSP_OK) e = cudaGraphLaunch(q->graph, q->stream);
    if (s == DSP_OK && e == cudaSuccess) q->launches += 1;
    if (s == DSP_OK && e == cudaSuccess) e = cudaStreamSynchronize(q->stream);
    unsigned long long h = 0;
    if (s == DSP_OK && e == cudaSuccess) e = cudaMemcpy(&h, q->d_head, sizeof(h), cudaMemcpyDeviceToHost);
    if (s != DSP_OK || e != cudaSuccess) {
      std::lock_guard<std::mutex> lock(q->mu);
      q->monitor_status = (int)(s != DSP_OK ? s : cuda_fail(e, "dsp_queue: persistent kernel"));
      q->shutdown = true;
      break;
    }
    q->consumed = h;
    if (q->shutdown && q->tail.load() <= h) break;
  }
}

}  // namespace
}  // namespace dsp

using namespace dsp;

extern "C" {

dsp_status dsp_queue_create(dsp_model* m, int32_t capacity, uint64_t idle_ns, dsp_queue** out) {
  if (!m || !out) return fail(DSP_E_INVALID, "dsp_queue_create: NULL argument");
  *out = nullptr;
  if (capacity < 1 || capacity > (1 << 20)) return fail(DSP_E_INVALID, "dsp_queue_create: capacity %d", capacity);
  if (idle_ns == 0) idle_ns = 2000000ull;
  dsp_queue* q = new dsp_queue();
  q->m = m;
  q->cap = capacity;
  q->idle_ns = idle_ns;
  size_t bytes = sizeof(unsigned long long) * 2 * (size_t)capacity + sizeof(dsp_leaf_job) * (size_t)capacity +
                 sizeof(unsigned int) * (size_t)capacity + 256;
  cudaError_t e = cudaHostAlloc((void**)&q->host, bytes, cudaHostAllocMapped | cudaHostAllocPortable);
  if (e != cudaSuccess) {
    delete q;
    return cuda_fail(e, "dsp_queue_create: ring");
  }
  std::memset(q->host, 0, bytes);
  q->seq = (unsigned long long*)q->host;
  q->done = q->seq + capacity;
  q->jobs = (dsp_leaf_job*)(q->done + capacity);
  q->plan_step = (unsigned int*)(q->jobs + capacity);
  q->close = q->plan_step + capacity;
  for (int i = 0; i < capacity; ++i) q->seq[i] = (unsigned long long)i;  // slot i takes ticket i first
  void* dp = nullptr;
  e = cudaHostGetDevicePointer(&dp, q->host, 0);
  if (e == cudaSuccess) {
    unsigned char* d = (unsigned char*)dp;
    q->ring.seq = (unsigned long long*)d;
    q->ring.done = q->ring.seq + capacity;
    q->ring.jobs = (dsp_leaf_job*)(q->ring.done + capacity);
    q->ring.plan_step = (unsigned int*)(q->ring.jobs + capacity);
    q->ring.close = q->ring.plan_step + capacity;
    q->ring.cap = capacity;
    // the kernel's CTAs per SM (its shared-memory limit is set here, before
    // any capture) and its scratch: per ring slot (Rock Sample, navigation:
    // one job's rollout items) or per CTA (car: one observation scratch)
    size_t scratch_words = 0;
    int per_sm = 1;
    if (m->host->kind == DSP_MODEL_CAR) {
      e = car_queue_setup(m, &per_sm);
      q->grid = std::max(1, per_sm) * m->num_sms;
      scratch_words = car_queue_scratch_words(q->grid);
    } else if (m->host->kind == DSP_MODEL_NAV) {
      e = nav_queue_setup(&per_sm);
      q->grid = std::max(1, per_sm) * m->num_sms;
      q->slot_words = nav_queue_slot_words(m);
      scratch_words = q->slot_words * (size_t)capacity;
    } else {
      q->grid = rs_queue_blocks_per_sm(m->host->robots, rs_key_words(m->host)) * m->num_sms;
      q->slot_words = rs_queue_slot_words(m->host->robots, m->host->num_actions);
      scratch_words = q->slot_words * (size_t)capacity;
    }
    q->scratch_words = scratch_words;
    if (e == cudaSuccess) e = cudaMalloc(&q->d_head, sizeof(unsigned long long));
  }
  if (e == cudaSuccess) e = cudaMemset(q->d_head, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&q->d_finished, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(q->d_finished, 0, sizeof(unsigned long long));
  q->ring.finished = q->d_finished;
  if (e == cudaSuccess) e = cudaMalloc(&q->d_scratch, sizeof(uint32_t) * q->scratch_words);
  if (e == cudaSuccess) e = cudaMalloc(&q->d_jcopy, sizeof(dsp_leaf_job) * (size_t)capacity);
  if (e == cudaSuccess) e = cudaMalloc(&q->d_share, sizeof(dsp::QueueShare) * (size_t)capacity);
  if (e == cudaSuccess) {
    std::vector<dsp::QueueShare> init(capacity);
    for (dsp::QueueShare& sh : init) {
      sh.claim = 0ull;  // closed (no chunks)
      sh.ticket = 0;
      sh.nchunks = 0;
      sh.remaining = 0;
      sh.grain = 1;
      sh.plan_step = 0;
    }
    e = cudaMemcpy(q->d_share, init.data(), sizeof(dsp::QueueShare) * (size_t)capacity, cudaMemcpyHostToDevice);
    q->ring.share = q->d_share;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    dsp_status st = cuda_fail(e, "dsp_queue_create");
    dsp_queue_destroy(q);
    return st;
  }
  q->monitor = std::thread(monitor_loop, q);
  *out = q;
  return DSP_OK;
}

dsp_status dsp_queue_submit(dsp_queue* q, const dsp_leaf_job* job, uint64_t timeout_ns, uint64_t* ticket) {
  if (!q || !job || !ticket) return fail(DSP_E_INVALID, "dsp_queue_submit: NULL argument");
  {
    std::lock_guard<std::mutex> lock(q->mu);
    if (q->shutdown)
      return q->monitor_status != DSP_OK ? (dsp_status)q->monitor_status.load() : fail(DSP_E_INVALID, "queue closed");
  }
  if (q->m->policy_on) return fail(DSP_E_UNSUPPORTED, "dsp_queue_submit: the queue rolls out the heuristic policy");
  ExpandPlan plan;
  if (job->n_scen > kMaxScen)
    return fail(DSP_E_UNSUPPORTED, "dsp_queue_submit: n_scen=%d above %d", job->n_scen, kMaxScen);
  dsp_status vs = plan_units(q->m, job, 1, plan);  // validation only
  if (vs != DSP_OK) return vs;
  // Claim ticket t only once its slot is free (the consumer of ticket t - cap
  // has taken its job), so a full queue times out without holding a ticket.
  auto t0 = std::chrono::steady_clock::now();
  unsigned long long t = 0;
  int slot = 0;
  while (true) {
    t = q->tail.load(std::memory_order_acquire);
    slot = (int)(t % (unsigned long long)q->cap);
    unsigned long long s = __atomic_load_n(&q->seq[slot], __ATOMIC_ACQUIRE);
    if (s == t) {
      if (q->tail.compare_exchange_weak(t, t + 1, std::memory_order_acq_rel)) break;
      continue;
    }
    if (s > t) continue;  // another producer took ticket t
    double ns = std::chrono::duration<double, std::nano>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ns > 0 && ns > (double)timeout_ns)
      return fail(DSP_E_QUEUE_FULL, "dsp_queue_submit: no free slot within %llu ns",
                  (unsigned long long)timeout_ns);
    std::this_thread::yield();
  }
  q->jobs[slot] = *job;
  q->plan_step[slot] = q->m->plan_step;  // the job's random streams: the model's plan step at submission
  __atomic_store_n(&q->seq[slot], t + 1, __ATOMIC_RELEASE);
  { std::lock_guard<std::mutex> lock(q->mu); }  // the monitor cannot miss this wake-up
  q->cv.notify_all();
  *ticket = t;
  return DSP_OK;
}

dsp_status dsp_queue_wait(dsp_queue* q, uint64_t ticket, uint64_t timeout_ns) {
  if (!q) return fail(DSP_E_INVALID, "dsp_queue_wait: queue is NULL");
  if (ticket >= q->tail.load()) return fail(DSP_E_INVALID, "dsp_queue_wait: ticket %llu was never issued",
                                            (unsigned long long)ticket);
  const int slot = (int)(ticket % (unsigned long long)q->cap);
  auto t0 = std::chrono::steady_clock::now();
  while (__atomic_load_n(&q->done[slot], __ATOMIC_ACQUIRE) < ticket + 1) {
    if (q->monitor_status.load() != DSP_OK) return (dsp_status)q->monitor_status.load();
    double ns = std::chrono::duration<double, std::nano>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_ns > 0 && ns > (double)timeout_ns)
      return fail(DSP_E_TIMEOUT, "dsp_queue_wait: ticket %llu not done within %llu ns", (unsigned long long)ticket,
                  (unsigned long long)timeout_ns);
    std::this_thread::yield();
  }
  return DSP_OK;
}

dsp_status dsp_queue_stats(dsp_queue* q, uint64_t* launches, uint64_t* submitted) {
  if (!q) return fail(DSP_E_INVALID, "dsp_queue_stats: queue is NULL");
  if (launches) *launches = q->launches.load();
  if (submitted) *submitted = q->tail.load();
  return DSP_OK;
}

void dsp_queue_destroy(dsp_queue* q) {
  if (!q) return;
  if (q->monitor.joinable()) {
    {
      std::lock_guard<std::mutex> lock(q->mu);
      q->shutdown = true;
    }
    if (q->close) __atomic_store_n(q->close, 1u, __ATOMIC_RELEASE);
    q->cv.notify_all();
    q->monitor.join();
  }
  if (q->stream) cudaStreamSynchronize(q->stream);
  if (q->graph) cudaGraphExecDestroy(q->graph);
  if (q->stream) cudaStreamDestroy(q->stream);
  if (q->d_head) cudaFree(q->d_head);
  if (q->d_scratch) cudaFree(q->d_scratch);
  if (q->d_jcopy) cudaFree(q->d_jcopy);
  if (q->d_share) cudaFree(q->d_share);
  if (q->d_finished) cudaFree(q->d_finished);
  if (q->host) cudaFreeHost(q->host);
  delete q;
}

}  // extern "C"
