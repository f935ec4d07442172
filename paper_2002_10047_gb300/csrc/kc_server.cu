// kc_server: a request loop that serves count and per-vertex count requests
// on device-resident oriented graphs with continuous batching.
//
// A dispatcher thread owns S slots (one CUDA stream each). Requests wait in
// a FIFO queue; the head is admitted as soon as a slot is free and its device
// footprint (per-vertex output, work block, global scratch of its largest
// roots) fits the memory budget beside the requests already in flight, so
// requests that arrive while others run join them on the GPU and their
// kernels overlap. Each admitted request gets grids sized to its own work
// and capped at a share of the GPU, so that one large request does not hold
// every SM while small ones wait.
// Completion is signalled by a host function enqueued after the request's
// copy-back, which only sets a flag and wakes the dispatcher (it takes no
// lock that is held across CUDA calls).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kc_host.cuh"
#include "kc_orient.cuh"

namespace {

// The device's globaltimer, to map host deadlines onto the clock the
// counting kernels check (calibrated once per server).
__global__ void read_globaltimer_kernel(unsigned long long *out) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t;
}

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t id = 0;
  const kc_dag *d = nullptr;
  int k = 0;
  bool pv = false;
  uint64_t t_submit = 0, t_admit = 0, t_done = 0;
  uint64_t timeout_us = 0;
  int status = KC_OK;
  uint64_t total = 0;
  uint64_t footprint = 0;  // bytes held against the budget until release (pv) or completion
  uint64_t held = 0;       // part of footprint still held after completion (the per-vertex output)
  unsigned long long *d_pv = nullptr;
  void *scratch = nullptr;
  int slot = -1;
  bool done = false;
  kc::LaunchPlan plan;
};

struct Slot {
  cudaStream_t stream = nullptr;
  uint8_t *work = nullptr;                  // device: total, status, queues
  unsigned long long *mirror = nullptr;     // pinned host copy of total and status
  std::atomic<int> finished{0};
  uint64_t req = 0;
  bool busy = false;
};

}  // namespace

struct kc_server {
  kc_server_config cfg{};
  int device = 0;
  std::mutex mu;                    // request table, queue, slots, budget
  std::condition_variable cv_done;  // clients waiting for a request
  std::mutex wake_mu;               // dispatcher wake-ups (never held across CUDA calls)
  std::condition_variable cv_wake;
  uint64_t wakeups = 0;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::vector<Slot> slots;
  uint64_t next_id = 1;
  uint64_t in_use = 0;  // bytes admitted and not yet returned
  int64_t gpu_minus_host = 0;  // globaltimer - steady_clock, ns
  bool stop = false;
  kc_server_stats st{};
  std::thread th;

  void wake() {
    {
      std::lock_guard<std::mutex> lk(wake_mu);
      ++wakeups;
    }
    cv_wake.notify_one();
  }
  void run();
  void admit(Request &r, int si);
  void finish(Request &r, Slot &s, int status);
};

namespace {

struct CbArg {
  kc_server *srv;
  int slot;
};

void CUDART_CB on_done(void *p) {
  CbArg *a = (CbArg *)p;
  a->srv->slots[a->slot].finished.store(1, std::memory_order_release);
  a->srv->wake();
  delete a;
}

}  // namespace

void kc_server::finish(Request &r, Slot &s, int status) {
  r.status = status;
  r.t_done = now_ns();
  r.done = true;
  if (r.scratch) cudaFreeAsync(r.scratch, s.stream);
  r.scratch = nullptr;
  in_use -= r.footprint - r.held;  // the per-vertex output stays until release
  r.footprint = r.held;
  s.busy = false;
  st.completed++;
}

// Enqueue one admitted request on slot si (called with mu held; only
// asynchronous CUDA calls).
void kc_server::admit(Request &r, int si) {
  Slot &s = slots[si];
  r.slot = si;
  r.t_admit = now_ns();
  s.busy = true;
  s.req = r.id;
  s.finished.store(0, std::memory_order_relaxed);
  in_use += r.footprint;
  st.admitted++;
  cudaError_t e = cudaSuccess;
  kc::CountArgs a = r.plan.a;
  const uint32_t n = r.d->n;
  if (r.pv) {
    e = kc::dev_malloc_async((void **)&r.d_pv, sizeof(unsigned long long) * std::max<uint32_t>(n, 1), s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(r.d_pv, 0, sizeof(unsigned long long) * n, s.stream);
  }
  if (e == cudaSuccess && r.plan.scratch_bytes) e = kc::dev_malloc_async(&r.scratch, r.plan.scratch_bytes, s.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s.work, 0, kc::kc_work_bytes(), s.stream);
  if (e == cudaSuccess && r.plan.a.n_light_end > 0) {
    kc::set_work(&a, s.work);
    a.pv = r.d_pv;
    if (r.timeout_us) a.deadline_ns = (uint64_t)((int64_t)(r.t_submit + r.timeout_us * 1000ull) + gpu_minus_host);
    a.scratch = (uint8_t *)r.scratch;
    // grids sized to the request (a block per block root, a warp per four
    // warp roots) and capped at its share of the GPU's resident blocks
    const uint32_t nwr = a.n_light_end - a.n_big;
    const uint32_t pct = cfg.grid_share_pct ? std::min<uint32_t>(cfg.grid_share_pct, 100u) : 100u;
    const uint64_t bcap = std::max<uint64_t>(1, (uint64_t)r.plan.block_grid * pct / 100);
    const uint64_t wcap = std::max<uint64_t>(1, (uint64_t)r.plan.warp_grid * pct / 100);
    int bg = (int)std::min<uint64_t>(bcap, a.n_big);
    int wg = (int)std::min<uint64_t>(wcap, ((uint64_t)nwr + 4 * 8 - 1) / (4 * 8));
    a.scratch_blocks = std::min<uint32_t>(a.scratch_blocks, (uint32_t)std::max(bg, 1));
    e = kc::launch_count(a, r.pv, false, std::max(bg, 1), std::max(wg, 1), r.plan.block_smem, s.stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.mirror, s.work, 16, cudaMemcpyDeviceToHost, s.stream);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s.stream, on_done, new CbArg{this, si});
  if (e != cudaSuccess) {
    kc::cuda_fail(e);
    cudaStreamSynchronize(s.stream);  // nothing of ours is left in flight on this slot
    finish(r, s, KC_ECUDA);
    cv_done.notify_all();
  }
}

void kc_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (!stop) {
    // completions
    bool any = false;
    for (size_t i = 0; i < slots.size(); ++i) {
      Slot &s = slots[i];
      if (!s.busy || !s.finished.load(std::memory_order_acquire)) continue;
      auto it = reqs.find(s.req);
      Request &r = it->second;
      r.total = s.mirror[0];
      finish(r, s, kc::status_code((unsigned)s.mirror[1]));
      any = true;
    }
    if (any) cv_done.notify_all();
    // admissions, first come first served: the head waits for a slot and for
    // budget room (admitted alone if nothing else is in flight)
    while (!queue.empty()) {
      int si = -1;
      for (size_t i = 0; i < slots.size(); ++i)
        if (!slots[i].busy) {
          si = (int)i;
          break;
        }
      if (si < 0) break;
      Request &r = reqs[queue.front()];
      bool alone = true;  // nothing running (outputs held for the client do not block admission)
      for (auto &sl : slots) alone = alone && !sl.busy;
      if (!alone && in_use + r.footprint > cfg.hbm_budget) break;
      queue.pop_front();
      admit(r, si);
      uint32_t inflight = 0;
      for (auto &s : slots) inflight += s.busy ? 1u : 0u;
      st.peak_in_flight = std::max<uint64_t>(st.peak_in_flight, inflight);
      st.peak_bytes = std::max<uint64_t>(st.peak_bytes, in_use);
    }
    // sleep until a completion or a submission
    lk.unlock();
    {
      std::unique_lock<std::mutex> wl(wake_mu);
      cv_wake.wait_for(wl, std::chrono::milliseconds(5), [&] { return wakeups > 0; });
      wakeups = 0;
    }
    lk.lock();
  }
}

extern "C" {

kc_status kc_server_create(const kc_server_config *cfg, kc_server **out) {
  if (!cfg || !out || cfg->slots == 0 || cfg->slots > 64) return KC_EINVAL;
  kc_server *s = new kc_server;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  s->slots = std::vector<Slot>(cfg->slots);
  cudaError_t e = cudaSuccess;
  for (auto &sl : s->slots) {
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void **)&sl.work, kc::kc_work_bytes());
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sl.mirror, 16);
  }
  if (e == cudaSuccess) {
    // clock offset: a globaltimer read bracketed by host reads, the tightest
    // bracket of a few tries (the first launch also loads the module)
    unsigned long long *d_t = nullptr, h_t = 0;
    e = cudaMalloc((void **)&d_t, 8);
    uint64_t best = ~0ull;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) {
      const uint64_t t0 = now_ns();
      read_globaltimer_kernel<<<1, 1, 0, s->slots[0].stream>>>(d_t);
      kc::note_launch();
      e = cudaMemcpyAsync(&h_t, d_t, 8, cudaMemcpyDeviceToHost, s->slots[0].stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->slots[0].stream);
      const uint64_t t1 = now_ns();
      if (e == cudaSuccess && t1 - t0 < best) {
        best = t1 - t0;
        s->gpu_minus_host = (int64_t)h_t - (int64_t)((t0 + t1) / 2);
      }
    }
    if (d_t) cudaFree(d_t);
  }
  if (e != cudaSuccess) {
    kc_server_destroy(s);
    return kc::cuda_fail(e);
  }
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return KC_OK;
}

kc_status kc_server_submit(kc_server *s, const kc_dag *d, int k, int per_vertex, uint64_t timeout_us,
                           uint64_t *req_id) {
  if (!s || !d || !req_id || k < 3 || k > KC_KMAX) return KC_EINVAL;
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;
  Request r;
  r.d = d;
  r.k = k;
  r.pv = per_vertex != 0;
  r.t_submit = now_ns();
  r.timeout_us = timeout_us;
  if ((uint32_t)(k - 1) <= d->max_out) {
    cudaError_t e = kc::plan_count(d, k, r.pv, false, nullptr, &r.plan);
    if (e != cudaSuccess) return kc::cuda_fail(e);
  } else {
    memset(&r.plan, 0, sizeof r.plan);  // no root can hold a k-clique: nothing to launch
  }
  r.held = r.pv ? sizeof(unsigned long long) * (uint64_t)std::max<uint32_t>(d->n, 1) : 0;
  r.footprint = r.held + r.plan.scratch_bytes + kc::kc_work_bytes();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return KC_EINVAL;
    r.id = s->next_id++;
    *req_id = r.id;
    s->reqs.emplace(r.id, r);
    s->queue.push_back(r.id);
    s->st.submitted++;
  }
  s->wake();
  return KC_OK;
}

kc_status kc_server_wait(kc_server *s, uint64_t req_id, int timeout_ms, kc_request_result *out) {
  if (!s || !out) return KC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(req_id);
  if (it == s->reqs.end()) return KC_EINVAL;
  auto pred = [&] { return s->reqs[req_id].done; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, pred);
  } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    return KC_ETIMEDOUT;
  }
  const Request &r = s->reqs[req_id];
  out->status = r.status;
  out->total = r.total;
  out->queue_ns = r.t_admit - r.t_submit;
  out->run_ns = r.t_done - r.t_admit;
  out->latency_ns = r.t_done - r.t_submit;
  out->slot = r.slot;
  if (!r.pv) s->reqs.erase(req_id);  // nothing left to fetch
  return KC_OK;
}

kc_status kc_server_fetch_per_vertex(kc_server *s, uint64_t req_id, uint64_t *dst, kc_stream_t stream) {
  if (!s || !dst) return KC_EINVAL;
  unsigned long long *src = nullptr;
  size_t bytes = 0;
  cudaStream_t slot_stream = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || !it->second.done || !it->second.pv || !it->second.d_pv) return KC_EINVAL;
    src = it->second.d_pv;
    bytes = sizeof(unsigned long long) * it->second.d->n;
    slot_stream = s->slots[it->second.slot].stream;
  }
  cudaStream_t cs = (cudaStream_t)stream;
  cudaEvent_t ev;
  KC_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  cudaEventRecord(ev, slot_stream);  // the output was written on the slot's stream
  cudaStreamWaitEvent(cs, ev, 0);
  cudaEventDestroy(ev);
  if (bytes) KC_CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, cs));
  KC_CK(cudaStreamSynchronize(cs));
  return KC_OK;
}

kc_status kc_server_release(kc_server *s, uint64_t req_id) {
  if (!s) return KC_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end() || !it->second.done) return KC_EINVAL;
    Request &r = it->second;
    if (r.d_pv) cudaFreeAsync(r.d_pv, s->slots[r.slot].stream);
    s->in_use -= r.footprint;
    s->reqs.erase(it);
  }
  s->wake();  // room in the budget
  return KC_OK;
}

kc_status kc_server_get_stats(kc_server *s, kc_server_stats *out) {
  if (!s || !out) return KC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->bytes_in_use = s->in_use;
  out->queued = s->queue.size();
  return KC_OK;
}

void kc_server_destroy(kc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->wake();
  if (s->th.joinable()) s->th.join();
  for (auto &sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  for (auto &kv : s->reqs) {
    Request &r = kv.second;
    cudaStream_t st = r.slot >= 0 ? s->slots[r.slot].stream : nullptr;
    if (r.d_pv) cudaFreeAsync(r.d_pv, st);
    if (r.scratch) cudaFreeAsync(r.scratch, st);
  }
  for (auto &sl : s->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    if (sl.work) cudaFree(sl.work);
    if (sl.mirror) cudaFreeHost(sl.mirror);
    if (sl.stream) cudaStreamDestroy(sl.stream);
  }
  delete s;
}

}  // extern "C"
