// kc_count_noalloc: the total k-clique count without any device allocation.
//
// Some callers cannot allocate device memory at the point where they count:
// callers that run under a fixed memory budget or behind a custom allocator
// that owns all of the device memory (a cudaMalloc from this library would
// fail or break the owner's accounting), and latency-critical paths that must
// not take the allocator's locks. kc_count allocates a small
// work block (and, for very large out-neighbourhoods, per-block slabs) on every
// call. This entry point takes that scratch from one statically sized device
// array instead.
//
// The array lives at file scope below, so every GPU that loads the library
// holds KC_NOALLOC_SCRATCH_BYTES of device memory until the process exits.
// Host code may not use the array's name as a device address (in host code it
// is only a stand-in symbol); its device address is looked up once per device
// with cudaGetSymbolAddress.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "kc_core.cuh"
#include "kc_dag.cuh"
#include "kc_host.cuh"
#include "kc_internal.cuh"
#include "kclique.h"

namespace {

// Work block (total, status word, three queue counters) in the first 256
// bytes, then the per-block slabs of roots whose matrix exceeds shared memory.
static __device__ __align__(256) uint8_t g_noalloc_scratch[KC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up on the
// first call for that device; make that first call before any stream capture).
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace


extern "C" kc_status kc_count_noalloc(const kc_dag *d, int k, uint64_t *h_total, kc_stream_t stream) {
  if (!d || !h_total || k < 1 || k > KC_KMAX) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (k == 1) {
    *h_total = d->n;
    return KC_OK;
  }
  if (k == 2) {
    *h_total = d->m;
    return KC_OK;
  }
  const uint32_t need = (uint32_t)(k - 1);
  if (need > d->max_out) {
    *h_total = 0;
    return KC_OK;
  }
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;

  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) return kc::cuda_fail(e);

  int dev = 0, optin = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return kc::cuda_fail(e);
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess)
    return kc::cuda_fail(e);
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return kc::cuda_fail(e);
  sms = std::max(1, sms);
  const size_t budget = (size_t)(optin > 4096 ? optin - 2048 : 48 * 1024);
  const uint32_t dcap = kc::block_root_capacity(budget, false, false);
  const uint32_t dsmem = std::min<uint32_t>(dcap, std::max<uint32_t>(d->max_out, kc::kLightMax + 1));
  const size_t block_smem = kc::block_root_smem(dsmem, false, false);
  int per_sm_b = 0, per_sm_w = 0;
  if ((e = kc::count_occupancy(false, false, block_smem, &per_sm_b, &per_sm_w)) != cudaSuccess)
    return kc::cuda_fail(e);
  const int block_grid = sms * std::max(1, per_sm_b);
  const int warp_grid = sms * std::max(1, per_sm_w);

  kc::CountArgs a;
  memset(&a, 0, sizeof a);
  a.ptr = d->ptr;
  a.col = d->col;
  a.order = d->order;
  a.k = k;
  auto ge = [&](uint64_t t) -> uint32_t { return t < d->ge.size() ? (uint32_t)d->ge[t] : 0u; };
  a.n_light_end = ge(need);
  a.n_big = ge(kc::kLightMax + 1);
  a.n_scratch = ge((uint64_t)dcap + 1);
  a.bulk_build = kc::bulk_build_enabled() ? 1u : 0u;
  const uint32_t ratio = kc::core_policy().ratio;
  if (d->core_bits && !a.bulk_build && ratio != 0xffffffffu) {  // the dense core is the DAG's own
    a.core_id = d->core_id;
    a.core_bits = (const unsigned long long *)d->core_bits;
    a.core_words = d->core_words;
    a.core_ratio = ratio;
  }
  uint8_t *b = (uint8_t *)base;
  a.total = (unsigned long long *)b;
  a.status = (unsigned *)(b + 8);
  a.queue = (unsigned *)(b + 16);
  if (a.n_scratch > 0) {
    const size_t slab = (kc::root_layout(d->max_out, false, false).bytes + 255) & ~(size_t)255;
    const size_t room = (size_t)KC_NOALLOC_SCRATCH_BYTES - 256;
    if (slab > room) return KC_ECAPACITY;  // one root's matrix does not fit the static scratch
    size_t nb = room / slab;
    nb = std::min<size_t>(nb, (size_t)block_grid);
    nb = std::min<size_t>(nb, (size_t)a.n_scratch);
    a.scratch = b + 256;
    a.scratch_stride = slab;
    a.scratch_blocks = (uint32_t)nb;
  }
  // the work block keeps the previous call's values: clear it first
  if ((e = cudaMemsetAsync(b, 0, 64, s)) != cudaSuccess) return kc::cuda_fail(e);
  if ((e = kc::launch_count(a, false, false, block_grid, warp_grid, block_smem, s)) != cudaSuccess)
    return kc::cuda_fail(e);
  unsigned long long h[2] = {0, 0};
  if ((e = cudaMemcpyAsync(h, b, sizeof h, cudaMemcpyDeviceToHost, s)) != cudaSuccess) return kc::cuda_fail(e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return kc::cuda_fail(e);
  const unsigned st = (unsigned)h[1];
  if (st & kc::ST_CAPACITY) return KC_ECAPACITY;
  if (st & kc::ST_OVERFLOW) return KC_ERANGE;
  if (st & kc::ST_TIMEOUT) return KC_ETIMEDOUT;
  *h_total = h[0];
  return KC_OK;
}
