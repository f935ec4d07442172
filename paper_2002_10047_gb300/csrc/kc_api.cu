// The C ABI of libkclique.so (declared in include/kclique.h): argument
// checks, device allocation (stream-ordered), launch orchestration and the
// mapping of device status words to kc_status codes.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "kc_dag.cuh"
#include "kc_internal.cuh"
#include "kc_orient.cuh"
#include "kclique.h"


#include <atomic>

#include "kc_core.cuh"
#include "kc_host.cuh"

namespace kc {
static std::atomic<unsigned long long> g_launches{0};
void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static std::atomic<int> g_bulk_build{0};
bool bulk_build_enabled() { return g_bulk_build.load(std::memory_order_relaxed) != 0; }

// allocations left before the injected failures start; negative: none injected
static std::atomic<long long> g_alloc_budget{-1};

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s) {
  long long b = g_alloc_budget.load(std::memory_order_relaxed);
  while (b >= 0) {
    if (b == 0) {
      *p = nullptr;
      return cudaErrorMemoryAllocation;
    }
    if (g_alloc_budget.compare_exchange_weak(b, b - 1, std::memory_order_relaxed)) break;
  }
  return cudaMallocAsync(p, bytes, s);
}

namespace {
thread_local std::string g_cuda_err;
}

kc_status cuda_fail(cudaError_t e) {
  g_cuda_err = cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return KC_ENOMEM;
  return KC_ECUDA;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

kc_status internal_fail(const char *what) {
  g_cuda_err = what;
  return KC_ECUDA;
}

kc_status status_code(unsigned st) {
  if (st & ST_STALL) {
    g_cuda_err = "a bulk copy of the counting kernels did not complete";
    return KC_ECUDA;
  }
  if (st & ST_CAPACITY) return KC_ECAPACITY;
  if (st & ST_OVERFLOW) return KC_ERANGE;
  if (st & ST_TIMEOUT) return KC_ETIMEDOUT;
  if (st & ST_BAD_ARG) return KC_EINVAL;
  return KC_OK;
}
}  // namespace kc

using kc::DevBuf;
using kc::cuda_fail;

extern "C" {

const char *kc_strerror(int status) {
  switch (status) {
    case KC_OK: return "ok";
    case KC_EINVAL: return "invalid argument or malformed graph";
    case KC_ERANGE: return "count does not fit in uint64";
    case KC_ENOMEM: return "device allocation failed";
    case KC_ETIMEDOUT: return "deadline passed or cancelled";
    case KC_ECUDA: return "CUDA runtime error";
    case KC_ECAPACITY: return "out-degree above KC_MAX_OUT_DEGREE";
    default: return "unknown status";
  }
}

const char *kc_last_cuda_error(void) { return kc::g_cuda_err.c_str(); }

uint64_t kc_kernel_launches(void) { return kc::g_launches.load(std::memory_order_relaxed); }

void kc_set_bulk_build(int enabled) { kc::g_bulk_build.store(enabled ? 1 : 0, std::memory_order_relaxed); }

void kc_debug_fail_allocations_after(int64_t count) {
  kc::g_alloc_budget.store(count < 0 ? -1 : (long long)count, std::memory_order_relaxed);
}

uint32_t kc_dag_n(const kc_dag *d) { return d ? d->n : 0; }
uint64_t kc_dag_m(const kc_dag *d) { return d ? d->m : 0; }
uint32_t kc_dag_max_out_degree(const kc_dag *d) { return d ? d->max_out : 0; }

void kc_dag_free(kc_dag *d) {
  if (!d) return;
  if (d->ptr) cudaFreeAsync(d->ptr, d->stream);
  if (d->col) cudaFreeAsync(d->col, d->stream);
  if (d->order) cudaFreeAsync(d->order, d->stream);
  if (d->key) cudaFreeAsync(d->key, d->stream);
  if (d->core_id) cudaFreeAsync(d->core_id, d->stream);
  if (d->core_bits) cudaFreeAsync(d->core_bits, d->stream);
  delete d;
}

kc_status kc_orient(const kc_csr *g, int method, kc_dag **out, kc_stream_t stream) {
  if (!g || !out) return KC_EINVAL;
  const int base = method & 0xff;
  const int sym = (method & KC_VALIDATE_SYMMETRY) ? 1 : 0;
  if (base != KC_ORIENT_DEGREE && base != KC_ORIENT_GP && base != KC_ORIENT_BE) return KC_EINVAL;
  if ((method & ~(0xff | KC_VALIDATE_SYMMETRY | KC_CORE_BITS | KC_NO_CORE_BITS)) != 0) return KC_EINVAL;
  if ((method & KC_CORE_BITS) && (method & KC_NO_CORE_BITS)) return KC_EINVAL;
  const int core_mode = (method & KC_CORE_BITS) ? kc::kCoreForce : (method & KC_NO_CORE_BITS) ? kc::kCoreOff : kc::kCoreAuto;
  if (g->n > 0 && (!g->d_row_ptr || (g->nnz > 0 && !g->d_col))) return KC_EINVAL;
  if (g->nnz % 2 != 0) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t n = g->n;

  kc_dag *D = new kc_dag();
  D->n = n;
  D->stream = s;
  cudaGetDevice(&D->device);
  struct Guard {
    kc_dag *d;
    ~Guard() {
      if (d) kc_dag_free(d);
    }
  } guard{D};

  DevBuf status;
  KC_CK(status.alloc(sizeof(unsigned) * 2, s));
  KC_CK(cudaMemsetAsync(status.p, 0, sizeof(unsigned) * 2, s));
  unsigned h_status[2] = {0, 0};
  if (n > 0) {
    KC_CK(kc::launch_validate(*g, sym, status.as<unsigned>(), s));
    KC_CK(cudaMemcpyAsync(h_status, status.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    if (h_status[0] & kc::ST_BAD_CSR) return KC_EINVAL;
  }

  KC_CK(kc::dev_malloc_async((void **)&D->ptr, sizeof(uint64_t) * ((size_t)n + 1), s));
  if (n == 0) {
    KC_CK(cudaMemsetAsync(D->ptr, 0, sizeof(uint64_t), s));
    KC_CK(kc::dev_malloc_async((void **)&D->col, 16, s));
    KC_CK(kc::dev_malloc_async((void **)&D->order, 16, s));
    D->ge.assign(2, 0);
    KC_CK(cudaStreamSynchronize(s));
    *out = D;
    guard.d = nullptr;
    return KC_OK;
  }

  DevBuf key, outdeg, scan_tmp;
  KC_CK(key.alloc(sizeof(uint64_t) * n, s));
  KC_CK(outdeg.alloc(sizeof(uint32_t) * n, s));
  if (base == KC_ORIENT_DEGREE) {
    KC_CK(kc::launch_degree_key(*g, key.as<uint64_t>(), s));
  } else {
    kc_status st = base == KC_ORIENT_GP ? kc::gp_rank(*g, key.as<uint64_t>(), s) : kc::be_rank(*g, key.as<uint64_t>(), s);
    if (st != KC_OK) return st;
  }
  unsigned *d_max = status.as<unsigned>() + 1;
  KC_CK(kc::launch_count_out(*g, key.as<uint64_t>(), outdeg.as<uint32_t>(), d_max, s));
  const size_t te = kc::scan_tmp_elems(n);
  KC_CK(scan_tmp.alloc(sizeof(uint64_t) * te, s));
  KC_CK(kc::exclusive_scan_u32(outdeg.as<uint32_t>(), D->ptr, n, scan_tmp.as<uint64_t>(), te, s));
  uint64_t h_m = 0;
  KC_CK(cudaMemcpyAsync(&h_m, D->ptr + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  KC_CK(cudaMemcpyAsync(&h_status[1], d_max, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  // exactly one arc per undirected edge is kept; any other total means the
  // CSR is not symmetric
  if (h_m != g->nnz / 2) return KC_EINVAL;
  D->m = h_m;
  D->max_out = h_status[1];
  // 16 bytes of padding: bulk copies of an out-list end on a 16-byte boundary
  KC_CK(kc::dev_malloc_async((void **)&D->col, sizeof(uint32_t) * (h_m + 4), s));
  KC_CK(kc::launch_write_out(*g, key.as<uint64_t>(), D->ptr, D->col, s));

  // roots ordered by out-degree, descending (counting sort)
  const uint32_t maxd = D->max_out;
  DevBuf hist;
  KC_CK(hist.alloc(sizeof(unsigned) * ((size_t)maxd + 1), s));
  KC_CK(cudaMemsetAsync(hist.p, 0, sizeof(unsigned) * ((size_t)maxd + 1), s));
  KC_CK(kc::launch_outdeg_hist(D->ptr, n, hist.as<unsigned>(), maxd, s));
  std::vector<unsigned> h_hist((size_t)maxd + 1);
  KC_CK(cudaMemcpyAsync(h_hist.data(), hist.p, sizeof(unsigned) * h_hist.size(), cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  D->ge.assign((size_t)maxd + 2, 0);
  for (int64_t t = maxd; t >= 0; --t) D->ge[t] = D->ge[t + 1] + h_hist[t];
  std::vector<unsigned> start((size_t)maxd + 1);
  for (uint32_t t = 0; t <= maxd; ++t) start[t] = (unsigned)D->ge[t + 1];
  KC_CK(cudaMemcpyAsync(hist.p, start.data(), sizeof(unsigned) * start.size(), cudaMemcpyHostToDevice, s));
  KC_CK(kc::dev_malloc_async((void **)&D->order, sizeof(uint32_t) * n, s));
  KC_CK(kc::launch_outdeg_scatter(D->ptr, n, hist.as<unsigned>(), maxd, D->order, s));
  // out-lists into the total order (positions inside N+(u) = ranks among N+(u))
  auto ge = [&](uint64_t t) -> uint32_t { return t < D->ge.size() ? (uint32_t)D->ge[t] : 0u; };
  KC_CK(kc::launch_sort_rows(D->ptr, D->col, key.as<uint64_t>(), D->order, ge(1025), ge(33), ge(2), maxd, s));
  KC_CK(cudaStreamSynchronize(s));  // `start` is a pageable host buffer read by the copy above
  const kc_status cst = kc::build_core(D, g->d_row_ptr, key.as<uint64_t>(), core_mode, s);
  if (cst != KC_OK) return cst;
  D->key = (uint64_t *)key.release();  // kept: peeling compares ranks
  *out = D;
  guard.d = nullptr;
  return KC_OK;
}

kc_status kc_dag_export(const kc_dag *d, uint64_t *d_ptr, uint32_t *d_col, kc_stream_t stream) {
  if (!d) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (d_ptr) KC_CK(cudaMemcpyAsync(d_ptr, d->ptr, sizeof(uint64_t) * ((size_t)d->n + 1), cudaMemcpyDeviceToDevice, s));
  if (d_col && d->m) KC_CK(cudaMemcpyAsync(d_col, d->col, sizeof(uint32_t) * d->m, cudaMemcpyDeviceToDevice, s));
  KC_CK(cudaStreamSynchronize(s));
  return KC_OK;
}

kc_status kc_dag_get_stats(const kc_dag *d, kc_dag_stats *h_stats, kc_stream_t stream) {
  if (!d || !h_stats) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf acc;
  KC_CK(acc.alloc(sizeof(unsigned long long) * 2, s));
  KC_CK(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * 2, s));
  if (d->n) KC_CK(kc::launch_dag_stats(d->ptr, d->col, d->n, acc.as<unsigned long long>(), s));
  unsigned long long h[2];
  KC_CK(cudaMemcpyAsync(h, acc.p, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  uint64_t tri = 0;
  const kc_status st = kc::run_count(d, 3, nullptr, nullptr, &tri, 0, s);
  if (st != KC_OK) return st;
  uint64_t scanned = 0, looked = 0;
  const kc_status st2 = kc::core_build_split(d, &scanned, &looked, s);
  if (st2 != KC_OK) return st2;
  h_stats->sum_out_sq = h[0];
  h_stats->sum_arc_head = h[1];
  h_stats->triangles = tri;
  h_stats->max_out = d->max_out;
  h_stats->core_vertices = d->core_n;
  h_stats->build_scanned = scanned;
  h_stats->build_lookups = looked;
  return KC_OK;
}

}  // extern "C"

namespace kc {

size_t kc_work_bytes() { return 64; }

// A pass with a time budget: the deadline is taken on the device when the
// pass starts (this kernel runs just before the counting kernels).
__global__ void stamp_deadline_kernel(unsigned long long *out, unsigned long long budget_ns) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *out = t + budget_ns;
}

// total at +0, status word at +8, the three root queues at +16, a device
// deadline at +32
void set_work(CountArgs *a, uint8_t *w) {
  a->total = (unsigned long long *)w;
  a->status = (unsigned *)(w + 8);
  a->queue = (unsigned *)(w + 16);
}

// Kernel configuration for a counting pass over d with smallest k = k_min:
// shared-memory capacity of a block root, grids from the occupancy, the root
// ranges of the order array, and the global scratch the largest roots need.
cudaError_t plan_count(const kc_dag *d, int k_min, bool pv, bool pa, const kc_params *prm, LaunchPlan *out) {
  LaunchPlan &P = *out;
  memset(&P, 0, sizeof P);
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t budget = (size_t)(optin > 4096 ? optin - 2048 : 48 * 1024);
  const uint32_t dcap = block_root_capacity(budget, pv, pa);
  uint32_t light = prm && prm->light_max ? prm->light_max : (uint32_t)kLightMax;
  if (light > (uint32_t)kLightMax) light = kLightMax;
  if (light < 2) light = 2;
  const uint32_t dsmem = std::min<uint32_t>(dcap, std::max<uint32_t>(d->max_out, light + 1));
  P.block_smem = block_root_smem(dsmem, pv, pa);
  P.dcap = dcap;
  P.light = light;
  int per_sm_b = 0, per_sm_w = 0;
  cudaError_t e = count_occupancy(pv, pa, P.block_smem, &per_sm_b, &per_sm_w);
  if (e != cudaSuccess) return e;
  const int sms = sm_count();
  P.block_grid = sms * std::max(1, per_sm_b);
  P.warp_grid = sms * std::max(1, per_sm_w);
  CountArgs &a = P.a;
  a.ptr = d->ptr;
  a.col = d->col;
  a.order = d->order;
  a.k = k_min;
  auto ge = [&](uint64_t t) -> uint32_t { return t < d->ge.size() ? (uint32_t)d->ge[t] : 0u; };
  a.n_light_end = ge((uint64_t)(k_min - 1));
  a.n_big = ge((uint64_t)light + 1);
  a.n_scratch = ge((uint64_t)dcap + 1);
  a.compact_max = prm ? prm->compact_max : 0;
  a.chunk = prm ? prm->chunk : 0;
  const uint32_t lo = prm ? prm->light_order : 0u;
  a.light_by_id = lo == KC_LIGHT_BY_ID ? 1u : 0u;
  a.n = d->n;
  a.light_min = (uint32_t)(k_min - 1);
  a.light_max = light;
  a.bulk_build = bulk_build_enabled() ? 1u : 0u;
  const uint32_t ratio = core_policy().ratio;
  if (d->core_bits && !a.bulk_build && ratio != 0xffffffffu) {
    a.core_id = d->core_id;
    a.core_bits = (const unsigned long long *)d->core_bits;
    a.core_words = d->core_words;
    a.core_ratio = ratio;
  }
  if (a.n_scratch > 0) {
    const size_t slab = (root_layout(d->max_out, pv, pa).bytes + 255) & ~(size_t)255;
    const size_t sbudget = (size_t)4 << 30;
    size_t nb = std::max<size_t>(1, sbudget / slab);
    nb = std::min<size_t>(nb, (size_t)P.block_grid);
    nb = std::min<size_t>(nb, (size_t)a.n_scratch);
    a.scratch_stride = slab;
    a.scratch_blocks = (uint32_t)nb;
    P.scratch_bytes = slab * nb;
  }
  return cudaSuccess;
}

// Shared driver of kc_count / kc_count_per_vertex / kc_count_per_arc.
kc_status run_count(const kc_dag *d, int k, unsigned long long *pv, unsigned long long *pa, uint64_t *h_total,
                    uint64_t deadline_ns, cudaStream_t s, uint64_t budget_ns) {
  if (!d || k < 1 || k > KC_KMAX) return KC_EINVAL;
  if (pa && k < 2) return KC_EINVAL;
  const uint32_t n = d->n;
  if (pv) KC_CK(cudaMemsetAsync(pv, 0, sizeof(unsigned long long) * n, s));
  if (pa && d->m) KC_CK(cudaMemsetAsync(pa, 0, sizeof(unsigned long long) * d->m, s));
  if (k == 1) {
    if (pv) KC_CK(launch_fill_u64(pv, n, 1ull, s));
    KC_CK(cudaStreamSynchronize(s));
    if (h_total) *h_total = n;
    return KC_OK;
  }
  if (k == 2) {
    if (pv && n) KC_CK(launch_degree_from_dag(d->ptr, d->col, n, pv, s));
    if (pa) KC_CK(launch_fill_u64(pa, d->m, 1ull, s));
    KC_CK(cudaStreamSynchronize(s));
    if (h_total) *h_total = d->m;
    return KC_OK;
  }
  const uint32_t need = (uint32_t)(k - 1);  // a root needs k-1 out-neighbours
  if (need > d->max_out) {
    KC_CK(cudaStreamSynchronize(s));
    if (h_total) *h_total = 0;
    return KC_OK;
  }
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;
  LaunchPlan P;
  KC_CK(plan_count(d, k, pv != nullptr, pa != nullptr, nullptr, &P));
  CountArgs &a = P.a;
  a.pv = pv;
  a.pa = pa;
  a.deadline_ns = deadline_ns;
  DevBuf work, scratch;
  KC_CK(work.alloc(kc_work_bytes(), s));
  KC_CK(cudaMemsetAsync(work.p, 0, kc_work_bytes(), s));
  set_work(&a, work.as<uint8_t>());
  if (P.scratch_bytes) {
    KC_CK(scratch.alloc(P.scratch_bytes, s));
    a.scratch = scratch.as<uint8_t>();
  }
  if (budget_ns) {
    unsigned long long *dl = (unsigned long long *)(work.as<uint8_t>() + 32);
    stamp_deadline_kernel<<<1, 1, 0, s>>>(dl, budget_ns);
    note_launch();
    KC_CK(cudaGetLastError());
    a.deadline_dev = dl;
  }
  KC_CK(launch_count(a, pv != nullptr, pa != nullptr, P.block_grid, P.warp_grid, P.block_smem, s));
  unsigned long long h[2] = {0, 0};
  KC_CK(cudaMemcpyAsync(h, work.p, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  const kc_status code = status_code((unsigned)h[1]);
  if (code != KC_OK) return code;
  if (h_total) *h_total = h[0];
  return KC_OK;
}

// Rooted counts of a list of roots: the roots are ordered by out-degree
// (descending) on the host, split into the same three classes as a whole
// pass, and counted by the same two kernels, each root writing its total to
// its caller position.
kc_status run_count_roots(const kc_dag *d, int k, const uint32_t *d_roots, uint32_t r, uint64_t *d_out,
                          uint64_t *h_total, cudaStream_t s) {
  if (!d || k < 1 || k > KC_KMAX || (r > 0 && (!d_roots || !d_out))) return KC_EINVAL;
  if (r == 0) {
    if (h_total) *h_total = 0;
    return KC_OK;
  }
  std::vector<uint32_t> roots(r);
  KC_CK(cudaMemcpyAsync(roots.data(), d_roots, sizeof(uint32_t) * r, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  {
    std::vector<uint32_t> sorted(roots);
    std::sort(sorted.begin(), sorted.end());
    if (sorted.back() >= d->n) return KC_EINVAL;
    for (uint32_t i = 1; i < r; ++i)
      if (sorted[i] == sorted[i - 1]) return KC_EINVAL;
  }
  DevBuf ddeg;
  KC_CK(ddeg.alloc(sizeof(uint32_t) * r, s));
  KC_CK(launch_root_outdeg(d->ptr, d_roots, r, ddeg.as<uint32_t>(), s));
  std::vector<uint32_t> deg(r);
  KC_CK(cudaMemcpyAsync(deg.data(), ddeg.p, sizeof(uint32_t) * r, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  if (k <= 2) {  // one 1-clique per root; its out-arcs are the 2-cliques it roots
    std::vector<uint64_t> out(r);
    uint64_t t = 0;
    for (uint32_t i = 0; i < r; ++i) t += (out[i] = k == 1 ? 1u : deg[i]);
    KC_CK(cudaMemcpyAsync(d_out, out.data(), sizeof(uint64_t) * r, cudaMemcpyHostToDevice, s));
    KC_CK(cudaStreamSynchronize(s));
    if (h_total) *h_total = t;
    return KC_OK;
  }
  KC_CK(cudaMemsetAsync(d_out, 0, sizeof(uint64_t) * r, s));
  const uint32_t need = (uint32_t)(k - 1);
  if (need > d->max_out) {
    KC_CK(cudaStreamSynchronize(s));
    if (h_total) *h_total = 0;
    return KC_OK;
  }
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;
  LaunchPlan P;
  KC_CK(plan_count(d, k, false, false, nullptr, &P));
  CountArgs &a = P.a;
  std::vector<uint32_t> idx(r);
  for (uint32_t i = 0; i < r; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](uint32_t x, uint32_t y) { return deg[x] > deg[y]; });
  std::vector<uint32_t> hb(2 * (size_t)r);  // order, then caller positions
  uint32_t n_scratch = 0, n_big = 0, n_end = 0, dmax = 0;
  for (uint32_t i = 0; i < r; ++i) {
    const uint32_t dg = deg[idx[i]];
    hb[i] = roots[idx[i]];
    hb[r + i] = idx[i];
    n_scratch += dg > P.dcap;
    n_big += dg > P.light;
    n_end += dg >= need;
    dmax = std::max(dmax, dg);
  }
  DevBuf ord, work, scratch;
  KC_CK(ord.alloc(sizeof(uint32_t) * 2 * (size_t)r, s));
  KC_CK(cudaMemcpyAsync(ord.p, hb.data(), sizeof(uint32_t) * 2 * (size_t)r, cudaMemcpyHostToDevice, s));
  a.order = ord.as<uint32_t>();
  a.rooted_pos = ord.as<uint32_t>() + r;
  a.rooted = (unsigned long long *)d_out;
  a.n_scratch = n_scratch;
  a.n_big = std::max(n_big, n_scratch);
  a.n_light_end = std::max(n_end, a.n_big);
  a.light_by_id = 0;
  a.scratch_blocks = 0;
  P.scratch_bytes = 0;
  if (n_scratch > 0) {
    const size_t slab = (root_layout(dmax, false, false).bytes + 255) & ~(size_t)255;
    size_t nb = std::max<size_t>(1, ((size_t)4 << 30) / slab);
    nb = std::min<size_t>(nb, (size_t)P.block_grid);
    nb = std::min<size_t>(nb, (size_t)n_scratch);
    a.scratch_stride = slab;
    a.scratch_blocks = (uint32_t)nb;
    P.scratch_bytes = slab * nb;
    KC_CK(scratch.alloc(P.scratch_bytes, s));
    a.scratch = scratch.as<uint8_t>();
  }
  KC_CK(work.alloc(kc_work_bytes(), s));
  KC_CK(cudaMemsetAsync(work.p, 0, kc_work_bytes(), s));
  set_work(&a, work.as<uint8_t>());
  KC_CK(launch_count(a, false, false, P.block_grid, P.warp_grid, P.block_smem, s));
  unsigned long long h[2] = {0, 0};
  KC_CK(cudaMemcpyAsync(h, work.p, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  const kc_status code = status_code((unsigned)h[1]);
  if (code != KC_OK) return code;
  if (h_total) *h_total = h[0];
  return KC_OK;
}

}  // namespace kc

extern "C" {

kc_status kc_count(const kc_dag *d, int k, uint64_t *h_total, kc_stream_t stream) {
  if (!h_total) return KC_EINVAL;
  return kc::run_count(d, k, nullptr, nullptr, h_total, 0, (cudaStream_t)stream);
}

kc_status kc_count_per_vertex(const kc_dag *d, int k, uint64_t *d_out, uint64_t *h_total, kc_stream_t stream) {
  if (!d_out) return KC_EINVAL;
  return kc::run_count(d, k, (unsigned long long *)d_out, nullptr, h_total, 0, (cudaStream_t)stream);
}

kc_status kc_count_per_arc(const kc_dag *d, int k, uint64_t *d_out, uint64_t *h_total, kc_stream_t stream) {
  if (!d_out) return KC_EINVAL;
  return kc::run_count(d, k, nullptr, (unsigned long long *)d_out, h_total, 0, (cudaStream_t)stream);
}

kc_status kc_count_budget(const kc_dag *d, int k, uint64_t *d_out, uint64_t budget_us, uint64_t *h_total,
                          kc_stream_t stream) {
  if (!h_total || budget_us == 0 || budget_us > (~0ull / 2000ull)) return KC_EINVAL;
  return kc::run_count(d, k, (unsigned long long *)d_out, nullptr, h_total, 0, (cudaStream_t)stream,
                       budget_us * 1000ull);
}

kc_status kc_count_roots(const kc_dag *d, int k, const uint32_t *d_roots, uint32_t num_roots, uint64_t *d_out,
                         uint64_t *h_total, kc_stream_t stream) {
  return kc::run_count_roots(d, k, d_roots, num_roots, d_out, h_total, (cudaStream_t)stream);
}

}  // extern "C"
