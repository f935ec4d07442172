// Dense-core adjacency of an oriented graph: a layout of the DAG, not a step
// of the paper. The level-2 build of a root u (the DAG induced on N+(u), the
// first-level induced subgraph of Section 3.4) reads the out-list of every
// member x of N+(u).
// On skewed graphs most of those reads are long out-lists of the few
// highest-ranked vertices, reached from millions of light roots: on a
// Chung-Lu graph the build scans sum over arcs u->x of d+(x), hundreds of
// times the arc count. The core C is a set of the highest-ranked vertices,
// C = {v : key[v] >= kappa}, with a bit matrix B over C: B[a][b] = 1 iff the
// core vertices numbered a and b have an arc a -> b. C is closed upwards in
// the total order: an out-neighbour of a core vertex ranks above it, so it is
// in C too. Hence when member x_i of N+(u) (sorted by rank) is in C, so is
// every later member, and row i of the induced subgraph can be read from B
// with one bit per later member instead of a scan of N+(x_i). The counting
// kernels take that path where it is cheaper (kc_count_impl.cuh).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <vector>

#include "kc_core.cuh"
#include "kc_host.cuh"
#include "kc_orient.cuh"

namespace kc {

namespace {

constexpr int kDigitBits = 11;
constexpr uint32_t kBins = 1u << kDigitBits;
constexpr int kCoreBlock = 512;

__device__ __forceinline__ unsigned lane_of() { return threadIdx.x & 31u; }

// Histogram of one digit (bits shift .. match_shift-1, at most 11) of the keys
// whose bits from match_shift up equal `prefix` (all keys when match_shift
// >= 64). Lanes with equal digits add once per group.
__global__ void __launch_bounds__(kCoreBlock) key_digit_hist_kernel(const uint64_t *__restrict__ key, uint32_t n,
                                                                    int shift, int match_shift, uint64_t prefix,
                                                                    unsigned *hist) {
  const uint32_t dmask = (1u << (match_shift - shift)) - 1u;
  __shared__ unsigned h[kBins];
  for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x) h[b] = 0;
  __syncthreads();
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const size_t v = base + threadIdx.x;
    bool ok = false;
    uint32_t dig = 0;
    if (v < n) {
      const uint64_t k = key[v];
      ok = match_shift >= 64 || (k >> match_shift) == prefix;
      dig = (uint32_t)(k >> shift) & dmask;
    }
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const unsigned grp = __match_any_sync(act, dig);
      if (lane_of() == (unsigned)(__ffs(grp) - 1)) atomicAdd(&h[dig], (unsigned)__popc(grp));
    }
  }
  __syncthreads();
  for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x)
    if (h[b]) atomicAdd(&hist[b], h[b]);
}

// core_id[v] = a number in [0, H) for key[v] >= kappa, kNoCore otherwise;
// counter[0] ends at H
__global__ void core_assign_kernel(const uint64_t *__restrict__ key, uint32_t n, uint64_t kappa,
                                   uint32_t *__restrict__ core_id, unsigned *counter) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const size_t v = base + threadIdx.x;
    const bool in = v < n && key[v] >= kappa;
    const unsigned m = __ballot_sync(0xffffffffu, in);
    unsigned at = 0;
    if (lane_of() == 0 && m) at = atomicAdd(counter, (unsigned)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0) + (unsigned)__popc(m & ((1u << lane_of()) - 1u));
    if (v < n) core_id[v] = in ? at : kNoCore;
  }
}

// cv[core_id[v]] = v for the core vertices
__global__ void core_list_kernel(const uint32_t *__restrict__ core_id, uint32_t n, uint32_t *__restrict__ cv) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    const uint32_t a = core_id[v];
    if (a != kNoCore) cv[a] = (uint32_t)v;
  }
}

// core_id[cv[i]] = i: core numbers in rank order
__global__ void core_renumber_kernel(const uint32_t *__restrict__ cv, uint32_t h, uint32_t *__restrict__ core_id) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < h; i += (size_t)gridDim.x * blockDim.x)
    core_id[cv[i]] = (uint32_t)i;
}

// B[a][b] for every arc a -> b between core vertices: one warp per vertex,
// the core vertices' out-lists (all of whose entries are core vertices)
__global__ void __launch_bounds__(kCoreBlock) core_bits_kernel(const uint64_t *__restrict__ ptr,
                                                               const uint32_t *__restrict__ col, uint32_t n,
                                                               const uint32_t *__restrict__ core_id, uint32_t words,
                                                               unsigned long long *bits, unsigned *status) {
  const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t v = warp; v < n; v += nwarps) {
    const uint32_t a = core_id[v];
    if (a == kNoCore) continue;
    unsigned long long *row = bits + (size_t)a * words;
    bool bad = false;
    for (uint64_t j = ptr[v] + lane_of(); j < ptr[v + 1]; j += 32) {
      const uint32_t b = core_id[col[j]];
      if (b == kNoCore) {
        bad = true;  // the set is not closed upwards: cannot happen for kappa from the keys
        continue;
      }
      atomicOr(&row[b >> 6], 1ull << (b & 63));
    }
    if (bad) atomicOr(status, ST_CAPACITY);
  }
}

// sum over vertices of in-degree * out-degree = sum over arcs u -> x of d+(x):
// the out-list entries the level-2 builds of all roots read
__global__ void __launch_bounds__(kCoreBlock) build_volume_kernel(const uint64_t *__restrict__ rp,
                                                                  const uint64_t *__restrict__ dp, uint32_t n,
                                                                  unsigned long long *acc) {
  unsigned long long s = 0;
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    const uint64_t out = dp[v + 1] - dp[v];
    const uint64_t in = (rp[v + 1] - rp[v]) - out;
    s += in * out;
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane_of() == 0 && s) atomicAdd(acc, s);
}

std::atomic<uint32_t> g_core_max{131072};
std::atomic<uint32_t> g_core_ratio{1};

// Out-list entries scanned and core bits looked up by the level-2 builds of
// all roots under the counting kernels' rule (acc[0], acc[1]): one warp per
// root, lanes over its members.
__global__ void __launch_bounds__(kCoreBlock) core_build_split_kernel(const uint64_t *__restrict__ ptr,
                                                                      const uint32_t *__restrict__ col, uint32_t n,
                                                                      const uint32_t *__restrict__ core_id,
                                                                      uint32_t ratio, unsigned long long *acc) {
  const size_t warp = ((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long scanned = 0, looked = 0;
  for (size_t u = warp; u < n; u += nwarps) {
    const uint64_t b = ptr[u];
    const uint32_t d = (uint32_t)(ptr[u + 1] - b);
    for (uint32_t i = lane_of(); i < d; i += 32) {
      const uint32_t x = col[b + i];
      const uint64_t len = ptr[x + 1] - ptr[x];
      const uint32_t later = d - 1 - i;
      if (core_id && core_id[x] != kNoCore && len >= (uint64_t)ratio * later) looked += later;
      else scanned += len;
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    scanned += __shfl_xor_sync(0xffffffffu, scanned, o);
    looked += __shfl_xor_sync(0xffffffffu, looked, o);
  }
  if (lane_of() == 0) {
    if (scanned) atomicAdd(&acc[0], scanned);
    if (looked) atomicAdd(&acc[1], looked);
  }
}

}  // namespace

kc_status core_build_split(const kc_dag *D, uint64_t *scanned, uint64_t *looked, cudaStream_t s) {
  *scanned = *looked = 0;
  if (D->n == 0 || D->m == 0) return KC_OK;
  const uint32_t ratio = core_policy().ratio;
  const bool use = D->core_bits && ratio != 0xffffffffu;
  DevBuf acc;
  KC_CK(acc.alloc(sizeof(unsigned long long) * 2, s));
  KC_CK(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long) * 2, s));
  core_build_split_kernel<<<(unsigned)sm_count() * 8, kCoreBlock, 0, s>>>(
      D->ptr, D->col, D->n, use ? D->core_id : nullptr, ratio, acc.as<unsigned long long>());
  note_launch();
  KC_CK(cudaGetLastError());
  unsigned long long h[2];
  KC_CK(cudaMemcpyAsync(h, acc.p, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  *scanned = h[0];
  *looked = h[1];
  return KC_OK;
}

CorePolicy core_policy() {
  CorePolicy p;
  p.max_vertices = g_core_max.load(std::memory_order_relaxed);
  p.ratio = g_core_ratio.load(std::memory_order_relaxed);
  p.min_max_out = 128;
  p.min_volume_per_arc = 16;
  return p;
}

namespace {

kc_status build_core_impl(kc_dag *D, const uint64_t *rp, const uint64_t *key, int mode, cudaStream_t s) {
  const uint32_t n = D->n;
  const CorePolicy pol = core_policy();
  if (mode == kCoreOff || pol.max_vertices == 0 || n == 0 || D->m == 0) return KC_OK;
  const unsigned grid = (unsigned)sm_count() * 4;
  if (mode != kCoreForce) {
    // automatic: only where the builds read long out-lists on average
    if (D->max_out < pol.min_max_out) return KC_OK;
    DevBuf acc;
    KC_CK(acc.alloc(sizeof(unsigned long long), s));
    KC_CK(cudaMemsetAsync(acc.p, 0, sizeof(unsigned long long), s));
    build_volume_kernel<<<grid, kCoreBlock, 0, s>>>(rp, D->ptr, n, acc.as<unsigned long long>());
    note_launch();
    KC_CK(cudaGetLastError());
    unsigned long long vol = 0;
    KC_CK(cudaMemcpyAsync(&vol, acc.p, sizeof vol, cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    D->build_volume = vol;
    if (vol < (unsigned long long)pol.min_volume_per_arc * D->m) return KC_OK;
  }
  // largest core: max_vertices, and a bit matrix no larger than the DAG's own
  // arrays (64 MiB at least) unless forced
  uint64_t hmax = pol.max_vertices;
  if (mode != kCoreForce) {
    const double dag_bytes = 8.0 * ((double)n + 1) + 4.0 * (double)D->m;
    const double cap_bits = 8.0 * std::max(dag_bytes, 64.0 * 1024 * 1024);
    const uint64_t by_mem = (uint64_t)std::sqrt(cap_bits);
    hmax = std::min<uint64_t>(hmax, by_mem & ~(uint64_t)63);
    // and at most a quarter of the device memory free now
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const uint64_t by_free = (uint64_t)std::sqrt(8.0 * (double)free_b / 4.0);
      hmax = std::min<uint64_t>(hmax, by_free & ~(uint64_t)63);
    } else {
      cudaGetLastError();
    }
  }
  hmax = std::min<uint64_t>(hmax, n);
  if (hmax < 64 && mode != kCoreForce) return KC_OK;
  // kappa: one above the (hmax+1)-th largest key, found one 11-bit digit at a
  // time from the top (radix selection); kappa = 0 when hmax >= n
  uint64_t kappa = 0;
  if (hmax < n) {
    DevBuf hist;
    KC_CK(hist.alloc(sizeof(unsigned) * kBins, s));
    std::vector<unsigned> h(kBins);
    uint64_t r = hmax + 1;  // rank from the top of the key sought
    uint64_t prefix = 0;
    for (int shift = 64 - kDigitBits; shift > -kDigitBits; shift -= kDigitBits) {
      const int sh = shift < 0 ? 0 : shift;
      const int width = shift < 0 ? kDigitBits + shift : kDigitBits;
      const int match_shift = sh + width;
      KC_CK(cudaMemsetAsync(hist.p, 0, sizeof(unsigned) * kBins, s));
      key_digit_hist_kernel<<<grid, kCoreBlock, 0, s>>>(key, n, sh, match_shift, prefix, hist.as<unsigned>());
      note_launch();
      KC_CK(cudaGetLastError());
      KC_CK(cudaMemcpyAsync(h.data(), hist.p, sizeof(unsigned) * kBins, cudaMemcpyDeviceToHost, s));
      KC_CK(cudaStreamSynchronize(s));
      const uint32_t top = (1u << width) - 1u;
      uint64_t cum = 0;
      int64_t b = top;
      for (; b >= 0; --b) {
        if (cum + h[b] >= r) break;
        cum += h[b];
      }
      if (b < 0) return internal_fail("dense core: key digit counts do not add up");
      r -= cum;
      prefix = (prefix << width) | (uint64_t)b;
    }
    kappa = prefix + 1;  // prefix is now the (hmax+1)-th largest key itself
  }
  DevBuf ctr;
  KC_CK(ctr.alloc(sizeof(unsigned) * 2, s));
  KC_CK(cudaMemsetAsync(ctr.p, 0, sizeof(unsigned) * 2, s));
  KC_CK(dev_malloc_async((void **)&D->core_id, sizeof(uint32_t) * n, s));
  core_assign_kernel<<<grid, kCoreBlock, 0, s>>>(key, n, kappa, D->core_id, ctr.as<unsigned>());
  note_launch();
  KC_CK(cudaGetLastError());
  unsigned H = 0;
  KC_CK(cudaMemcpyAsync(&H, ctr.p, sizeof H, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  if (H == 0 || H > hmax) {  // no core (kappa above every key), or a miscount
    cudaFreeAsync(D->core_id, s);
    D->core_id = nullptr;
    return H == 0 ? KC_OK : internal_fail("dense core: more vertices above the threshold than selected");
  }
  // number the core in rank order, so that the later members of a root (in
  // rank order) have increasing core numbers and the lookups of one row fall
  // into few words: the core vertices as one row sorted by (key, id)
  if (H > 1) {
    DevBuf cv, rptr, rord;
    KC_CK(cv.alloc(sizeof(uint32_t) * H, s));
    KC_CK(rptr.alloc(sizeof(uint64_t) * 2, s));
    KC_CK(rord.alloc(sizeof(uint32_t), s));
    const uint64_t hp[2] = {0, H};
    KC_CK(cudaMemcpyAsync(rptr.p, hp, sizeof hp, cudaMemcpyHostToDevice, s));
    KC_CK(cudaMemsetAsync(rord.p, 0, sizeof(uint32_t), s));
    core_list_kernel<<<grid, kCoreBlock, 0, s>>>(D->core_id, n, cv.as<uint32_t>());
    note_launch();
    KC_CK(cudaGetLastError());
    const uint32_t big = H > 1024 ? 1u : 0u, mid = H > 32 ? 1u : 0u;
    KC_CK(launch_sort_rows(rptr.as<uint64_t>(), cv.as<uint32_t>(), key, rord.as<uint32_t>(), big, mid, 1u, H, s));
    core_renumber_kernel<<<grid, kCoreBlock, 0, s>>>(cv.as<uint32_t>(), H, D->core_id);
    note_launch();
    KC_CK(cudaGetLastError());
    KC_CK(cudaStreamSynchronize(s));  // hp is a host buffer read by the copy above
  }
  const uint32_t words = (H + 63u) / 64u;
  const size_t bytes = (size_t)H * words * 8;
  KC_CK(dev_malloc_async((void **)&D->core_bits, bytes, s));
  KC_CK(cudaMemsetAsync(D->core_bits, 0, bytes, s));
  core_bits_kernel<<<grid * 2, kCoreBlock, 0, s>>>(D->ptr, D->col, n, D->core_id, words,
                                                   (unsigned long long *)D->core_bits, ctr.as<unsigned>() + 1);
  note_launch();
  KC_CK(cudaGetLastError());
  unsigned st = 0;
  KC_CK(cudaMemcpyAsync(&st, ctr.as<unsigned>() + 1, sizeof st, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  if (st) return internal_fail("dense core: an out-neighbour of a core vertex is outside the core");
  D->core_n = H;
  D->core_words = words;
  return KC_OK;
}

}  // namespace

kc_status build_core(kc_dag *D, const uint64_t *rp, const uint64_t *key, int mode, cudaStream_t s) {
  const kc_status st = build_core_impl(D, rp, key, mode, s);
  if (st == KC_ENOMEM && mode == kCoreAuto) {
    // the core is optional: without memory for it the handle has none
    if (D->core_id) cudaFreeAsync(D->core_id, s);
    if (D->core_bits) cudaFreeAsync(D->core_bits, s);
    D->core_id = nullptr;
    D->core_bits = nullptr;
    D->core_n = D->core_words = 0;
    return KC_OK;
  }
  return st;
}

}  // namespace kc

extern "C" {

void kc_set_core_policy(uint32_t max_vertices, uint32_t ratio) {
  kc::g_core_max.store(max_vertices, std::memory_order_relaxed);
  kc::g_core_ratio.store(ratio, std::memory_order_relaxed);
}

uint32_t kc_dag_core_vertices(const kc_dag *d) { return d ? d->core_n : 0; }

}  // extern "C"
