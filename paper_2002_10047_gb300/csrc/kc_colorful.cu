// Colorful sparsification (Section 3.3, "Sampling"; the estimator theorem in
// Appendix B): approximate k-clique counting. Every vertex takes one of c colors
// uniformly at random, only the edges whose endpoints share a color are kept,
// and the exact k-clique count C of that sparser graph gives the unbiased
// estimate C * c^(k-1) of the count of the whole graph.
//
// Colors come from the splitmix64 generator (Steele, Lea and Flood, 2014):
// vertex v's draw is splitmix64's output for state seed + (v + 1) * gamma,
// gamma = 0x9E3779B97F4A7C15, and its color is the high 32 bits of the draw
// scaled to [0, c) (the bias this leaves is below c / 2^32).
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "kc_host.cuh"
#include "kc_orient.cuh"

namespace kc {
namespace {

constexpr int kColorBlock = 256;

__device__ __forceinline__ uint32_t vertex_color(uint64_t seed, uint32_t v, uint32_t c) {
  uint64_t z = seed + (uint64_t)(v + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (uint32_t)(((z >> 32) * (uint64_t)c) >> 32);
}

__global__ void color_kernel(uint32_t n, uint64_t seed, uint32_t c, uint32_t *__restrict__ color) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    color[v] = vertex_color(seed, (uint32_t)v, c);
}

// kept arcs per row: both endpoints of the same color (one warp per row)
__global__ void mono_count_kernel(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col, uint32_t n,
                                  const uint32_t *__restrict__ color, uint32_t *__restrict__ deg) {
  const unsigned lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t v = w0; v < n; v += nw) {
    const uint32_t cv = color[v];
    unsigned c = 0;
    for (uint64_t e = rp[v] + lane; e < rp[v + 1]; e += 32) c += color[col[e]] == cv ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) deg[v] = c;
  }
}

// the kept arcs, in the row's (ascending) order
__global__ void mono_write_kernel(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col, uint32_t n,
                                  const uint32_t *__restrict__ color, const uint64_t *__restrict__ rp2,
                                  uint32_t *__restrict__ col2) {
  const unsigned lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t v = w0; v < n; v += nw) {
    const uint32_t cv = color[v];
    const uint64_t e1 = rp[v + 1], end = rp2[v + 1];
    uint64_t out = rp2[v];
    for (uint64_t b = rp[v]; b < e1; b += 32) {  // warp-uniform trip count
      const uint64_t e = b + lane;
      uint32_t u = 0;
      bool keep = false;
      if (e < e1) {
        u = col[e];
        keep = color[u] == cv;
      }
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      const uint64_t at = out + (unsigned)__popc(m & ((1u << lane) - 1u));
      if (keep && at < end) col2[at] = u;
      out += (unsigned)__popc(m);
    }
  }
}

unsigned grid_for(size_t work, int block) {
  size_t g = (work + block - 1) / block;
  return (unsigned)std::max<size_t>(1, std::min<size_t>(g, (size_t)sm_count() * 32));
}

}  // namespace
}  // namespace kc

extern "C" kc_status kc_count_colorful(const kc_csr *g, int k, uint32_t colors, uint64_t seed, int method,
                                       uint64_t *h_sparse_count, double *h_estimate, kc_stream_t stream) {
  using namespace kc;
  if (!g || !h_sparse_count || colors == 0 || k < 1 || k > KC_KMAX) return KC_EINVAL;
  const uint32_t n = g->n;
  if (n > 0 && (!g->d_row_ptr || (g->nnz > 0 && !g->d_col))) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf color, deg, rp2, col2, tmp;
  KC_CK(color.alloc(sizeof(uint32_t) * std::max<uint32_t>(n, 1), s));
  KC_CK(deg.alloc(sizeof(uint32_t) * std::max<uint32_t>(n, 1), s));
  KC_CK(rp2.alloc(sizeof(uint64_t) * ((size_t)n + 1), s));
  uint64_t nnz2 = 0;
  if (n > 0) {
    color_kernel<<<grid_for(n, kColorBlock), kColorBlock, 0, s>>>(n, seed, colors, color.as<uint32_t>());
    note_launch();
    mono_count_kernel<<<grid_for((size_t)n * 32, kColorBlock), kColorBlock, 0, s>>>(
        g->d_row_ptr, g->d_col, n, color.as<uint32_t>(), deg.as<uint32_t>());
    note_launch();
    const size_t te = scan_tmp_elems(n);
    KC_CK(tmp.alloc(sizeof(uint64_t) * te, s));
    KC_CK(exclusive_scan_u32(deg.as<uint32_t>(), rp2.as<uint64_t>(), n, tmp.as<uint64_t>(), te, s));
    KC_CK(cudaMemcpyAsync(&nnz2, rp2.as<uint64_t>() + n, 8, cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    if (nnz2 > g->nnz) return KC_ECUDA;
  } else {
    KC_CK(cudaMemsetAsync(rp2.p, 0, sizeof(uint64_t), s));
  }
  KC_CK(col2.alloc(sizeof(uint32_t) * std::max<uint64_t>(nnz2, 1), s));
  if (n > 0) {
    mono_write_kernel<<<grid_for((size_t)n * 32, kColorBlock), kColorBlock, 0, s>>>(
        g->d_row_ptr, g->d_col, n, color.as<uint32_t>(), rp2.as<uint64_t>(), col2.as<uint32_t>());
    note_launch();
    KC_CK(cudaGetLastError());
  }
  // the sparse graph is simple and symmetric whenever g is (a kept arc's
  // reverse has the same two colors), so it is oriented and counted as is
  const kc_csr g2 = {n, nnz2, rp2.as<uint64_t>(), col2.as<uint32_t>()};
  kc_dag *d2 = nullptr;
  kc_status st = kc_orient(&g2, method & 0xff, &d2, stream);
  if (st != KC_OK) return st;
  uint64_t cnt = 0;
  st = kc_count(d2, k, &cnt, stream);
  kc_dag_free(d2);
  if (st != KC_OK) return st;
  *h_sparse_count = cnt;
  if (h_estimate) {
    double scale = 1.0;
    for (int i = 1; i < k; ++i) scale *= (double)colors;
    *h_estimate = (double)cnt * scale;
  }
  return KC_OK;
}
