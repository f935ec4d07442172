// Orientation (Section 3.1) and the device primitives it needs: CSR
// validation, ranking, the filter that keeps low->high arcs, an exclusive
// scan, and the out-degree bucketing of roots used by the counting kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.cuh"
#include "kc_orient.cuh"

namespace kc {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- validation
// Section 2 assumes simple undirected graphs: every row strictly ascending
// (no duplicates), no self-loops, ids < n, offsets consistent; optionally
// every arc u->v has its reverse v->u.
__global__ void __launch_bounds__(kBlock) validate_csr_kernel(const uint64_t *__restrict__ rp,
                                                              const uint32_t *__restrict__ col, uint32_t n,
                                                              uint64_t nnz, int check_sym, unsigned *status) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = lane_id();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rp[0] != 0 || rp[n] != nnz) atomicOr(status, ST_BAD_CSR);
  }
  for (size_t v = warp; v < n; v += nwarps) {
    const uint64_t b = rp[v], e = rp[v + 1];
    if (b > e || e > nnz) {
      if (lane == 0) atomicOr(status, ST_BAD_CSR);
      continue;
    }
    bool bad = false;
    for (uint64_t j = b + lane; j < e; j += 32) {
      const uint32_t y = col[j];
      bad |= (y >= n) || (y == (uint32_t)v);
      if (j + 1 < e) bad |= col[j + 1] <= y;
      if (!bad && check_sym) {
        uint64_t lo = rp[y], hi = rp[y + 1];
        if (lo > hi || hi > nnz) continue;  // that row is flagged by its own warp
        while (lo < hi) {
          const uint64_t mid = (lo + hi) >> 1;
          if (col[mid] < (uint32_t)v) lo = mid + 1; else hi = mid;
        }
        bad |= !(lo < rp[y + 1] && col[lo] == (uint32_t)v);
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, ST_BAD_CSR);
  }
}

// ------------------------------------------------------------ ranking keys
// Degree ordering (Section 5): key(v) = deg(v); ties broken by id.
__global__ void degree_key_kernel(const uint64_t *__restrict__ rp, uint32_t n, uint64_t *__restrict__ key) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    key[v] = rp[v + 1] - rp[v];
}

__device__ __forceinline__ bool ranks_below(uint64_t ku, uint32_t u, uint64_t kv, uint32_t v) {
  return ku < kv || (ku == kv && u < v);
}

// -------------------------------------------------------------- direction
// Filter of Section 3.1: keep u->v iff u precedes v in the order. Pass 1
// counts the kept arcs of every row; pass 2 writes them at the scanned
// offsets, in the row's (ascending) order.
__global__ void __launch_bounds__(kBlock) count_out_kernel(const uint64_t *__restrict__ rp,
                                                           const uint32_t *__restrict__ col, uint32_t n,
                                                           const uint64_t *__restrict__ key,
                                                           uint32_t *__restrict__ outdeg, unsigned *maxdeg) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = lane_id();
  unsigned cmax = 0;  // one atomic per warp: a per-row atomic on one word serialises
  for (size_t u = warp; u < n; u += nwarps) {
    const uint64_t ku = key[u];
    unsigned c = 0;
    for (uint64_t j = rp[u] + lane; j < rp[u + 1]; j += 32) {
      const uint32_t v = col[j];
      c += ranks_below(ku, (uint32_t)u, key[v], v);
    }
    c = warp_sum(c);
    if (lane == 0) outdeg[u] = c;
    cmax = c > cmax ? c : cmax;
  }
  if (lane == 0 && cmax) atomicMax(maxdeg, cmax);
}

__global__ void __launch_bounds__(kBlock) write_out_kernel(const uint64_t *__restrict__ rp,
                                                           const uint32_t *__restrict__ col, uint32_t n,
                                                           const uint64_t *__restrict__ key,
                                                           const uint64_t *__restrict__ dag_ptr,
                                                           uint32_t *__restrict__ dag_col) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = lane_id();
  const unsigned below = (1u << lane) - 1u;
  for (size_t u = warp; u < n; u += nwarps) {
    const uint64_t ku = key[u];
    uint64_t w = dag_ptr[u];
    const uint64_t wend = dag_ptr[u + 1];
    for (uint64_t j0 = rp[u]; j0 < rp[u + 1]; j0 += 32) {
      const uint64_t j = j0 + lane;
      bool keep = false;
      uint32_t v = 0;
      if (j < rp[u + 1]) {
        v = col[j];
        keep = ranks_below(ku, (uint32_t)u, key[v], v);
      }
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      const uint64_t at = w + __popc(bal & below);
      if (keep && at < wend) dag_col[at] = v;
      w += __popc(bal);
    }
  }
}

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

__device__ uint64_t block_exclusive_scan(uint64_t v, uint64_t *total) {
  __shared__ uint64_t warp_tot[kWarps];
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5;
  uint64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= (unsigned)o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  uint64_t off = 0, all = 0;
  for (int w = 0; w < kWarps; ++w) {
    if (w < (int)wid) off += warp_tot[w];
    all += warp_tot[w];
  }
  __syncthreads();
  *total = all;
  return off + x - v;
}

__global__ void __launch_bounds__(kBlock) scan_reduce_kernel(const uint32_t *__restrict__ in, size_t n,
                                                             uint64_t *__restrict__ sums) {
  const size_t base = (size_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kBlock)
    if (base + i < n) s += in[base + i];
  uint64_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of nb block sums in place; sums[nb] = grand total
__global__ void __launch_bounds__(kBlock) scan_sums_kernel(uint64_t *sums, size_t nb) {
  uint64_t carry = 0;
  for (size_t base = 0; base < nb; base += kBlock) {
    const size_t i = base + threadIdx.x;
    const uint64_t v = i < nb ? sums[i] : 0;
    uint64_t tot;
    const uint64_t ex = block_exclusive_scan(v, &tot);
    if (i < nb) sums[i] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kBlock) scan_final_kernel(const uint32_t *__restrict__ in, size_t n,
                                                            const uint64_t *__restrict__ sums,
                                                            uint64_t *__restrict__ out) {
  const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = base + i < n ? in[base + i] : 0u;
    s += v[i];
  }
  uint64_t tot;
  uint64_t run = sums[blockIdx.x] + block_exclusive_scan(s, &tot);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) {
    const size_t nb = gridDim.x;
    out[n] = sums[nb];
  }
}

size_t scan_tmp_elems(size_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t exclusive_scan_u32(const uint32_t *in, uint64_t *out, size_t n, uint64_t *tmp, size_t tmp_elems,
                               cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(uint64_t), s);
  const size_t nb = (n + kScanTile - 1) / kScanTile;
  if (tmp_elems < nb + 1) return cudaErrorInvalidValue;
  scan_reduce_kernel<<<(unsigned)nb, kBlock, 0, s>>>(in, n, tmp);
  note_launch();
  scan_sums_kernel<<<1, kBlock, 0, s>>>(tmp, nb);
  note_launch();
  scan_final_kernel<<<(unsigned)nb, kBlock, 0, s>>>(in, n, tmp, out);
  note_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------- root work ordering
// Most vertices share a few small out-degrees, so lanes with equal
// out-degrees add once per group (one atomic per distinct value in a warp).
__global__ void outdeg_hist_kernel(const uint64_t *__restrict__ dp, uint32_t n, unsigned *hist, uint32_t maxd) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t base = (size_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const size_t v = base + threadIdx.x;
    const uint64_t d = v < n ? dp[v + 1] - dp[v] : ~0ull;
    const bool ok = d <= maxd;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const unsigned grp = __match_any_sync(act, (unsigned)d);
      if (lane_id() == (unsigned)(__ffs(grp) - 1)) atomicAdd(&hist[d], (unsigned)__popc(grp));
    }
  }
}

// cursor[d] starts at the first slot of out-degree d in descending order; a
// group of lanes with equal out-degree reserves its slots with one atomic
__global__ void outdeg_scatter_kernel(const uint64_t *__restrict__ dp, uint32_t n, unsigned *cursor,
                                      uint32_t maxd, uint32_t *__restrict__ order) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  const unsigned lane = lane_id();
  for (size_t base = (size_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const size_t v = base + threadIdx.x;
    const uint64_t d = v < n ? dp[v + 1] - dp[v] : ~0ull;
    const bool ok = d <= maxd;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (ok) {
      const unsigned grp = __match_any_sync(act, (unsigned)d);
      const int leader = __ffs(grp) - 1;
      unsigned at = 0;
      if (lane == (unsigned)leader) at = atomicAdd(&cursor[d], (unsigned)__popc(grp));
      at = __shfl_sync(grp, at, leader) + (unsigned)__popc(grp & ((1u << lane) - 1u));
      if (at < n) order[at] = (uint32_t)v;
    }
  }
}

// ------------------------------------------------------------- small k
__global__ void fill_u64_kernel(unsigned long long *out, size_t n, unsigned long long v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = v;
}

// k = 2: per-vertex count = degree = out-degree + in-degree in the DAG
__global__ void degree_from_dag_kernel(const uint64_t *__restrict__ dp, const uint32_t *__restrict__ dc, uint32_t n,
                                       unsigned long long *out) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = lane_id();
  for (size_t u = warp; u < n; u += nwarps) {
    if (lane == 0) atomicAdd(&out[u], (unsigned long long)(dp[u + 1] - dp[u]));
    for (uint64_t j = dp[u] + lane; j < dp[u + 1]; j += 32) atomicAdd(&out[dc[j]], 1ull);
  }
}

// out-degree of each listed root (ids already checked to be < n)
__global__ void root_outdeg_kernel(const uint64_t *__restrict__ dp, const uint32_t *__restrict__ roots, uint32_t r,
                                   uint32_t *out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < r; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t u = roots[i];
    out[i] = (uint32_t)(dp[u + 1] - dp[u]);
  }
}

// ------------------------------------------------------------- statistics
// sum over roots of d+(u)^2 and over arcs u->v of d+(v)
__global__ void __launch_bounds__(kBlock) dag_stats_kernel(const uint64_t *__restrict__ dp,
                                                           const uint32_t *__restrict__ dc, uint32_t n,
                                                           unsigned long long *acc /*2*/) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = lane_id();
  unsigned long long sq = 0, head = 0;
  for (size_t u = warp; u < n; u += nwarps) {
    const uint64_t ub = dp[u], ue = dp[u + 1];
    const uint64_t du = ue - ub;
    if (lane == 0) sq += du * du;
    for (uint64_t a = ub + lane; a < ue; a += 32) {
      const uint32_t v = dc[a];
      head += dp[v + 1] - dp[v];
    }
  }
  sq = warp_sum(sq);
  head = warp_sum(head);
  if (lane == 0) {
    atomicAdd(&acc[0], sq);
    atomicAdd(&acc[1], head);
  }
}

// ------------------------------------------------------------ launchers
static unsigned grid_for(size_t work, size_t per_block) {
  size_t g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > 152 * 64) g = 152 * 64;
  return (unsigned)g;
}

cudaError_t launch_validate(const kc_csr &g, int sym, unsigned *status, cudaStream_t s) {
  validate_csr_kernel<<<grid_for((size_t)g.n * 32, kBlock), kBlock, 0, s>>>(g.d_row_ptr, g.d_col, g.n, g.nnz, sym,
                                                                             status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_degree_key(const kc_csr &g, uint64_t *key, cudaStream_t s) {
  degree_key_kernel<<<grid_for(g.n, kBlock), kBlock, 0, s>>>(g.d_row_ptr, g.n, key);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_count_out(const kc_csr &g, const uint64_t *key, uint32_t *outdeg, unsigned *maxdeg,
                             cudaStream_t s) {
  count_out_kernel<<<grid_for((size_t)g.n * 32, kBlock), kBlock, 0, s>>>(g.d_row_ptr, g.d_col, g.n, key, outdeg,
                                                                          maxdeg);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_write_out(const kc_csr &g, const uint64_t *key, const uint64_t *dag_ptr, uint32_t *dag_col,
                             cudaStream_t s) {
  write_out_kernel<<<grid_for((size_t)g.n * 32, kBlock), kBlock, 0, s>>>(g.d_row_ptr, g.d_col, g.n, key, dag_ptr,
                                                                          dag_col);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_outdeg_hist(const uint64_t *dp, uint32_t n, unsigned *hist, uint32_t maxd, cudaStream_t s) {
  outdeg_hist_kernel<<<grid_for(n, kBlock), kBlock, 0, s>>>(dp, n, hist, maxd);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_outdeg_scatter(const uint64_t *dp, uint32_t n, unsigned *cursor, uint32_t maxd, uint32_t *order,
                                  cudaStream_t s) {
  outdeg_scatter_kernel<<<grid_for(n, kBlock), kBlock, 0, s>>>(dp, n, cursor, maxd, order);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long *out, size_t n, unsigned long long v, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  fill_u64_kernel<<<grid_for(n, kBlock), kBlock, 0, s>>>(out, n, v);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_root_outdeg(const uint64_t *dp, const uint32_t *roots, uint32_t r, uint32_t *out,
                               cudaStream_t s) {
  if (r == 0) return cudaSuccess;
  root_outdeg_kernel<<<grid_for(r, kBlock), kBlock, 0, s>>>(dp, roots, r, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_degree_from_dag(const uint64_t *dp, const uint32_t *dc, uint32_t n, unsigned long long *out,
                                   cudaStream_t s) {
  degree_from_dag_kernel<<<grid_for((size_t)n * 32, kBlock), kBlock, 0, s>>>(dp, dc, n, out);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_dag_stats(const uint64_t *dp, const uint32_t *dc, uint32_t n, unsigned long long *acc,
                             cudaStream_t s) {
  dag_stats_kernel<<<grid_for((size_t)n * 32, kBlock), kBlock, 0, s>>>(dp, dc, n, acc);
  note_launch();
  return cudaGetLastError();
}

}  // namespace kc
