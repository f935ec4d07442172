// Sort every out-list of the oriented graph into the total order (by
// (key, id), the same order that decided the arc directions). With out-lists
// in rank order, the position of a vertex inside N+(u) is its rank among
// N+(u), so the counting kernels can keep one symmetric bit matrix per root
// and read the direction of an arc from the positions of its ends.
//
// Bitonic sorting networks: one warp per row for rows of at most 32 (in
// registers), one warp per row through shared memory up to 1024, one block per
// row through shared memory up to 8192, and one block per row through a
// global buffer beyond that.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.cuh"
#include "kc_orient.cuh"

namespace kc {

__device__ __forceinline__ bool key_less(uint64_t ka, uint32_t a, uint64_t kb, uint32_t b) {
  return ka < kb || (ka == kb && a < b);
}

constexpr uint32_t kPadId = 0xffffffffu;
constexpr uint64_t kPadKey = 0xffffffffffffffffull;

// rows of length 2..32: lane i holds element i, padded with (max, max)
__global__ void __launch_bounds__(kBlock) sort_rows_warp_kernel(const uint64_t *__restrict__ ptr,
                                                                uint32_t *__restrict__ col,
                                                                const uint64_t *__restrict__ key,
                                                                const uint32_t *__restrict__ rows, uint32_t nrows) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (size_t r = warp; r < nrows; r += nwarps) {
    const uint32_t u = rows[r];
    const uint64_t b = ptr[u];
    const uint32_t d = (uint32_t)(ptr[u + 1] - b);
    uint32_t id = lane < d ? col[b + lane] : kPadId;
    uint64_t k = lane < d ? key[id] : kPadKey;
    for (unsigned size = 2; size <= 32; size <<= 1) {
      for (unsigned stride = size >> 1; stride; stride >>= 1) {
        const uint32_t oid = __shfl_xor_sync(0xffffffffu, id, stride);
        const uint64_t ok = __shfl_xor_sync(0xffffffffu, k, stride);
        const bool up = (lane & size) == 0;     // ascending block
        const bool lower = (lane & stride) == 0;
        const bool mine_less = key_less(k, id, ok, oid);
        const bool keep = (lower == up) ? mine_less : !mine_less;
        if (!keep) {
          id = oid;
          k = ok;
        }
      }
    }
    if (lane < d) col[b + lane] = id;
  }
}

// in-place bitonic sort of n (a power of two) (key, id) pairs by `team`
// threads starting at `t0`; stages are ordered by __syncwarp (WARP) or
// __syncthreads
template <bool WARP>
__device__ __forceinline__ void bitonic(uint64_t *k, uint32_t *id, uint32_t n, uint32_t t0, uint32_t team) {
  for (uint32_t size = 2; size <= n; size <<= 1) {
    for (uint32_t stride = size >> 1; stride; stride >>= 1) {
      for (uint32_t i = t0; i < n / 2; i += team) {
        const uint32_t lo = 2 * i - (i & (stride - 1));
        const uint32_t hi = lo + stride;
        const bool up = (lo & size) == 0;
        const bool sw = up ? key_less(k[hi], id[hi], k[lo], id[lo]) : key_less(k[lo], id[lo], k[hi], id[hi]);
        if (sw) {
          const uint64_t tk = k[lo];
          k[lo] = k[hi];
          k[hi] = tk;
          const uint32_t ti = id[lo];
          id[lo] = id[hi];
          id[hi] = ti;
        }
      }
      if (WARP) __syncwarp();
      else __syncthreads();
    }
  }
}

constexpr uint32_t kMidMax = 1024;
constexpr int kMidWarps = 4;

// rows of length 33..1024: one warp per row through shared memory
__global__ void __launch_bounds__(kMidWarps * 32) sort_rows_mid_kernel(const uint64_t *__restrict__ ptr,
                                                                       uint32_t *__restrict__ col,
                                                                       const uint64_t *__restrict__ key,
                                                                       const uint32_t *__restrict__ rows,
                                                                       uint32_t nrows) {
  __shared__ uint64_t sk[kMidWarps][kMidMax];
  __shared__ uint32_t si[kMidWarps][kMidMax];
  const unsigned lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t r = warp; r < nrows; r += nwarps) {
    const uint32_t u = rows[r];
    const uint64_t b = ptr[u];
    const uint32_t d = (uint32_t)(ptr[u + 1] - b);
    if (d > kMidMax) continue;
    uint32_t n = 32;
    while (n < d) n <<= 1;
    for (uint32_t i = lane; i < n; i += 32) {
      const uint32_t v = i < d ? col[b + i] : kPadId;
      si[w][i] = v;
      sk[w][i] = i < d ? key[v] : kPadKey;
    }
    __syncwarp();
    bitonic<true>(sk[w], si[w], n, lane, 32);
    for (uint32_t i = lane; i < d; i += 32) col[b + i] = si[w][i];
    __syncwarp();
  }
}

// rows above 1024: one block per row through shared memory (<= kBigMax) or a
// global buffer of the block's own
constexpr uint32_t kBigMax = 8192;

__global__ void __launch_bounds__(1024) sort_rows_big_kernel(const uint64_t *__restrict__ ptr, uint32_t *__restrict__ col,
                                                             const uint64_t *__restrict__ key,
                                                             const uint32_t *__restrict__ rows, uint32_t nrows,
                                                             uint64_t *gk, uint32_t *gi, size_t gstride) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint64_t *sk = (uint64_t *)smem;
  uint32_t *si = (uint32_t *)(smem + (size_t)kBigMax * 8);
  for (uint32_t r = blockIdx.x; r < nrows; r += gridDim.x) {
    const uint32_t u = rows[r];
    const uint64_t b = ptr[u];
    const uint32_t d = (uint32_t)(ptr[u + 1] - b);
    uint32_t n = 32;
    while (n < d) n <<= 1;
    uint64_t *K = sk;
    uint32_t *I = si;
    if (n > kBigMax) {
      if (!gk || (size_t)n > gstride) continue;  // the caller sized the buffer for the longest row
      K = gk + (size_t)blockIdx.x * gstride;
      I = gi + (size_t)blockIdx.x * gstride;
    }
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t v = i < d ? col[b + i] : kPadId;
      I[i] = v;
      K[i] = i < d ? key[v] : kPadKey;
    }
    __syncthreads();
    bitonic<false>(K, I, n, threadIdx.x, blockDim.x);
    for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) col[b + i] = I[i];
    __syncthreads();
  }
}

cudaError_t launch_sort_rows(const uint64_t *ptr, uint32_t *col, const uint64_t *key, const uint32_t *order,
                             uint32_t n_big, uint32_t n_mid_end, uint32_t n_small_end, uint32_t max_out,
                             cudaStream_t s) {
  // order[] lists roots by out-degree, descending: [0, n_big) have d > 1024,
  // [n_big, n_mid_end) 33..1024, [n_mid_end, n_small_end) 2..32
  if (n_small_end > n_mid_end) {
    size_t g = ((size_t)(n_small_end - n_mid_end) * 32 + kBlock - 1) / kBlock;
    g = g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g);
    sort_rows_warp_kernel<<<(unsigned)g, kBlock, 0, s>>>(ptr, col, key, order + n_mid_end, n_small_end - n_mid_end);
    note_launch();
  }
  if (n_mid_end > n_big) {
    size_t g = (n_mid_end - n_big + kMidWarps - 1) / kMidWarps;
    g = g < 1 ? 1 : (g > 152 * 8 ? 152 * 8 : g);
    sort_rows_mid_kernel<<<(unsigned)g, kMidWarps * 32, 0, s>>>(ptr, col, key, order + n_big, n_mid_end - n_big);
    note_launch();
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_big == 0) return e;
  const size_t smem = (size_t)kBigMax * 12;
  e = cudaFuncSetAttribute(sort_rows_big_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  uint32_t nmax = 32;
  while (nmax < max_out) nmax <<= 1;
  uint64_t *gk = nullptr;
  uint32_t *gi = nullptr;
  const unsigned grid = n_big < 152 ? n_big : 152;
  if (nmax > kBigMax) {
    e = kc::dev_malloc_async((void **)&gk, (size_t)grid * nmax * 8, s);
    if (e != cudaSuccess) return e;
    e = kc::dev_malloc_async((void **)&gi, (size_t)grid * nmax * 4, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(gk, s);
      return e;
    }
  }
  sort_rows_big_kernel<<<grid, 1024, smem, s>>>(ptr, col, key, order, n_big, gk, gi, nmax);
  note_launch();
  e = cudaGetLastError();
  if (gk) cudaFreeAsync(gk, s);
  if (gi) cudaFreeAsync(gi, s);
  return e;
}

}  // namespace kc
