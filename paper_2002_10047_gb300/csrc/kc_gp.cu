// Goodrich-Pszona orientation (Algorithm 3 with epsilon = 1, Section 3.1).
//
// Round r removes the c = ceil(n'/3) of the n' remaining vertices that are
// smallest by (induced degree, id) -- the epsilon/(2+epsilon) fraction of
// what remains, so O(log n) rounds -- and then decrements the induced degree
// of their remaining neighbours with atomics (the proof of Theorem 3.1).
// The selection is an exact radix select of the c-th smallest 64-bit key
// (degree << 32 | id) over the compacted list of remaining vertices; all keys
// are distinct, so the removed set is exactly {key <= that key}. The order
// key written for each removed vertex is (round << 32 | degree at removal),
// compared with ties broken by id, which reproduces "append S to L" with the
// vertices of one round in (degree, id) order.
//
// The round sizes depend on n only, so the host issues every launch up front
// with no synchronisation; the select state lives in device memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kc_host.cuh"
#include "kc_internal.cuh"
#include "kc_orient.cuh"

namespace kc {

struct SelectState {
  unsigned long long prefix, mask;
  unsigned want;  // 1-based rank still to find inside the current prefix
  unsigned pad;
};

__global__ void gp_init_kernel(const uint64_t *__restrict__ rp, uint32_t n, uint32_t *__restrict__ deg,
                               uint8_t *__restrict__ state, uint32_t *__restrict__ list) {
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x) {
    deg[v] = (uint32_t)(rp[v + 1] - rp[v]);
    state[v] = 1;
    list[v] = (uint32_t)v;
  }
}

__global__ void gp_select_init_kernel(SelectState *st, unsigned c) {
  st->prefix = 0;
  st->mask = 0;
  st->want = c;
}

__device__ __forceinline__ unsigned long long gp_key(const uint32_t *deg, uint32_t v) {
  return ((unsigned long long)deg[v] << 32) | v;
}

__global__ void __launch_bounds__(kBlock) gp_hist_kernel(const uint32_t *__restrict__ list, uint32_t cnt,
                                                         const uint32_t *__restrict__ deg, const SelectState *st,
                                                         int shift, unsigned *__restrict__ hist) {
  __shared__ unsigned h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  const unsigned long long prefix = st->prefix, mask = st->mask;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const unsigned long long kv = gp_key(deg, list[i]);
    if ((kv & mask) == prefix) atomicAdd(&h[(kv >> shift) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// one warp: find the digit holding the want-th key, narrow the prefix
__global__ void gp_digit_kernel(SelectState *st, const unsigned *__restrict__ hist, int shift) {
  if (threadIdx.x != 0) return;
  unsigned want = st->want, cum = 0;
  int b = 0;
  for (; b < 256; ++b) {
    if (cum + hist[b] >= want) break;
    cum += hist[b];
  }
  if (b > 255) b = 255;  // cannot happen when want <= remaining count
  st->want = want - cum;
  st->prefix |= (unsigned long long)b << shift;
  st->mask |= 255ull << shift;
}

__global__ void gp_mark_kernel(const uint32_t *__restrict__ list, uint32_t cnt, const uint32_t *__restrict__ deg,
                               const SelectState *st, uint32_t round, uint8_t *__restrict__ state,
                               uint64_t *__restrict__ okey, uint32_t *__restrict__ sel, unsigned *sel_count,
                               uint32_t cap) {
  const unsigned long long kth = st->prefix;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t v = list[i];
    if (gp_key(deg, v) <= kth) {
      state[v] = 2;
      okey[v] = ((uint64_t)round << 32) | deg[v];
      const unsigned at = atomicAdd(sel_count, 1u);
      if (at < cap) sel[at] = v;
    }
  }
}

__global__ void __launch_bounds__(kBlock) gp_decrement_kernel(const uint32_t *__restrict__ sel, uint32_t cnt,
                                                              const uint64_t *__restrict__ rp,
                                                              const uint32_t *__restrict__ col,
                                                              const uint8_t *__restrict__ state,
                                                              uint32_t *__restrict__ deg) {
  const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  for (size_t i = warp; i < cnt; i += nwarps) {
    const uint32_t v = sel[i];
    for (uint64_t j = rp[v] + lane; j < rp[v + 1]; j += 32) {
      const uint32_t w = col[j];
      if (state[w] == 1) atomicSub(&deg[w], 1u);
    }
  }
}

__global__ void gp_compact_kernel(const uint32_t *__restrict__ list, uint32_t cnt, uint8_t *__restrict__ state,
                                  uint32_t *__restrict__ out, unsigned *out_count, uint32_t cap) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t v = list[i];
    if (state[v] == 1) {
      const unsigned at = atomicAdd(out_count, 1u);
      if (at < cap) out[at] = v;
    } else {
      state[v] = 0;
    }
  }
}

static unsigned gp_grid(size_t work) {
  size_t g = (work + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)g;
}

kc_status gp_rank(const kc_csr &g, uint64_t *okey, cudaStream_t s) {
  const uint32_t n = g.n;
  if (n == 0) return KC_OK;
  uint32_t *deg = nullptr, *la = nullptr, *lb = nullptr, *sel = nullptr;
  uint8_t *state = nullptr;
  unsigned *hist = nullptr;
  SelectState *st = nullptr;
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  ck(kc::dev_malloc_async((void **)&deg, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&la, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&lb, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&sel, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&state, n, s));
  // hist[256] + two counters
  ck(kc::dev_malloc_async((void **)&hist, sizeof(unsigned) * 260, s));
  ck(kc::dev_malloc_async((void **)&st, sizeof(SelectState), s));
  if (e == cudaSuccess) {
    gp_init_kernel<<<gp_grid(n), kBlock, 0, s>>>(g.d_row_ptr, n, deg, state, la);
    note_launch();
    uint32_t remaining = n, round = 0;
    while (remaining > 0 && e == cudaSuccess) {
      const uint32_t c = (remaining + 2) / 3;
      gp_select_init_kernel<<<1, 1, 0, s>>>(st, c);
      note_launch();
      for (int shift = 56; shift >= 0; shift -= 8) {
        ck(cudaMemsetAsync(hist, 0, sizeof(unsigned) * 256, s));
        gp_hist_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, deg, st, shift, hist);
        note_launch();
        gp_digit_kernel<<<1, 32, 0, s>>>(st, hist, shift);
        note_launch();
      }
      ck(cudaMemsetAsync(hist + 256, 0, sizeof(unsigned) * 2, s));
      gp_mark_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, deg, st, round, state, okey, sel,
                                                          hist + 256, n);
      note_launch();
      gp_decrement_kernel<<<gp_grid((size_t)c * 32), kBlock, 0, s>>>(sel, c, g.d_row_ptr, g.d_col, state, deg);
      note_launch();
      gp_compact_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, state, lb, hist + 257, n);
      note_launch();
      uint32_t *t = la;
      la = lb;
      lb = t;
      remaining -= c;
      ++round;
      ck(cudaGetLastError());
    }
  }
  void *bufs[] = {deg, la, lb, sel, state, hist, st};
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  if (e != cudaSuccess) return kc::cuda_fail(e);
  return KC_OK;
}

// ---------------------------------------------------------------------------
// Barenboim-Elkin orientation (Section 3.1), epsilon = 1. Each round removes
// every remaining vertex of induced degree below (2 + eps) * alpha~, where
// alpha~ bounds the arboricity from the approximate densest subgraph: a
// first peel removes, each round, the vertices of induced degree at most
// 2 (1 + eps) rho(S), rho(S) = |E(S)| / |S|, and keeps the largest rho seen,
// rho~; then rho* <= 2 (1 + eps) rho~ =: alpha~ for the densest subgraph's
// density rho*, and every subgraph has a vertex of degree at most
// 2 rho* < (2 + eps) alpha~, so each round removes at least one vertex (the
// paper's argument gives a constant fraction). Thresholds are exact integer
// fractions. The order key is (round << 32 | degree at removal), ties by id,
// as for Goodrich-Pszona.

__global__ void be_mark_kernel(const uint32_t *__restrict__ list, uint32_t cnt, const uint32_t *__restrict__ deg,
                               uint32_t thr, uint32_t round, uint8_t *__restrict__ state,
                               uint64_t *__restrict__ okey, uint32_t *__restrict__ sel, unsigned *sel_count,
                               uint32_t cap) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t v = list[i];
    if (deg[v] <= thr) {
      state[v] = 2;
      if (okey) okey[v] = ((uint64_t)round << 32) | deg[v];
      const unsigned at = atomicAdd(sel_count, 1u);
      if (at < cap) sel[at] = v;
    }
  }
}

// sum of the induced degrees of the remaining vertices (2 |E(S)|)
__global__ void be_degsum_kernel(const uint32_t *__restrict__ list, uint32_t cnt, const uint32_t *__restrict__ deg,
                                 unsigned long long *sum) {
  unsigned long long acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += (size_t)gridDim.x * blockDim.x)
    acc += deg[list[i]];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(sum, acc);
}

kc_status be_rank(const kc_csr &g, uint64_t *okey, cudaStream_t s) {
  const uint32_t n = g.n;
  if (n == 0) return KC_OK;
  uint32_t *deg = nullptr, *la = nullptr, *lb = nullptr, *sel = nullptr;
  uint8_t *state = nullptr;
  unsigned long long *cnts = nullptr;  // [0] degree sum, [1] selected, [2] kept
  cudaError_t e = cudaSuccess;
  auto ck = [&](cudaError_t x) {
    if (e == cudaSuccess && x != cudaSuccess) e = x;
  };
  ck(kc::dev_malloc_async((void **)&deg, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&la, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&lb, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&sel, sizeof(uint32_t) * n, s));
  ck(kc::dev_malloc_async((void **)&state, n, s));
  ck(kc::dev_malloc_async((void **)&cnts, sizeof(unsigned long long) * 3, s));
  kc_status st = KC_OK;
  // phase 1: the approximate densest subgraph's density rho~ = best_m / best_n
  // phase 2: Barenboim-Elkin rounds with threshold deg < 12 rho~ (eps = 1:
  // (2 + eps) * 2 (1 + eps) = 12)
  uint64_t best_m = 0, best_n = 1;
  for (int phase = 0; phase < 2 && e == cudaSuccess && st == KC_OK; ++phase) {
    gp_init_kernel<<<gp_grid(n), kBlock, 0, s>>>(g.d_row_ptr, n, deg, state, la);
    note_launch();
    uint32_t remaining = n, round = 0;
    while (remaining > 0 && e == cudaSuccess) {
      uint32_t thr;
      if (phase == 0) {
        ck(cudaMemsetAsync(cnts, 0, sizeof(unsigned long long), s));
        be_degsum_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, deg, cnts);
        note_launch();
        unsigned long long dsum = 0;
        ck(cudaMemcpyAsync(&dsum, cnts, 8, cudaMemcpyDeviceToHost, s));
        ck(cudaStreamSynchronize(s));
        if (e != cudaSuccess) break;
        const uint64_t mS = dsum / 2;
        if ((unsigned __int128)mS * best_n > (unsigned __int128)best_m * remaining) {
          best_m = mS;
          best_n = remaining;
        }
        // deg <= 2 (1 + eps) mS / |S| = 4 mS / |S|
        thr = (uint32_t)std::min<uint64_t>(0xffffffffu, (4 * mS) / remaining);
      } else {
        // deg < 12 best_m / best_n  <=>  deg <= floor((12 best_m - 1) / best_n)
        thr = best_m == 0 ? 0u
                          : (uint32_t)std::min<uint64_t>(0xffffffffu, (12 * best_m - 1) / best_n);
      }
      ck(cudaMemsetAsync(cnts + 1, 0, sizeof(unsigned long long) * 2, s));
      be_mark_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, deg, thr, round, state,
                                                          phase == 1 ? okey : nullptr, sel,
                                                          (unsigned *)(cnts + 1), n);
      note_launch();
      unsigned long long h_sel = 0;
      ck(cudaMemcpyAsync(&h_sel, cnts + 1, 8, cudaMemcpyDeviceToHost, s));
      ck(cudaStreamSynchronize(s));
      if (e != cudaSuccess) break;
      const uint32_t c = (uint32_t)(h_sel & 0xffffffffu);
      if (c == 0 || c > remaining) {  // the bound above rules this out
        st = KC_ECUDA;
        break;
      }
      gp_decrement_kernel<<<gp_grid((size_t)c * 32), kBlock, 0, s>>>(sel, c, g.d_row_ptr, g.d_col, state, deg);
      note_launch();
      gp_compact_kernel<<<gp_grid(remaining), kBlock, 0, s>>>(la, remaining, state, lb, (unsigned *)(cnts + 2), n);
      note_launch();
      uint32_t *t = la;
      la = lb;
      lb = t;
      remaining -= c;
      ++round;
      ck(cudaGetLastError());
    }
  }
  void *bufs[] = {deg, la, lb, sel, state, cnts};
  for (void *b : bufs)
    if (b) cudaFreeAsync(b, s);
  if (e != cudaSuccess) return kc::cuda_fail(e);
  return st;
}

}  // namespace kc
