// Internal declarations shared by the libkclique translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "kclique.h"

namespace kc {

// Device status word bits (or-ed by kernels, read by the host after a launch).
enum : unsigned {
  ST_OVERFLOW = 1u,   // a count wrapped uint64
  ST_BAD_CSR = 2u,    // validation failed
  ST_TIMEOUT = 4u,    // deadline / cancel
  ST_CAPACITY = 8u,   // an internal capacity check failed (the access was skipped)
};

constexpr int kBlock = 256;              // threads per block of every kernel here
constexpr int kWarps = kBlock / 32;
constexpr int kLightMax = 64;            // roots with d+ <= 64 use one warp and one-word rows
constexpr int kMaxFrames = KC_KMAX - 2;  // depth of the explicit DFS stack

struct CountArgs {
  const uint64_t *ptr;       // DAG offsets, n+1
  const uint32_t *col;       // DAG out-lists, m
  const uint32_t *order;     // roots sorted by out-degree, descending
  uint32_t n_huge;           // order[0, n_huge): d+ > dsmem (matrix in global scratch)
  uint32_t n_heavy_end;      // order[n_huge, n_heavy_end): kLightMax < d+ <= dsmem (block, smem)
  uint32_t n_light_end;      // order[n_heavy_end, n_light_end): k-1 <= d+ <= kLightMax (warp)
  int k;
  uint32_t dsmem;            // largest out-degree whose matrix fits the block's shared memory
  unsigned long long *total; // global sum
  unsigned long long *pv;    // per-vertex output (n) or null
  unsigned long long *pa;    // per-arc output (m) or null
  unsigned *status;
  unsigned *queue;           // [0] huge, [1] heavy, [2] light
  uint64_t *scratch;         // huge roots: per-block slabs
  size_t scratch_stride;     // bytes per slab
  uint32_t scratch_blocks;   // blocks that take huge roots
  uint64_t deadline_ns;      // globaltimer deadline, 0 = none
};

// Bytes of the per-root working set for a block-level root with out-degree d
// (list, rows, transposed rows, per-vertex counters, per-arc sums, pair prefix).
__host__ __device__ inline size_t root_words(uint32_t d) { return (d + 63u) / 64u; }
__host__ __device__ inline uint32_t group_for_words(uint32_t w) {
  uint32_t g = 1;
  while (g < w && g < 32) g <<= 1;
  return g;
}
// Words per row in memory: the group width G (a power of two >= the row's
// 64-bit word count) for d <= 2048, else 32 lanes x NW words, NW in {2,4,8}.
__host__ __device__ inline uint32_t row_stride(uint32_t d) {
  uint32_t w = (uint32_t)root_words(d);
  if (w <= 32) return group_for_words(w);
  uint32_t nw = (w + 31u) / 32u;
  nw = nw <= 2 ? 2u : (nw <= 4 ? 4u : 8u);
  return 32u * nw;
}
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline size_t root_bytes(uint32_t d, bool pv, bool pa) {
  size_t rs = row_stride(d);
  size_t b = align16((size_t)d * 4);                 // list
  b += align16((size_t)d * rs * 8);                  // rows
  if (pv) b += align16((size_t)d * rs * 8);          // colT
  if (pv) b += align16((size_t)d * 8);               // cnt
  if (pa) b += align16((size_t)d * 8);               // per-arc sums
  b += align16(((size_t)d + 1) * 4);                 // pair prefix
  return b;
}
constexpr size_t kBlockMisc = 256;  // block scalars (counters, reduction slots)
__host__ __device__ inline size_t light_slot_bytes(bool pv, bool pa) { return root_bytes(kLightMax, pv, pa); }

// Process-wide count of kernel launches issued by this library.
void note_launch(unsigned n = 1);

// Launch helpers implemented in kc_count.cu / kc_orient.cu
cudaError_t launch_count(const CountArgs &a, bool pv, bool pa, int grid, size_t smem, cudaStream_t s);
int count_blocks_per_sm(bool pv, bool pa, size_t smem);
cudaError_t set_count_smem(bool pv, bool pa, size_t smem);

cudaError_t exclusive_scan_u32(const uint32_t *in, uint64_t *out, size_t n, uint64_t *tmp, size_t tmp_elems,
                               cudaStream_t s);
size_t scan_tmp_elems(size_t n);

}  // namespace kc
