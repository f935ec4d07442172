// Internal declarations shared by the libkclique translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kclique.h"

namespace kc {

// Device status word bits (or-ed by kernels, read by the host after a launch).
enum : unsigned {
  ST_OVERFLOW = 1u,   // a count wrapped uint64
  ST_BAD_CSR = 2u,    // validation failed
  ST_TIMEOUT = 4u,    // deadline / cancel
  ST_CAPACITY = 8u,   // an internal capacity check failed (the access was skipped)
  ST_BAD_ARG = 16u,   // a per-graph k of a batch outside [3, KC_KMAX]
  ST_STALL = 32u,     // a bulk copy did not complete within its bounded wait
};

constexpr uint32_t kNoCore = 0xffffffffu;  // core number of a vertex outside the dense core (kc_core.cu)
constexpr int kBlock = 256;              // threads per block of the orientation kernels
constexpr int kWarps = kBlock / 32;
constexpr int kRootBlock = 512;          // threads per block of the block-root counting kernel
constexpr int kRootWarps = kRootBlock / 32;
constexpr int kLightMax = 64;            // roots with d+ <= 64 use one warp and one-word rows
constexpr int kMaxFrames = KC_KMAX - 2;  // depth of the explicit DFS stack
constexpr int kCompactMax = 128;         // largest candidate set compacted to local ids
constexpr int kCompactWords = 32;        // compaction needs the root's rows to fit 32 words (d+ <= 2048)

__host__ __device__ inline uint32_t words_of(uint32_t d) { return (d + 63u) / 64u; }
__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline uint32_t hash_slots(uint32_t d) {
  uint32_t t = 64;
  while (t < 2 * d) t <<= 1;
  return t;
}

// Positions inside N+(u) follow the total order (out-lists are sorted by
// rank), so an arc between positions i < t always points from i to t and one
// symmetric bit matrix holds both directions.
//
// Per-root working set of a block-level root with out-degree d:
//   L      uint32[d]        N+(u), in rank order
//   rb, rl uint64/uint32[d] start and length of N+(L[i]) in the DAG
//   hslot  uint64[T]        open-addressing table: (vertex id << 16 | position in L)
//   adj    uint64[d*W]      the DAG induced on N+(u), symmetric: bit t of row i
//                           <=> L[i] and L[t] adjacent (i < t: arc i -> t)
//   cnt    uint64[d]        per-vertex counters (per-vertex only)
//   asub   uint64[d]        per-arc sums (per-arc only)
//   pre    uint32[d+1]      prefix of split-arc sizes (k >= 6)
struct RootLayout {
  size_t L, rb, rl, hslot, adj, cnt, asub, pre, bytes;
};
__host__ __device__ inline RootLayout root_layout(uint32_t d, bool pv, bool pa) {
  RootLayout o;
  const uint32_t W = words_of(d), T = hash_slots(d);
  size_t off = 0;
  o.L = off; off += align16((size_t)d * 4);
  o.rb = off; off += align16((size_t)d * 8);
  o.rl = off; off += align16((size_t)d * 4);
  o.hslot = off; off += align16((size_t)T * 8);
  o.adj = off; off += align16((size_t)d * W * 8);
  o.cnt = off; if (pv) off += align16((size_t)d * 8);
  o.asub = off; if (pa) off += align16((size_t)d * 8);
  o.pre = off; off += align16(((size_t)d + 1) * 4);
  o.bytes = off;
  return o;
}

// Per-warp slot of the block-root kernel (item scratch): mask words and their
// prefix counts, the root positions of the compacted vertices, the compacted
// symmetric rows, and local per-vertex counters.
struct SlotLayout {
  size_t mask, pfx, P, S, cs, bytes;
};
__host__ __device__ inline SlotLayout slot_layout(bool pv) {
  SlotLayout o;
  size_t off = 0;
  o.mask = off; off += 32 * 8;
  o.pfx = off; off += 33 * 4;
  off = align16(off);
  o.P = off; off += align16(kCompactMax * 2);
  o.S = off; off += kCompactMax * 2 * 8;
  o.cs = off; if (pv) off += kCompactMax * 8;
  o.bytes = align16(off);
  return o;
}

// Per-warp slot of the warp-root kernel (roots with d+ <= 64).
struct LightLayout {
  size_t L, rb, hkey, hpos, adj, cnt, asub, pre, epre, bytes;
};
__host__ __device__ inline LightLayout light_layout(bool pv, bool pa) {
  LightLayout o;
  size_t off = 0;
  o.L = off; off += kLightMax * 4;
  o.rb = off; off += kLightMax * 8;
  o.hkey = off; off += 128 * 4;
  o.hpos = off; off += 128 * 2;
  o.adj = off; off += kLightMax * 8;
  o.cnt = off; if (pv) off += kLightMax * 8;
  o.asub = off; if (pa) off += kLightMax * 8;
  o.pre = off; off += align16((kLightMax + 1) * 4);
  o.epre = off; off += align16((kLightMax + 1) * 4);
  o.bytes = align16(off);
  return o;
}

struct CountArgs {
  const uint64_t *ptr;       // DAG offsets, n+1
  const uint32_t *col;       // DAG out-lists, m
  const uint32_t *order;     // roots sorted by out-degree, descending
  uint32_t n_big;            // order[0, n_big): d+ above the light threshold (block roots)
  uint32_t n_scratch;        // order[0, n_scratch): block roots whose matrices live in global scratch
  uint32_t n_light_end;      // order[n_big, n_light_end): k-1 <= d+ <= light threshold <= kLightMax (warp roots)
  int k;
  unsigned long long *total; // global sum
  unsigned long long *pv;    // per-vertex output (n) or null
  unsigned long long *pa;    // per-arc output (m) or null
  unsigned *status;
  unsigned *queue;           // [0] scratch roots, [1] shared-memory block roots, [2] warp roots
  uint8_t *scratch;          // global slabs for roots that do not fit shared memory
  size_t scratch_stride;     // bytes per slab
  uint32_t scratch_blocks;   // blocks that take scratch roots
  uint64_t deadline_ns;      // globaltimer deadline, 0 = none
  // set for a pass with a time budget: the deadline written on the device by
  // the kernel that starts the pass (takes the place of deadline_ns)
  const unsigned long long *deadline_dev;
  // level-2 build of block roots: stage the members' out-lists with bulk
  // copies (kc_set_bulk_build)
  uint32_t bulk_build;
  // batches of disjoint graphs (null for a single graph): graph g owns
  // vertices [goff[g], goff[g+1]), counts its gk[g]-cliques, sums into gtotal[g]
  const uint64_t *goff;
  const uint8_t *gk;
  unsigned long long *gtotal;
  uint32_t ngraphs;
  // tunables (kc_params; 0 = default): largest candidate set compacted
  // (<= kCompactMax), roots a warp takes per queue pull in the warp-root kernel
  uint32_t compact_max;
  uint32_t chunk;
  // warp roots in vertex-id order instead of the order array: the roots
  // u < n with light_min <= d+(u) <= light_max (queue[2] counts pulls of
  // 32*chunk ids)
  uint32_t light_by_id;
  uint32_t n;
  uint32_t light_min, light_max;
  // peeling: root q's candidate row is rcol[rptr[q] .. rptr[q+1]) (sorted
  // by rank) and its vertex is rvert[q]; order[] then lists row indices.
  // Members' rows are still the DAG's. Null: roots are vertices.
  const uint64_t *rptr;
  const uint32_t *rcol;
  const uint32_t *rvert;
  // rooted counts of a root list (null otherwise): the root at position i of
  // the order array writes its total to rooted[rooted_pos[i]]
  unsigned long long *rooted;
  const uint32_t *rooted_pos;
  // dense core (kc_core.cu; null: none): core_id[v] numbers the core
  // vertices, core_bits row a (core_words words) has bit b set iff core
  // vertex a has an arc to core vertex b. A member x_i of N+(u) whose
  // out-list holds at least core_ratio entries per later member takes its
  // row of the induced subgraph from core_bits.
  const uint32_t *core_id;
  const unsigned long long *core_bits;
  uint32_t core_words;
  uint32_t core_ratio;
};

// A configured counting pass (kc_api.cu).
struct LaunchPlan {
  CountArgs a;
  int block_grid, warp_grid;
  size_t block_smem, scratch_bytes;
  uint32_t dcap;   // largest out-degree whose root matrix fits shared memory
  uint32_t light;  // largest out-degree of a warp root
};

// Process-wide count of kernel launches issued by this library.
void note_launch(unsigned n = 1);

// Process-wide choice of the block-root build: bulk-copy staging or direct loads.
bool bulk_build_enabled();

// Every stream-ordered device allocation of the library goes through here
// (cudaMallocAsync, or the injected failure set by
// kc_debug_fail_allocations_after).
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s);

// Launch helpers implemented in kc_count.cu / kc_orient.cu
size_t block_root_smem(uint32_t dsmem, bool pv, bool pa);
uint32_t block_root_capacity(size_t smem_budget, bool pv, bool pa);
cudaError_t launch_count(const CountArgs &a, bool pv, bool pa, int block_grid, int warp_grid, size_t block_smem,
                         cudaStream_t s);
cudaError_t count_occupancy(bool pv, bool pa, size_t block_smem, int *block_per_sm, int *warp_per_sm);

size_t kc_work_bytes();
void set_work(CountArgs *a, uint8_t *w);

cudaError_t exclusive_scan_u32(const uint32_t *in, uint64_t *out, size_t n, uint64_t *tmp, size_t tmp_elems,
                               cudaStream_t s);
size_t scan_tmp_elems(size_t n);

}  // namespace kc
