// The opaque oriented-graph handle behind kc_dag* (include/kclique.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

struct kc_dag {
  uint32_t n = 0;
  uint64_t m = 0;
  uint32_t max_out = 0;
  uint64_t *ptr = nullptr;    // n+1
  uint32_t *col = nullptr;    // m
  uint32_t *order = nullptr;  // n, roots by out-degree descending
  uint64_t *key = nullptr;    // n, the ranking key: v precedes w iff (key[v], v) < (key[w], w)
  std::vector<uint64_t> ge;   // ge[t] = #roots with out-degree >= t, t = 0 .. max_out+1
  // dense core (kc_core.cu), absent when core_n = 0: core_id[v] in [0, core_n)
  // or kNoCore; core_bits = core_n rows of core_words words
  uint32_t *core_id = nullptr;
  uint64_t *core_bits = nullptr;
  uint32_t core_n = 0, core_words = 0;
  uint64_t build_volume = 0;  // sum over arcs u->x of d+(x), when computed
  cudaStream_t stream = nullptr;
  int device = 0;
};
