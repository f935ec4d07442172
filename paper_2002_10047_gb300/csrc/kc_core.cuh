// Dense-core adjacency of an oriented graph (kc_core.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_dag.cuh"
#include "kclique.h"

namespace kc {

enum : int { kCoreAuto = 0, kCoreForce = 1, kCoreOff = 2 };

struct CorePolicy {
  uint32_t max_vertices;        // largest core (0: never build one)
  uint32_t ratio;               // lookup rule of the counting kernels (UINT32_MAX: never look up)
  uint32_t min_max_out;         // automatic build: largest out-degree at least this
  uint32_t min_volume_per_arc;  // automatic build: build volume at least this many entries per arc
};
CorePolicy core_policy();

// Builds D's core after the out-lists are final (rp: the input CSR's row
// offsets, key: the ranking keys). kCoreAuto builds it where the level-2
// builds read long out-lists on average; kCoreForce always (up to
// max_vertices); kCoreOff never.
kc_status build_core(kc_dag *D, const uint64_t *rp, const uint64_t *key, int mode, cudaStream_t s);

// Out-list entries scanned and core bits looked up by the level-2 builds of
// all roots of D under the current lookup rule (no core: scanned = sum over
// arcs u->x of d+(x), looked = 0).
kc_status core_build_split(const kc_dag *D, uint64_t *scanned, uint64_t *looked, cudaStream_t s);

}  // namespace kc
