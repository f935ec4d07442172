// Counting kernels, variant per-vertex=true per-arc=true (one translation
// unit per variant so the variants compile in parallel).
#include "kc_count_impl.cuh"

namespace kc {
template cudaError_t occupancy_variant<true, true>(size_t, int *, int *);
template cudaError_t launch_variant<true, true>(const CountArgs &, int, int, size_t, cudaStream_t);
}  // namespace kc
