// Counting kernels, variant per-vertex=true per-arc=false (one translation
// unit per variant so the variants compile in parallel).
#include "kc_count_impl.cuh"

namespace kc {
template cudaError_t occupancy_variant<true, false>(size_t, int *, int *);
template cudaError_t launch_variant<true, false>(const CountArgs &, int, int, size_t, cudaStream_t);
}  // namespace kc
