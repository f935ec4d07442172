// Host-side dispatch of the counting kernels (kc_count_impl.cuh holds the
// kernels; kc_count_v*.cu instantiate the four variants).
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <tuple>
#include <utility>

#include "kc_internal.cuh"

namespace kc {

template <bool PV, bool PA>
cudaError_t occupancy_variant(size_t block_smem, int *block_per_sm, int *warp_per_sm);
template <bool PV, bool PA>
cudaError_t launch_variant(const CountArgs &a, int block_grid, int warp_grid, size_t block_smem, cudaStream_t s);
extern template cudaError_t occupancy_variant<false, false>(size_t, int *, int *);
extern template cudaError_t occupancy_variant<false, true>(size_t, int *, int *);
extern template cudaError_t occupancy_variant<true, false>(size_t, int *, int *);
extern template cudaError_t occupancy_variant<true, true>(size_t, int *, int *);
extern template cudaError_t launch_variant<false, false>(const CountArgs &, int, int, size_t, cudaStream_t);
extern template cudaError_t launch_variant<false, true>(const CountArgs &, int, int, size_t, cudaStream_t);
extern template cudaError_t launch_variant<true, false>(const CountArgs &, int, int, size_t, cudaStream_t);
extern template cudaError_t launch_variant<true, true>(const CountArgs &, int, int, size_t, cudaStream_t);

size_t block_root_smem(uint32_t dsmem, bool pv, bool pa) {
  return (size_t)kRootWarps * slot_layout(pv).bytes + (dsmem ? root_layout(dsmem, pv, pa).bytes : 0);
}

uint32_t block_root_capacity(size_t smem_budget, bool pv, bool pa) {
  uint32_t d = kLightMax;
  while (d < 4096 && block_root_smem(d + 1, pv, pa) <= smem_budget) ++d;
  return d;
}

cudaError_t count_occupancy(bool pv, bool pa, size_t block_smem, int *block_per_sm, int *warp_per_sm) {
  // the answer depends only on (device, variant, shared-memory size): cached,
  // since repeated passes (peeling rounds, served requests) ask again and again
  static std::mutex mu;
  static std::map<std::tuple<int, int, size_t>, std::pair<int, int>> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const auto key = std::make_tuple(dev, (pv ? 2 : 0) | (pa ? 1 : 0), block_smem);
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      *block_per_sm = it->second.first;
      *warp_per_sm = it->second.second;
      return cudaSuccess;
    }
  }
  if (pv) e = pa ? occupancy_variant<true, true>(block_smem, block_per_sm, warp_per_sm)
                 : occupancy_variant<true, false>(block_smem, block_per_sm, warp_per_sm);
  else e = pa ? occupancy_variant<false, true>(block_smem, block_per_sm, warp_per_sm)
              : occupancy_variant<false, false>(block_smem, block_per_sm, warp_per_sm);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = std::make_pair(*block_per_sm, *warp_per_sm);
  }
  return e;
}

cudaError_t launch_count(const CountArgs &a, bool pv, bool pa, int block_grid, int warp_grid, size_t block_smem,
                         cudaStream_t s) {
  if (pv) return pa ? launch_variant<true, true>(a, block_grid, warp_grid, block_smem, s)
                    : launch_variant<true, false>(a, block_grid, warp_grid, block_smem, s);
  return pa ? launch_variant<false, true>(a, block_grid, warp_grid, block_smem, s)
            : launch_variant<false, false>(a, block_grid, warp_grid, block_smem, s);
}

}  // namespace kc
