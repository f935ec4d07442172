// Wrap-checked 64-bit additions used by every count reduction: a sum that
// does not fit in uint64 sets ST_OVERFLOW in the caller's flag (and the
// entry points report KC_ERANGE) instead of wrapping.
#pragma once
#include <cuda_runtime.h>

#include "kc_internal.cuh"

namespace kc {

__device__ __forceinline__ unsigned long long add_ck(unsigned long long a, unsigned long long b, unsigned &ovf) {
  const unsigned long long s = a + b;
  ovf |= (s < a) ? ST_OVERFLOW : 0u;
  return s;
}

__device__ __forceinline__ void atomic_add_ck(unsigned long long *p, unsigned long long v, unsigned &ovf) {
  if (v == 0) return;
  const unsigned long long old = atomicAdd(p, v);
  ovf |= (old + v < old) ? ST_OVERFLOW : 0u;
}

// warp butterfly sum: if the warp's total fits, no partial sum wraps; if it
// does not, some partial sum does
__device__ __forceinline__ unsigned long long warp_sum64_ck(unsigned long long v, unsigned &ovf) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, v, o);
    const unsigned long long s = v + y;
    ovf |= (s < v) ? ST_OVERFLOW : 0u;
    v = s;
  }
  return v;
}

}  // namespace kc
