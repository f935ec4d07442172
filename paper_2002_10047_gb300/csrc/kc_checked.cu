// kc_checked_sum: the counting kernels' wrap-checked 64-bit reduction applied
// to a caller's array. Each thread sums its values with add_ck, and the block
// then ends exactly as every counting kernel does, in finish_block (warp
// butterfly, the warps' sums added by one thread, one checked atomic per
// block). Counts large enough to wrap uint64 cannot be enumerated in test
// time, so this is how the overflow path of the reductions is exercised.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kc_checked.cuh"
#include "kc_count_impl.cuh"
#include "kc_host.cuh"

namespace kc {
namespace {

__global__ void checked_sum_kernel(const unsigned long long *__restrict__ v, uint64_t n, unsigned long long *total,
                                   unsigned *status) {
  __shared__ unsigned long long red[kBlock / 32];
  unsigned ovf = 0;
  unsigned long long acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc = add_ck(acc, v[i], ovf);
  CountArgs a;
  a.total = total;
  a.status = status;
  finish_block(a, acc, ovf, red, kBlock / 32);
}

}  // namespace
}  // namespace kc

extern "C" kc_status kc_checked_sum(const uint64_t *d_values, uint64_t n, uint64_t *h_total, kc_stream_t stream) {
  using namespace kc;
  if (!h_total || (n > 0 && !d_values)) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  DevBuf work;
  KC_CK(work.alloc(16, s));
  KC_CK(cudaMemsetAsync(work.p, 0, 16, s));
  if (n > 0) {
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n + kBlock - 1) / kBlock, (uint64_t)sm_count() * 8));
    checked_sum_kernel<<<grid, kBlock, 0, s>>>((const unsigned long long *)d_values, n, work.as<unsigned long long>(),
                                            (unsigned *)(work.as<uint8_t>() + 8));
    note_launch();
    KC_CK(cudaGetLastError());
  }
  unsigned long long h[2] = {0, 0};
  KC_CK(cudaMemcpyAsync(h, work.p, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  const kc_status st = status_code((unsigned)h[1]);
  if (st != KC_OK) return st;
  *h_total = h[0];
  return KC_OK;
}
