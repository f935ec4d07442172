// Calibration: the sustained rate of the counting kernels' unit of work, a
// 64-bit AND followed by a population count ("word operation"), measured on
// the device at hand. The counting passes for k >= 5 are bound by this
// integer work (the intersect of Algorithm 1 on bitsets), so their roofline
// is reported against this measured rate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_internal.cuh"
#include "kclique.h"

namespace kc {

constexpr int kProbeStreams = 8;

// Every thread runs kProbeStreams independent chains of
// acc += popc(a & b); a ^= acc (so the AND/POPC cannot be hoisted).
__global__ void __launch_bounds__(256) word_op_probe_kernel(uint64_t seed, int iters, unsigned long long *sink) {
  uint64_t a[kProbeStreams], b[kProbeStreams];
  unsigned acc[kProbeStreams];
#pragma unroll
  for (int s = 0; s < kProbeStreams; ++s) {
    a[s] = seed * (threadIdx.x + 1 + s) + blockIdx.x;
    b[s] = ~seed ^ ((uint64_t)s << 17) ^ threadIdx.x;
    acc[s] = 0;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int s = 0; s < kProbeStreams; ++s) {
      acc[s] += (unsigned)__popcll(a[s] & b[s]);
      a[s] ^= acc[s];
    }
  }
  unsigned t = 0;
#pragma unroll
  for (int s = 0; s < kProbeStreams; ++s) t += acc[s];
  if (t == 0x7fffffffu) atomicAdd(sink, 1ull);  // keeps the loop live
}

}  // namespace kc

extern "C" kc_status kc_measure_word_op_rate(double *h_rate, kc_stream_t stream) {
  if (!h_rate) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned long long *sink = nullptr;
  if (kc::dev_malloc_async((void **)&sink, 8, s) != cudaSuccess) return KC_ENOMEM;
  cudaMemsetAsync(sink, 0, 8, s);
  const int blocks = sms * 8, threads = 256, iters = 1 << 14;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  kc::word_op_probe_kernel<<<blocks, threads, 0, s>>>(0x9E3779B97F4A7C15ull, 256, sink);  // warm-up
  kc::note_launch();
  cudaEventRecord(e0, s);
  kc::word_op_probe_kernel<<<blocks, threads, 0, s>>>(0x9E3779B97F4A7C15ull, iters, sink);
  kc::note_launch();
  cudaEventRecord(e1, s);
  const cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, s);
  if (err != cudaSuccess || ms <= 0.f) return KC_ECUDA;
  const double ops = (double)blocks * threads * (double)iters * kc::kProbeStreams;
  *h_rate = ops / (ms * 1e-3);
  return KC_OK;
}
