// Host-side helpers shared by the C-ABI translation units: CUDA error
// mapping, stream-ordered buffers and the launch planner of a counting pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kc_dag.cuh"
#include "kc_internal.cuh"
#include "kclique.h"

namespace kc {

// Records the CUDA error text for kc_last_cuda_error and maps it to a status.
kc_status cuda_fail(cudaError_t e);
// An internal consistency check failed: records `what` for
// kc_last_cuda_error and returns KC_ECUDA.
kc_status internal_fail(const char *what);
// Device status word (ST_* bits) to the kc_status the caller sees.
kc_status status_code(unsigned st);
int sm_count();

#define KC_CK(call)                                 \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) return kc::cuda_fail(e_); \
  } while (0)

// Stream-ordered device buffer released when the scope ends.
struct DevBuf {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t st) {
    s = st;
    return kc::dev_malloc_async(&p, bytes ? bytes : 16, st);
  }
  template <typename T>
  T *as() const {
    return (T *)p;
  }
  void *release() {
    void *q = p;
    p = nullptr;
    return q;
  }
};

// Kernel configuration for a counting pass over d whose smallest clique size
// is k_min; prm may be null (defaults: warp roots by out-degree). Fills everything in P.a except the
// outputs, the work block and the scratch pointer; P.scratch_bytes is the
// global scratch the largest roots need (0 if none).
cudaError_t plan_count(const kc_dag *d, int k_min, bool pv, bool pa, const kc_params *prm, LaunchPlan *P);

// deadline_ns: absolute globaltimer deadline (0 = none); budget_ns: a time
// budget that starts when the pass starts on the device (0 = none)
kc_status run_count(const kc_dag *d, int k, unsigned long long *pv, unsigned long long *pa, uint64_t *h_total,
                    uint64_t deadline_ns, cudaStream_t s, uint64_t budget_ns = 0);

}  // namespace kc
