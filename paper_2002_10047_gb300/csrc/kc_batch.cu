// Batched counting: one pass of the persistent counting kernels over the
// disjoint union of many graphs, each root counting its own graph's k and
// adding into its graph's total (include/kclique.h, "Batches"). A prepared
// plan makes the pass capturable into a CUDA graph; the autotuner picks the
// warp-root order, the warp/block threshold, the compacted bitset width and
// the queue chunk.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "kc_host.cuh"

struct kc_plan {
  kc::LaunchPlan P;
  uint32_t num_graphs = 0;
  uint64_t *totals = nullptr;  // caller's d_totals
  void *work = nullptr;        // owned: total, status, queues
  void *scratch = nullptr;     // owned: slabs for roots beyond shared memory
  cudaStream_t stream = nullptr;
};

namespace {

kc_status check_batch(const kc_dag *d, const kc_batch *b, const kc_params *prm) {
  if (!d || !b || b->num_graphs == 0 || !b->d_vertex_offsets || !b->d_k) return KC_EINVAL;
  if (b->k_min < 3 || b->k_min > KC_KMAX) return KC_EINVAL;
  if (prm && (prm->light_max > (uint32_t)kc::kLightMax || prm->compact_max > (uint32_t)kc::kCompactMax ||
              prm->light_order > KC_LIGHT_BY_ID))
    return KC_EINVAL;
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;
  return KC_OK;
}

}  // namespace

extern "C" {

kc_status kc_plan_create(const kc_dag *d, const kc_batch *b, const kc_params *prm, uint64_t *d_totals,
                         kc_plan **out, kc_stream_t stream) {
  if (!out || !d_totals) return KC_EINVAL;
  const kc_status c = check_batch(d, b, prm);
  if (c != KC_OK) return c;
  cudaStream_t s = (cudaStream_t)stream;
  kc_plan *p = new kc_plan;
  p->num_graphs = b->num_graphs;
  p->totals = d_totals;
  p->stream = s;
  cudaError_t e = kc::plan_count(d, b->k_min, false, false, prm, &p->P);
  if (e == cudaSuccess) e = kc::dev_malloc_async(&p->work, kc::kc_work_bytes(), s);
  if (e == cudaSuccess && p->P.scratch_bytes) e = kc::dev_malloc_async(&p->scratch, p->P.scratch_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->work, 0, kc::kc_work_bytes(), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    kc_plan_free(p);
    return kc::cuda_fail(e);
  }
  kc::CountArgs &a = p->P.a;
  kc::set_work(&a, (uint8_t *)p->work);
  a.scratch = (uint8_t *)p->scratch;
  a.goff = b->d_vertex_offsets;
  a.gk = b->d_k;
  a.gtotal = (unsigned long long *)d_totals;
  a.ngraphs = b->num_graphs;
  *out = p;
  return KC_OK;
}

kc_status kc_plan_launch(kc_plan *p, kc_stream_t stream) {
  if (!p) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  KC_CK(cudaMemsetAsync(p->totals, 0, sizeof(uint64_t) * p->num_graphs, s));
  KC_CK(cudaMemsetAsync(p->work, 0, kc::kc_work_bytes(), s));
  const kc::LaunchPlan &P = p->P;
  if (P.a.n_light_end > 0) KC_CK(kc::launch_count(P.a, false, false, P.block_grid, P.warp_grid, P.block_smem, s));
  return KC_OK;
}

kc_status kc_plan_result(kc_plan *p, uint64_t *h_total, kc_stream_t stream) {
  if (!p) return KC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long h[2] = {0, 0};
  KC_CK(cudaMemcpyAsync(h, p->work, sizeof h, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  const kc_status code = kc::status_code((unsigned)h[1]);
  if (code != KC_OK) return code;
  if (h_total) *h_total = h[0];
  return KC_OK;
}

void kc_plan_free(kc_plan *p) {
  if (!p) return;
  if (p->scratch) cudaFreeAsync(p->scratch, p->stream);
  if (p->work) cudaFreeAsync(p->work, p->stream);
  delete p;
}

kc_status kc_count_batched(const kc_dag *d, const kc_batch *b, const kc_params *prm, uint64_t *d_totals,
                           uint64_t *h_total, kc_stream_t stream) {
  kc_plan *p = nullptr;
  kc_status st = kc_plan_create(d, b, prm, d_totals, &p, stream);
  if (st != KC_OK) return st;
  st = kc_plan_launch(p, stream);
  if (st == KC_OK) st = kc_plan_result(p, h_total, stream);
  kc_plan_free(p);
  return st;
}

kc_status kc_autotune_batched(const kc_dag *d, const kc_batch *b, uint64_t *d_totals, kc_params *out,
                              float *h_best_ms, kc_stream_t stream) {
  if (!out || !d_totals) return KC_EINVAL;
  const kc_status c = check_batch(d, b, nullptr);
  if (c != KC_OK) return c;
  cudaStream_t s = (cudaStream_t)stream;
  static const uint32_t kOrder[] = {KC_LIGHT_BY_ID, KC_LIGHT_BY_DEGREE};
  static const uint32_t kLight[] = {32, 48, 64};
  static const uint32_t kCompact[] = {64, 128};
  static const uint32_t kChunk[] = {1, 4, 16};
  cudaEvent_t e0, e1;
  KC_CK(cudaEventCreate(&e0));
  KC_CK(cudaEventCreate(&e1));
  float best = -1.f;
  kc_params best_p = {0, 0, 0, 0};
  kc_status st = KC_OK;
  for (uint32_t lo : kOrder)
    for (uint32_t lm : kLight)
      for (uint32_t cm : kCompact)
        for (uint32_t ch : kChunk) {
          if (st != KC_OK) break;
          const kc_params prm = {lm, cm, ch, lo};
          kc_plan *p = nullptr;
          st = kc_plan_create(d, b, &prm, d_totals, &p, stream);
          if (st != KC_OK) break;
          st = kc_plan_launch(p, stream);  // warm-up
          if (st == KC_OK) st = kc_plan_result(p, nullptr, stream);
          float ms = 0.f;
          if (st == KC_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && st == KC_OK; ++r) st = kc_plan_launch(p, stream);
            cudaEventRecord(e1, s);
            if (st == KC_OK) st = kc_plan_result(p, nullptr, stream);
            if (st == KC_OK) cudaEventElapsedTime(&ms, e0, e1);
          }
          kc_plan_free(p);
          if (st == KC_OK && (best < 0.f || ms < best)) {
            best = ms;
            best_p = prm;
          }
        }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != KC_OK) return st;
  KC_CK(cudaStreamSynchronize(s));
  *out = best_p;
  if (h_best_ms) *h_best_ms = best * 0.5f;
  return KC_OK;
}

}  // extern "C"
