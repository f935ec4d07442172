// Launchers of the orientation-side kernels (kc_orient.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kclique.h"

namespace kc {
cudaError_t launch_validate(const kc_csr &g, int sym, unsigned *status, cudaStream_t s);
cudaError_t launch_degree_key(const kc_csr &g, uint64_t *key, cudaStream_t s);
cudaError_t launch_count_out(const kc_csr &g, const uint64_t *key, uint32_t *outdeg, unsigned *maxdeg,
                             cudaStream_t s);
cudaError_t launch_write_out(const kc_csr &g, const uint64_t *key, const uint64_t *dag_ptr, uint32_t *dag_col,
                             cudaStream_t s);
cudaError_t launch_outdeg_hist(const uint64_t *dp, uint32_t n, unsigned *hist, uint32_t maxd, cudaStream_t s);
cudaError_t launch_outdeg_scatter(const uint64_t *dp, uint32_t n, unsigned *cursor, uint32_t maxd, uint32_t *order,
                                  cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long *out, size_t n, unsigned long long v, cudaStream_t s);
cudaError_t launch_root_outdeg(const uint64_t *dp, const uint32_t *roots, uint32_t r, uint32_t *out,
                               cudaStream_t s);
cudaError_t launch_degree_from_dag(const uint64_t *dp, const uint32_t *dc, uint32_t n, unsigned long long *out,
                                   cudaStream_t s);
// Sort every out-list by (key, id): order[] lists roots by out-degree,
// descending; [0, n_big) have d > 1024, [n_big, n_mid_end) 33..1024,
// [n_mid_end, n_small_end) 2..32 (kc_sortrows.cu)
cudaError_t launch_sort_rows(const uint64_t *ptr, uint32_t *col, const uint64_t *key, const uint32_t *order,
                             uint32_t n_big, uint32_t n_mid_end, uint32_t n_small_end, uint32_t max_out,
                             cudaStream_t s);
// Goodrich-Pszona order keys (kc_gp.cu): okey[v] = round << 32 | degree at removal
kc_status gp_rank(const kc_csr &g, uint64_t *okey, cudaStream_t s);
// Barenboim-Elkin order keys (kc_gp.cu), epsilon = 1, arboricity bound from
// the approximate densest subgraph: okey[v] = round << 32 | degree at removal
kc_status be_rank(const kc_csr &g, uint64_t *okey, cudaStream_t s);
cudaError_t launch_dag_stats(const uint64_t *dp, const uint32_t *dc, uint32_t n, unsigned long long *acc,
                             cudaStream_t s);
}  // namespace kc
