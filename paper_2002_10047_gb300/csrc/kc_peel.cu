// arb-peel (Algorithm 2, Section 4.1): exact k-clique densest-subgraph
// peeling, seeded by the per-vertex counts of arb-count-v; and
// arb-approx-peel (Section 4.2), which removes every vertex with at most
// k(1+eps) times the current density in k-cliques each round.
//
// Every round peels all live vertices of minimum current k-clique count (the
// set A). Update recounts only what A removes: for each v in A it counts the
// (k-1)-cliques of I(v) = {live neighbours of v} plus {neighbours of v in A
// ranked after v}, so a clique holding several members of A is counted once,
// at its lowest-ranked member of A. Those counts run on the same persistent
// counting kernels as arb-count, with v as the root and I(v), sorted by rank,
// as its candidate row; the per-vertex credits of that pass are subtracted
// from the live members' counts. The density of what remains after each
// round is compared exactly, as a fraction, with the best so far.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "kc_host.cuh"
#include "kc_orient.cuh"

namespace kc {
namespace {

constexpr uint32_t kAlive = 0xffffffffu;
constexpr int kPeelBlock = 256;

__device__ __forceinline__ bool rank_lt(uint64_t ka, uint32_t a, uint64_t kb, uint32_t b) {
  return ka < kb || (ka == kb && a < b);
}

// largest row length of a CSR
__global__ void row_len_max_kernel(const uint64_t *__restrict__ rp, uint32_t n, unsigned *out) {
  unsigned m = 0;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned)(rp[v + 1] - rp[v]));
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

// smallest current count among live vertices
__global__ void peel_min_kernel(const unsigned long long *__restrict__ C, const uint32_t *__restrict__ round,
                                uint32_t n, unsigned long long *minv) {
  unsigned long long m = ~0ull;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    if (round[v] == kAlive && C[v] < m) m = C[v];
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
    m = y < m ? y : m;
  }
  if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(minv, m);
}

// A = live vertices whose count is at most the threshold (the minimum for
// arb-peel, so exactly the vertices at the minimum; k(1+eps) times the
// density for arb-approx-peel); they get this round's index. The threshold
// is read from thr_ptr when it is given, else thr_value.
__global__ void peel_mark_kernel(const unsigned long long *__restrict__ C, uint32_t *__restrict__ round, uint32_t n,
                                 const unsigned long long *thr_ptr, unsigned long long thr_value, uint32_t r,
                                 uint32_t *__restrict__ A, unsigned *nA) {
  const unsigned long long mv = thr_ptr ? *thr_ptr : thr_value;
  for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += (size_t)gridDim.x * blockDim.x)
    if (round[v] == kAlive && C[v] <= mv) {
      round[v] = r;
      A[atomicAdd(nA, 1u)] = (uint32_t)v;
    }
}

__device__ __forceinline__ bool in_I(uint32_t u, uint32_t v, uint64_t kv, const uint32_t *round, const uint64_t *key,
                                     uint32_t r) {
  const uint32_t ru = round[u];
  return ru == kAlive || (ru == r && rank_lt(kv, v, key[u], u));
}

// |I(v)| for every v in A (one warp per member of A)
__global__ void peel_len_kernel(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                const uint64_t *__restrict__ key, const uint32_t *__restrict__ round,
                                const uint32_t *__restrict__ A, uint32_t nA, uint32_t r, uint32_t *__restrict__ len,
                                unsigned *maxlen) {
  const unsigned lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t q = w0; q < nA; q += nw) {
    const uint32_t v = A[q];
    const uint64_t kv = key[v], e1 = rp[v + 1];
    unsigned c = 0;
    for (uint64_t e = rp[v] + lane; e < e1; e += 32) c += in_I(col[e], v, kv, round, key, r) ? 1u : 0u;
    c = __reduce_add_sync(0xffffffffu, c);
    if (lane == 0) {
      len[q] = c;
      atomicMax(maxlen, c);
    }
  }
}

// the rows I(v) (in the CSR's id order; sorted by rank afterwards)
__global__ void peel_fill_kernel(const uint64_t *__restrict__ rp, const uint32_t *__restrict__ col,
                                 const uint64_t *__restrict__ key, const uint32_t *__restrict__ round,
                                 const uint32_t *__restrict__ A, uint32_t nA, uint32_t r,
                                 const uint64_t *__restrict__ rptr, uint32_t *__restrict__ rcol) {
  const unsigned lane = threadIdx.x & 31;
  const size_t w0 = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
  const size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
  for (size_t q = w0; q < nA; q += nw) {
    const uint32_t v = A[q];
    const uint64_t kv = key[v], e0 = rp[v], e1 = rp[v + 1];
    uint64_t out = rptr[q];
    const uint64_t end = rptr[q + 1];
    for (uint64_t b = e0; b < e1; b += 32) {  // warp-uniform trip count
      const uint64_t e = b + lane;
      uint32_t u = 0;
      bool inc = false;
      if (e < e1) {
        u = col[e];
        inc = in_I(u, v, kv, round, key, r);
      }
      const unsigned m = __ballot_sync(0xffffffffu, inc);
      const uint64_t at = out + (unsigned)__popc(m & ((1u << lane) - 1u));
      if (inc && at < end) rcol[at] = u;
      out += (unsigned)__popc(m);
    }
  }
}

// subtract the credits of this round from the live vertices' counts and
// clear the credit array where it was written (each entry is taken once)
__global__ void peel_apply_kernel(unsigned long long *__restrict__ C, unsigned long long *__restrict__ dec,
                                  const uint32_t *__restrict__ round, const uint32_t *__restrict__ rcol, uint64_t nr,
                                  const uint32_t *__restrict__ A, uint32_t nA, unsigned *status) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nr + nA; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t x = i < nr ? rcol[i] : A[i - nr];
    const unsigned long long val = atomicExch(&dec[x], 0ull);
    if (val && round[x] == kAlive) {
      if (val > C[x]) {
        atomicOr(status, ST_CAPACITY);  // counts inconsistent: cannot happen with exact counts
        continue;
      }
      C[x] -= val;
    }
  }
}

// end of a round's Update: the cliques it removed and its counting pass's
// status go to the peel's running totals, read back with the next round's
// |A| (one host synchronisation fewer per round)
__global__ void peel_epilogue_kernel(const unsigned long long *__restrict__ cwork, unsigned long long *removed,
                                     unsigned *status) {
  const unsigned long long t = cwork[0];
  const unsigned long long old = *removed;
  *removed = old + t;
  unsigned st = (unsigned)cwork[1];
  if (old + t < old) st |= ST_OVERFLOW;
  if (st) *status |= st;
}

unsigned grid_for(size_t work, int block) {
  size_t g = (work + block - 1) / block;
  g = std::max<size_t>(1, std::min<size_t>(g, (size_t)sm_count() * 32));
  return (unsigned)g;
}

// 128-bit a*b > c*d for the density comparison
bool frac_gt(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
  return (unsigned __int128)a * b > (unsigned __int128)c * d;
}

}  // namespace
}  // namespace kc

namespace {

// Both peels; approx selects arb-approx-peel with epsilon = eps_num / eps_den.
kc_status peel_run(const kc_csr *g, const kc_dag *d, int k, bool approx, uint64_t eps_num, uint64_t eps_den,
                   uint32_t *d_round, kc_peel_result *out, cudaStream_t s) {
  using namespace kc;
  if (!g || !d || !out || k < 3 || k > KC_KMAX) return KC_EINVAL;
  if (approx && eps_den == 0) return KC_EINVAL;
  if (g->n != d->n || g->nnz != 2 * d->m) return KC_EINVAL;
  const uint32_t n = d->n;
  memset(out, 0, sizeof *out);
  if (n == 0) return KC_OK;
  if (!d_round || !g->d_row_ptr || !d->key) return KC_EINVAL;
  if (d->max_out > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;

  DevBuf C, dec, A, len, rptr, rcol, scan_tmp, work, rorder;
  KC_CK(C.alloc(sizeof(unsigned long long) * n, s));
  KC_CK(dec.alloc(sizeof(unsigned long long) * n, s));
  KC_CK(A.alloc(sizeof(uint32_t) * n, s));
  KC_CK(len.alloc(sizeof(uint32_t) * n, s));
  KC_CK(rptr.alloc(sizeof(uint64_t) * ((size_t)n + 1), s));
  KC_CK(rcol.alloc(sizeof(uint32_t) * std::max<uint64_t>(g->nnz, 1), s));
  KC_CK(rorder.alloc(sizeof(uint32_t) * n, s));
  const size_t te = scan_tmp_elems(n);
  KC_CK(scan_tmp.alloc(sizeof(uint64_t) * te, s));
  KC_CK(work.alloc(64, s));  // min @0, |A| @8, max |I| @12, status @16, cliques removed @24
  // per-round buffers, sized once: the length histogram (|I(v)| <= the
  // largest degree), the counting pass's work block, and global scratch
  // grown on demand for rows too long for shared memory
  uint32_t maxdeg = 0;
  {
    DevBuf dmax;
    KC_CK(dmax.alloc(sizeof(unsigned), s));
    KC_CK(cudaMemsetAsync(dmax.p, 0, sizeof(unsigned), s));
    row_len_max_kernel<<<grid_for(n, kPeelBlock), kPeelBlock, 0, s>>>(g->d_row_ptr, n, dmax.as<unsigned>());
    note_launch();
    KC_CK(cudaGetLastError());
    KC_CK(cudaMemcpyAsync(&maxdeg, dmax.p, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
  }
  DevBuf hist, cwork, scratch;
  size_t scratch_cap = 0;
  KC_CK(hist.alloc(sizeof(unsigned) * ((size_t)maxdeg + 1), s));
  KC_CK(cwork.alloc(kc_work_bytes(), s));
  uint8_t *w = work.as<uint8_t>();
  unsigned long long *d_min = (unsigned long long *)w;
  unsigned *d_nA = (unsigned *)(w + 8), *d_maxlen = (unsigned *)(w + 12), *d_status = (unsigned *)(w + 16);
  unsigned long long *d_removed = (unsigned long long *)(w + 24);  // cliques removed by all Updates so far
  KC_CK(cudaMemsetAsync(dec.p, 0, sizeof(unsigned long long) * n, s));
  KC_CK(cudaMemsetAsync(d_round, 0xff, sizeof(uint32_t) * n, s));
  KC_CK(cudaMemsetAsync(w + 16, 0, 16, s));

  // the seed: per-vertex counts of the whole graph (arb-count-v)
  uint64_t total = 0;
  kc_status st = run_count(d, k, C.as<unsigned long long>(), nullptr, &total, 0, s);
  if (st != KC_OK) return st;

  uint64_t t_rem = total, f = 0;
  uint64_t best_num = total, best_den = n;
  uint32_t best_rounds = 0, r = 0;
  std::vector<unsigned> start;
  // the round whose Update's result is read back with the next round's |A|
  bool pending = false;
  uint64_t pending_f = 0;
  struct Readback {
    unsigned long long min;
    unsigned nA, maxlen, status, pad;
    unsigned long long removed;
  } hw{};
  // applies a readback: the removed cliques of the rounds so far give the
  // remaining count, and the pending round's density is compared
  auto settle = [&]() -> kc_status {
    const kc_status cs = status_code(hw.status);
    if (cs != KC_OK) return cs;
    if (hw.removed > total) return KC_ECUDA;  // removed more cliques than there were: cannot happen
    t_rem = total - hw.removed;
    if (pending) {
      if (pending_f < n && frac_gt(t_rem, best_den, best_num, n - pending_f)) {
        best_num = t_rem;
        best_den = n - pending_f;
        best_rounds = r;
      }
      pending = false;
    }
    return KC_OK;
  };
  while (f < n) {
    KC_CK(cudaMemsetAsync(w + 8, 0, 8, s));
    if (approx) {
      // the threshold needs the remaining count now
      KC_CK(cudaMemcpyAsync(&hw, w, sizeof hw, cudaMemcpyDeviceToHost, s));
      KC_CK(cudaStreamSynchronize(s));
      if ((st = settle()) != KC_OK) return st;
      // threshold floor(k (1 + eps) t / |S|) with S the remaining vertices,
      // exact in 128-bit integers: k (den + num) t / (|S| den)
      const unsigned __int128 num = (unsigned __int128)(uint64_t)k * (eps_den + eps_num) * t_rem;
      const unsigned __int128 q = num / ((unsigned __int128)(n - f) * eps_den);
      const unsigned long long thr = q > (unsigned __int128)~0ull ? ~0ull : (unsigned long long)q;
      peel_mark_kernel<<<grid_for(n, kPeelBlock), kPeelBlock, 0, s>>>(C.as<unsigned long long>(), d_round, n,
                                                                      nullptr, thr, r, A.as<uint32_t>(), d_nA);
      note_launch();
    } else {
      KC_CK(cudaMemsetAsync(d_min, 0xff, 8, s));
      peel_min_kernel<<<grid_for(n, kPeelBlock), kPeelBlock, 0, s>>>(C.as<unsigned long long>(), d_round, n, d_min);
      note_launch();
      peel_mark_kernel<<<grid_for(n, kPeelBlock), kPeelBlock, 0, s>>>(C.as<unsigned long long>(), d_round, n, d_min,
                                                                      0ull, r, A.as<uint32_t>(), d_nA);
      note_launch();
    }
    // |A|, and the cliques removed by the Updates so far (the last round's too)
    KC_CK(cudaMemcpyAsync(&hw, w, sizeof hw, cudaMemcpyDeviceToHost, s));
    KC_CK(cudaStreamSynchronize(s));
    if ((st = settle()) != KC_OK) return st;
    const unsigned h_nA = hw.nA;
    if (h_nA == 0) return KC_ECUDA;  // no live vertex found although f < n: cannot happen
    f += h_nA;
    if (t_rem > 0) {
      // Update (Algorithm 2): the k-cliques that A removes
      peel_len_kernel<<<grid_for((size_t)h_nA * 32, kPeelBlock), kPeelBlock, 0, s>>>(
          g->d_row_ptr, g->d_col, d->key, d_round, A.as<uint32_t>(), h_nA, r, len.as<uint32_t>(), d_maxlen);
      note_launch();
      KC_CK(exclusive_scan_u32(len.as<uint32_t>(), rptr.as<uint64_t>(), h_nA, scan_tmp.as<uint64_t>(), te, s));
      // the rows and the histogram of their lengths (|I(v)| <= the largest
      // degree) before the one read-back of the sizes
      peel_fill_kernel<<<grid_for((size_t)h_nA * 32, kPeelBlock), kPeelBlock, 0, s>>>(
          g->d_row_ptr, g->d_col, d->key, d_round, A.as<uint32_t>(), h_nA, r, rptr.as<uint64_t>(),
          rcol.as<uint32_t>());
      note_launch();
      KC_CK(cudaMemsetAsync(hist.p, 0, sizeof(unsigned) * ((size_t)maxdeg + 1), s));
      KC_CK(launch_outdeg_hist(rptr.as<uint64_t>(), h_nA, hist.as<unsigned>(), maxdeg, s));
      uint64_t h_nr = 0;
      unsigned h_maxlen = 0;
      std::vector<unsigned> h_hist((size_t)maxdeg + 1);
      KC_CK(cudaMemcpyAsync(&h_nr, rptr.as<uint64_t>() + h_nA, 8, cudaMemcpyDeviceToHost, s));
      KC_CK(cudaMemcpyAsync(&h_maxlen, d_maxlen, 4, cudaMemcpyDeviceToHost, s));
      KC_CK(cudaMemcpyAsync(h_hist.data(), hist.p, sizeof(unsigned) * h_hist.size(), cudaMemcpyDeviceToHost, s));
      KC_CK(cudaStreamSynchronize(s));
      if (h_nr > g->nnz) return KC_ECUDA;
      if (h_maxlen > maxdeg) return KC_ECUDA;  // |I(v)| <= deg(v): cannot happen
      if (h_maxlen + 1 >= (unsigned)k && h_nr > 0) {
        if (h_maxlen > KC_MAX_OUT_DEGREE) return KC_ECAPACITY;
        // rows by length, descending (the counting kernels' root order), then
        // each row into rank order
        kc_dag rows;  // the round's rows in the shape the planner reads
        rows.n = n;
        rows.m = h_nr;
        rows.max_out = h_maxlen;
        rows.ptr = d->ptr;
        rows.col = d->col;
        rows.order = rorder.as<uint32_t>();
        // candidate rows are subsets of out-lists, sorted by rank: the DAG's
        // dense core serves their builds as it serves the out-lists'
        rows.core_id = d->core_id;
        rows.core_bits = d->core_bits;
        rows.core_words = d->core_words;
        rows.core_n = d->core_n;
        rows.ge.assign((size_t)h_maxlen + 2, 0);
        for (int64_t t = h_maxlen; t >= 0; --t) rows.ge[t] = rows.ge[t + 1] + h_hist[t];
        // `start` outlives the copy: it is rewritten only after the next
        // read-back, which completes after every earlier copy on the stream
        start.assign((size_t)h_maxlen + 1, 0u);
        for (uint32_t t = 0; t <= h_maxlen; ++t) start[t] = (unsigned)rows.ge[t + 1];
        KC_CK(cudaMemcpyAsync(hist.p, start.data(), sizeof(unsigned) * start.size(), cudaMemcpyHostToDevice, s));
        KC_CK(launch_outdeg_scatter(rptr.as<uint64_t>(), h_nA, hist.as<unsigned>(), h_maxlen, rorder.as<uint32_t>(), s));
        auto ge = [&](uint64_t t) -> uint32_t { return t < rows.ge.size() ? (uint32_t)rows.ge[t] : 0u; };
        KC_CK(launch_sort_rows(rptr.as<uint64_t>(), rcol.as<uint32_t>(), d->key, rorder.as<uint32_t>(), ge(1025), ge(33),
                               ge(2), h_maxlen, s));
        LaunchPlan P;
        KC_CK(plan_count(&rows, k, true, false, nullptr, &P));
        CountArgs &a = P.a;
        a.rptr = rptr.as<uint64_t>();
        a.rcol = rcol.as<uint32_t>();
        a.rvert = A.as<uint32_t>();
        a.pv = dec.as<unsigned long long>();
        KC_CK(cudaMemsetAsync(cwork.p, 0, kc_work_bytes(), s));
        set_work(&a, cwork.as<uint8_t>());
        if (P.scratch_bytes) {
          if (P.scratch_bytes > scratch_cap) {
            if (scratch.p) cudaFreeAsync(scratch.release(), s);
            KC_CK(scratch.alloc(P.scratch_bytes, s));
            scratch_cap = P.scratch_bytes;
          }
          a.scratch = scratch.as<uint8_t>();
        }
        if (a.n_light_end > 0) KC_CK(launch_count(a, true, false, P.block_grid, P.warp_grid, P.block_smem, s));
        peel_apply_kernel<<<grid_for(h_nr + h_nA, kPeelBlock), kPeelBlock, 0, s>>>(
            C.as<unsigned long long>(), dec.as<unsigned long long>(), d_round, rcol.as<uint32_t>(), h_nr,
            A.as<uint32_t>(), h_nA, d_status);
        note_launch();
        peel_epilogue_kernel<<<1, 1, 0, s>>>(cwork.as<unsigned long long>(), d_removed, d_status);
        note_launch();
        KC_CK(cudaGetLastError());
      }
    }
    ++r;
    pending = true;
    pending_f = f;
    if (f >= n) break;
  }
  // the last round's Update
  KC_CK(cudaMemcpyAsync(&hw, w, sizeof hw, cudaMemcpyDeviceToHost, s));
  KC_CK(cudaStreamSynchronize(s));
  if ((st = settle()) != KC_OK) return st;
  out->rounds = r;
  out->best_rounds = best_rounds;
  out->best_cliques = best_num;
  out->best_vertices = best_den;
  out->total = total;
  return KC_OK;
}

}  // namespace

extern "C" kc_status kc_peel(const kc_csr *g, const kc_dag *d, int k, uint32_t *d_round, kc_peel_result *out,
                             kc_stream_t stream) {
  return peel_run(g, d, k, false, 0, 1, d_round, out, (cudaStream_t)stream);
}

extern "C" kc_status kc_peel_approx(const kc_csr *g, const kc_dag *d, int k, uint32_t eps_num, uint32_t eps_den,
                                    uint32_t *d_round, kc_peel_result *out, kc_stream_t stream) {
  return peel_run(g, d, k, true, eps_num, eps_den, d_round, out, (cudaStream_t)stream);
}
