// Counting kernels: arb-count and arb-count-v (Algorithm 1, Section 3.2)
// with the practical optimizations of Section 3.4, laid out for sm_103a.
//
// Every k-clique is found exactly once, below its lowest vertex u in the total
// order (the root), as a (k-1)-clique of the DAG induced on N+(u). For each
// root the team (one warp when d+(u) <= 64, one block otherwise) builds that
// induced subgraph once -- "the induced subgraph on N_DG(v)" of Section 3.4 --
// as a bit matrix over positions 0..d-1 in N+(u) (the relabelling to
// [0, O(alpha)] of Section 3.4). Out-lists are sorted by rank, so position
// order is rank order: an arc between positions i < t points from i to t. One
// matrix (adj) holds the subgraph: its upper triangle (bit t of row i, t > i)
// is the arc set; per-vertex counting also fills the mirrored lower triangle,
// so that row v holds all of v's neighbours. Membership of an out-neighbour in
// N+(u) is found through a shared-memory hash table.
//
// Rec-Count-Cliques (Algorithm 1) runs on bitsets: the candidates are visited
// in increasing position, and when x is taken the candidates still left are
// exactly those ranked after x, so "intersect I with N+(x)" is the remaining
// candidates AND adj[x]; |I| is a population count; the base case l = 1 is
// folded into the level above (l = 2: the number of arcs inside the candidate
// set); a branch is cut when it has fewer candidates than vertices still
// needed.
//
// Work split below the root (edge parallelism, Section 3.4): one warp item per
// arc u->x_i (k <= 5, and k >= 6 when the arc has at most 128 candidates) or
// per triangle u->x_i->x_a (k >= 6 when the arc has more). For k >= 6 the
// item's candidate set is compacted to local ids 0..s-1 (s <= 128, one or two
// words per row) and the warp's lanes split its first level, each running the
// recursion in registers.
//
// Per-vertex counts (arb-count-v): the cliques completed at an l = 2 level of
// candidate set C are the arcs inside C; vertex v in C lies on |C & adj[v]| of
// them. Vertices higher on the path get the totals of their sub-trees and the
// root gets the root total. Counters are flushed to global memory once per
// root. Every addition is checked for uint64 wrap-around.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kc_checked.cuh"
#include "kc_internal.cuh"

namespace kc {

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Adds into a root's (or an item's) local per-vertex counters. No wrap check
// is needed: an entry counts cliques of that root containing the vertex, so
// it never exceeds the root's total, whose additions are checked; the flush
// into the global per-vertex array is checked again.
__device__ __forceinline__ void cnt_add(unsigned long long *p, unsigned long long v) {
  if (v) atomicAdd(p, v);
}

__device__ __forceinline__ unsigned warp_incl_scan(unsigned v) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= (unsigned)o) v += y;
  }
  return v;
}

// bits strictly above position x, restricted to word w
__device__ __forceinline__ uint64_t above_word(uint32_t x, uint32_t w) {
  const uint32_t xw = x >> 6;
  if (w < xw) return 0ull;
  if (w > xw) return ~0ull;
  const uint32_t b = x & 63u;
  return b == 63u ? 0ull : (~0ull << (b + 1u));
}

// ------------------------------------------------------------ hash table
constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ uint32_t hslot(uint32_t y, uint32_t mask) {
  const uint32_t h = y * 2654435761u;
  return (h ^ (h >> 15)) & mask;
}

// keys are distinct and the table has at least twice as many slots as keys
__device__ __forceinline__ void hinsert(uint32_t *hkey, uint16_t *hpos, uint32_t T, uint32_t y, uint32_t pos) {
  uint32_t s = hslot(y, T - 1);
  for (uint32_t probe = 0; probe < T; ++probe) {
    if (atomicCAS(&hkey[s], kEmpty, y) == kEmpty) {
      hpos[s] = (uint16_t)pos;
      return;
    }
    s = (s + 1) & (T - 1);
  }
}

__device__ __forceinline__ int hlookup(const uint32_t *hkey, const uint16_t *hpos, uint32_t T, uint32_t y) {
  uint32_t s = hslot(y, T - 1);
  for (uint32_t probe = 0; probe < T; ++probe) {
    const uint32_t k = hkey[s];
    if (k == y) return hpos[s];
    if (k == kEmpty) return -1;
    s = (s + 1) & (T - 1);
  }
  return -1;
}

// Set bit t of row r (stride W words) for every lane with `hit`, one shared
// atomic per distinct (row, word) of the warp: lanes walking one row would
// otherwise serialise on the same words. Called by all 32 lanes.
__device__ __forceinline__ void warp_set_bits(uint64_t *adj, uint32_t W, bool hit, uint32_t r, uint32_t t) {
  const unsigned lane = lane_id();
  const uint32_t key = r * 256u + (t >> 6);
  unsigned todo = __ballot_sync(0xffffffffu, hit);
  while (todo) {
    const int ld = __ffs(todo) - 1;
    const uint32_t kl = __shfl_sync(0xffffffffu, key, ld);
    const bool mine = hit && key == kl;
    const uint64_t b = mine ? (1ull << (t & 63)) : 0ull;
    const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)b);
    const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(b >> 32));
    if (lane == (unsigned)ld)
      atomicOr((unsigned long long *)&adj[(size_t)r * W + (t >> 6)], ((unsigned long long)hi << 32) | lo);
    todo &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// Packed table (id << 16 | position), one 64-bit load per probe (block roots).
constexpr unsigned long long kEmptySlot = ~0ull;

__device__ __forceinline__ void pinsert(unsigned long long *tab, uint32_t T, uint32_t y, uint32_t pos) {
  uint32_t s = hslot(y, T - 1);
  const unsigned long long v = ((unsigned long long)y << 16) | pos;
  for (uint32_t probe = 0; probe < T; ++probe) {
    if (atomicCAS(&tab[s], kEmptySlot, v) == kEmptySlot) return;
    s = (s + 1) & (T - 1);
  }
}

__device__ __forceinline__ int plookup(const unsigned long long *tab, uint32_t T, uint32_t y) {
  uint32_t s = hslot(y, T - 1);
  for (uint32_t probe = 0; probe < T; ++probe) {
    const unsigned long long v = tab[s];
    if (v == kEmptySlot) return -1;
    if ((uint32_t)(v >> 16) == y) return (int)(v & 0xffffu);
    s = (s + 1) & (T - 1);
  }
  return -1;
}

// ---------------------------------------------------------- DFS engine
// A symmetric bit matrix as the DFS sees it: row x at adj + x*RS, W words in use.
struct MatView {
  const uint64_t *adj;
  unsigned long long *cnt;  // per-vertex counters (per-vertex only)
  unsigned *cnt32;          // 32-bit counters used instead of cnt when set
  uint32_t RS, W;
};

// Adds v to the per-vertex counter of x. The 32-bit counters are used where
// no entry can reach 2^32 (a root with at most 64 out-neighbours at k <= 10,
// a compacted item of at most 128 vertices with at most 6 picks); their
// shared-memory atomics are several times cheaper than 64-bit ones.
__device__ __forceinline__ void credit(const MatView &V, int x, unsigned long long v) {
  if (!v) return;
  if (V.cnt32) atomicAdd(&V.cnt32[x], (unsigned)v);
  else atomicAdd(&V.cnt[x], v);
}

template <int G>
__device__ __forceinline__ unsigned gsum32(unsigned v) {
  if constexpr (G == 1) return v;
  else return __reduce_add_sync(0xffffffffu, v);
}

// Lane j of a G-lane group (G = 1 or 32) holds words r*G + j (r < NW) of a
// set; words at or past W read as zero.
template <int G, int NW>
__device__ __forceinline__ void load_row(const uint64_t *base, uint32_t W, int j, uint64_t (&out)[NW]) {
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    const uint32_t w = (uint32_t)(r * G + j);
    out[r] = (NW == 1 && G == 1) ? base[0] : (w < W ? base[w] : 0ull);
  }
}

// Next set bit of a group-distributed set (ascending); clears it, so T then
// holds exactly the members after x.
template <int G, int NW>
__device__ __forceinline__ bool next_bit(uint64_t (&T)[NW], int j, int &x) {
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    if constexpr (G == 1) {
      if (T[r]) {
        x = r * 64 + __ffsll((long long)T[r]) - 1;
        T[r] &= T[r] - 1;
        return true;
      }
    } else {
      const unsigned bal = __ballot_sync(0xffffffffu, T[r] != 0ull);
      if (bal) {
        const int jj = __ffs(bal) - 1;
        const uint64_t w = __shfl_sync(0xffffffffu, T[r], jj);
        x = (r * G + jj) * 64 + __ffsll((long long)w) - 1;
        if (j == jj) T[r] &= T[r] - 1;
        return true;
      }
    }
  }
  return false;
}

// l = 2 below candidate set C: the number of arcs inside C (lane partials).
// Per vertex: every v in C is credited |C & adj[v]| and the (group-uniform)
// total is half their sum.
//
// One lane (G = 1): the members are walked word by word (the word loop is
// unrolled, so every word index is static); while word r is walked, the
// candidates still left have no bits below word r, so the AND/POPC of the
// count skips those words.
template <int G, int NW, bool PV>
__device__ __forceinline__ unsigned long long leaf2(const uint64_t (&C)[NW], const MatView V, int j,
                                                    unsigned &ovf_out) {
  unsigned ovf = 0;
  unsigned long long acc = 0;
  if constexpr (G == 1 && !PV) {
#pragma unroll
    for (int r = 0; r < NW; ++r) {
      uint64_t t = C[r];
      while (t) {
        const int x = r * 64 + __ffsll((long long)t) - 1;
        t &= t - 1;
        const uint64_t *row = V.adj + (size_t)x * V.RS;
        unsigned a = __popcll(t & row[r]);
#pragma unroll
        for (int q = r + 1; q < NW; ++q) a += __popcll(C[q] & row[q]);
        acc += a;
      }
    }
  } else {
    uint64_t T[NW];
#pragma unroll
    for (int r = 0; r < NW; ++r) T[r] = C[r];
    int x;
    while (next_bit<G, NW>(T, j, x)) {
      uint64_t R[NW];
      load_row<G, NW>(V.adj + (size_t)x * V.RS, V.W, j, R);
      unsigned a = 0;
      if (PV) {
#pragma unroll
        for (int r = 0; r < NW; ++r) a += __popcll(C[r] & R[r]);
        a = gsum32<G>(a);
        if (j == 0) credit(V, x, a);
      } else {
#pragma unroll
        for (int r = 0; r < NW; ++r) a += __popcll(T[r] & R[r]);
      }
      acc += a;
    }
  }
  ovf_out |= ovf;
  return PV ? (acc >> 1) : acc;
}

// Rec-Count-Cliques with L >= 3 vertices still to pick from C, L fixed at
// compile time so the levels stay in registers.
template <int G, int NW, bool PV, int L>
__device__ __forceinline__ unsigned long long dfs_fixed(const uint64_t (&C)[NW], const MatView V, int j,
                                                        unsigned &ovf_out) {
  if constexpr (L == 2) {
    return leaf2<G, NW, PV>(C, V, j, ovf_out);
  } else {
    unsigned ovf = 0;
    unsigned long long sum = 0;
    if constexpr (G == 1) {
      // one loop body (no per-word copies of the deeper levels): the next
      // member is found branch-free with static word indices
      uint64_t T[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) T[r] = C[r];
      for (;;) {
        int x = -1;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
          if (x < 0 && T[r]) {
            x = r * 64 + __ffsll((long long)T[r]) - 1;
            T[r] &= T[r] - 1;
          }
        }
        if (x < 0) break;
        const uint64_t *row = V.adj + (size_t)x * V.RS;
        uint64_t Cn[NW];
        unsigned c = 0;
#pragma unroll
        for (int q = 0; q < NW; ++q) {
          Cn[q] = T[q] & row[q];
          c += __popcll(Cn[q]);
        }
        if ((int)c < L - 1) continue;
        const unsigned long long sub = dfs_fixed<G, NW, PV, L - 1>(Cn, V, j, ovf);
        sum = add_ck(sum, sub, ovf);
        if (PV) credit(V, x, sub);
      }
    } else {
      uint64_t T[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) T[r] = C[r];
      int x;
      while (next_bit<G, NW>(T, j, x)) {
        uint64_t R[NW], Cn[NW];
        load_row<G, NW>(V.adj + (size_t)x * V.RS, V.W, j, R);
        unsigned c = 0;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
          Cn[r] = T[r] & R[r];
          c += __popcll(Cn[r]);
        }
        c = gsum32<G>(c);
        if ((int)c < L - 1) continue;
        const unsigned long long sub = dfs_fixed<G, NW, PV, L - 1>(Cn, V, j, ovf);
        sum = add_ck(sum, sub, ovf);
        if (PV && j == 0) credit(V, x, sub);
      }
    }
    ovf_out |= ovf;
    return sum;
  }
}

constexpr int kFixedMax = 6;  // deeper recursions use the explicit stack

// Rec-Count-Cliques for any ell >= 2 with an explicit stack (ell > kFixedMax).
template <int G, int NW, bool PV>
__device__ unsigned long long dfs_stack(const uint64_t (&C0)[NW], int ell, const MatView V, int j, unsigned &ovf_out) {
  unsigned ovf = 0;
  uint64_t Cs[kMaxFrames][NW], Ts[kMaxFrames][NW];
  unsigned long long subs[kMaxFrames];
  int xs[kMaxFrames];
  int top = 0;
#pragma unroll
  for (int r = 0; r < NW; ++r) Cs[0][r] = Ts[0][r] = C0[r];
  subs[0] = 0;
  unsigned long long ret = 0;
  for (;;) {
    const int l = ell - top;
    unsigned long long a = 0;
    bool done = false;
    if (l == 2) {
      uint64_t C[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) C[r] = Cs[top][r];
      a = leaf2<G, NW, PV>(C, V, j, ovf);
      done = true;
    } else {
      uint64_t T[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) T[r] = Ts[top][r];
      int x;
      const bool has = next_bit<G, NW>(T, j, x);
#pragma unroll
      for (int r = 0; r < NW; ++r) Ts[top][r] = T[r];
      if (!has) {
        a = subs[top];
        done = true;
      } else {
        uint64_t R[NW], Cn[NW];
        load_row<G, NW>(V.adj + (size_t)x * V.RS, V.W, j, R);
        unsigned c = 0;
#pragma unroll
        for (int r = 0; r < NW; ++r) {
          Cn[r] = T[r] & R[r];
          c += __popcll(Cn[r]);
        }
        c = gsum32<G>(c);
        if (top + 1 >= kMaxFrames) ovf |= ST_CAPACITY;
        if ((int)c >= l - 1 && top + 1 < kMaxFrames) {
          xs[top] = x;
          ++top;
#pragma unroll
          for (int r = 0; r < NW; ++r) Cs[top][r] = Ts[top][r] = Cn[r];
          subs[top] = 0;
        }
      }
    }
    if (done) {
      if (top == 0) {
        ret = a;
        break;
      }
      --top;
      subs[top] = add_ck(subs[top], a, ovf);
      if (PV && j == 0) credit(V, xs[top], a);
    }
  }
  { const auto ret_ = (ret); ovf_out |= ovf; return ret_; }
}

// ell >= 2 vertices still to pick from C. Register-resident levels are used
// while their sets stay small (two words: six levels, four words: four
// levels, wider: the leaf only); deeper recursions use the explicit stack.
template <int G, int NW, bool PV>
__device__ __forceinline__ unsigned long long dfs(const uint64_t (&C)[NW], int ell, const MatView V, int j,
                                                  unsigned &ovf) {
  constexpr int kFix = (G == 1 && NW <= 2) ? kFixedMax : ((G == 1 && NW <= 4) ? 4 : 2);
  if (ell == 2) return leaf2<G, NW, PV>(C, V, j, ovf);
  if constexpr (kFix >= 3) {
    if (ell == 3) return dfs_fixed<G, NW, PV, 3>(C, V, j, ovf);
  }
  if constexpr (kFix >= 4) {
    if (ell == 4) return dfs_fixed<G, NW, PV, 4>(C, V, j, ovf);
  }
  if constexpr (kFix >= 5) {
    if (ell == 5) return dfs_fixed<G, NW, PV, 5>(C, V, j, ovf);
  }
  if constexpr (kFix >= 6) {
    if (ell == 6) return dfs_fixed<G, NW, PV, 6>(C, V, j, ovf);
  }
  return dfs_stack<G, NW, PV>(C, ell, V, j, ovf);
}

// ----------------------------------------------------- warp item engines
struct Slot {
  uint64_t *mask;          // up to 32 mask words of the current candidate set (root positions)
  uint32_t *pfx;           // exclusive prefix of their population counts (33 entries)
  uint16_t *P;             // root positions of the compacted vertices
  uint64_t *S;             // compacted symmetric rows (s x NWc words)
  unsigned long long *cs;  // local per-vertex counters
};

__device__ __forceinline__ Slot carve_slot(uint8_t *base, bool pv) {
  const SlotLayout o = slot_layout(pv);
  Slot s;
  s.mask = (uint64_t *)(base + o.mask);
  s.pfx = (uint32_t *)(base + o.pfx);
  s.P = (uint16_t *)(base + o.P);
  s.S = (uint64_t *)(base + o.S);
  s.cs = pv ? (unsigned long long *)(base + o.cs) : nullptr;
  return s;
}

// Lane w (< W <= 32) holds word w of a candidate set over root positions:
// store the words and their prefix counts in the slot; returns |set|.
__device__ __forceinline__ uint32_t slot_set(const Slot sl, uint64_t mword, uint32_t W) {
  const unsigned lane = lane_id();
  const unsigned c = lane < W ? (unsigned)__popcll(mword) : 0u;
  const unsigned incl = warp_incl_scan(c);
  if (lane < W) {
    sl.mask[lane] = mword;
    sl.pfx[lane] = incl - c;
  }
  const uint32_t s = __shfl_sync(0xffffffffu, incl, 31);
  if (lane == 0) sl.pfx[W] = s;
  __syncwarp();
  return s;
}

// position of the r-th member of the slot's set
__device__ __forceinline__ uint32_t slot_select(const Slot sl, uint32_t W, uint32_t r) {
  uint32_t lo = 0, hi = W - 1;  // last word with pfx <= r
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (sl.pfx[mid] <= r) lo = mid; else hi = mid - 1;
  }
  uint64_t bb = sl.mask[lo];
  for (uint32_t q = r - sl.pfx[lo]; q; --q) bb &= bb - 1;
  return lo * 64 + (uint32_t)(__ffsll((long long)bb) - 1);
}

// Per-lane deadline check before a first-level subproblem of a block root
// (served passes with a time budget): past it, the subproblem is skipped and
// the pass reports ST_TIMEOUT.
__device__ __forceinline__ bool lane_past(uint64_t dl_ns, unsigned *dl_status) {
  if (dl_ns == 0) return false;
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  if (t <= dl_ns) return false;
  atomicOr(dl_status, ST_TIMEOUT);
  return true;
}

// Cliques taking `picks` (>= 2) more vertices from the slot's set of
// s <= kCompactMax root positions: the set is compacted to local ids 0..s-1
// (rank order is kept), its induced symmetric rows are extracted from the
// root matrix, and the lanes split the first pick. Per-vertex credits of the
// picked vertices go to the root counters rc. Returns the warp-uniform total.
template <bool PV>
__device__ unsigned long long compact_count(const MatView M, uint32_t s, int picks, const Slot sl,
                                            unsigned long long *rc, unsigned &ovf_out, uint64_t dl_ns = 0,
                                            unsigned *dl_status = nullptr) {
  unsigned ovf = 0;
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  if (lane < W) {
    uint64_t bw = sl.mask[lane];
    unsigned r = sl.pfx[lane];
    while (bw) {
      if (r < (unsigned)kCompactMax) sl.P[r] = (uint16_t)(lane * 64 + __ffsll((long long)bw) - 1);
      ++r;
      bw &= bw - 1;
    }
  }
  // per-item counters: an entry counts the item's cliques through one of its
  // s <= 128 vertices, at most C(127, picks - 1), below 2^32 for picks <= 6
  const bool c32 = picks <= 6;
  unsigned *cs32 = (unsigned *)sl.cs;
  if (PV)
    for (uint32_t q = lane; q < s; q += 32) {
      if (c32) cs32[q] = 0;
      else sl.cs[q] = 0;
    }
  __syncwarp();
  const uint32_t NWc = s <= 64 ? 1u : 2u;
  // bit b of compacted row q <=> P[b] adjacent to P[q]
  for (uint32_t q = lane; q < s; q += 32) {
    const uint64_t *src = M.adj + (size_t)sl.P[q] * M.RS;
    uint64_t o0 = 0, o1 = 0;
    for (uint32_t w = 0; w < W; ++w) {
      const uint64_t mk = sl.mask[w];
      uint64_t bits = src[w] & mk;
      while (bits) {
        const int bb = __ffsll((long long)bits) - 1;
        bits &= bits - 1;
        const uint32_t loc = sl.pfx[w] + (uint32_t)__popcll(mk & ((1ull << bb) - 1ull));
        if (loc < 64) o0 |= 1ull << loc;
        else o1 |= 1ull << (loc - 64);
      }
    }
    sl.S[q * NWc] = o0;
    if (NWc == 2) sl.S[q * NWc + 1] = o1;
  }
  __syncwarp();
  unsigned long long acc = 0;
  MatView V;
  V.adj = sl.S;
  V.cnt = sl.cs;
  V.cnt32 = c32 ? cs32 : nullptr;
  V.RS = NWc;
  V.W = NWc;
  for (uint32_t q = lane; q < s; q += 32) {
    unsigned long long sub = 0;
    if (NWc == 1) {
      uint64_t C[1] = {sl.S[q] & above_word(q, 0)};
      const int pc = __popcll(C[0]);
      if (picks == 2) sub = (unsigned long long)pc;
      else if (pc >= picks - 1 && !lane_past(dl_ns, dl_status)) sub = dfs<1, 1, PV>(C, picks - 1, V, 0, ovf);
    } else {
      uint64_t C[2] = {sl.S[2 * q] & above_word(q, 0), sl.S[2 * q + 1] & above_word(q, 1)};
      const int pc = __popcll(C[0]) + __popcll(C[1]);
      if (picks == 2) sub = (unsigned long long)pc;
      else if (pc >= picks - 1 && !lane_past(dl_ns, dl_status)) sub = dfs<1, 2, PV>(C, picks - 1, V, 0, ovf);
    }
    if (PV && picks > 2) credit(V, (int)q, sub);
    acc = add_ck(acc, sub, ovf);
  }
  if (PV && picks == 2) {
    // each arc of the compacted subgraph is one clique: q lies on all its arcs
    for (uint32_t q = lane; q < s; q += 32) {
      unsigned b = (unsigned)__popcll(sl.S[q * NWc]);
      if (NWc == 2) b += (unsigned)__popcll(sl.S[q * NWc + 1]);
      credit(V, (int)q, b);
    }
  }
  __syncwarp();
  if (PV)
    for (uint32_t q = lane; q < s; q += 32) atomic_add_ck(&rc[sl.P[q]], c32 ? cs32[q] : sl.cs[q], ovf);
  const unsigned long long tot = warp_sum64_ck(acc, ovf);
  __syncwarp();
  { const auto ret_ = (tot); ovf_out |= ovf; return ret_; }
}

// root positions that the slot's S and cs areas hold 32-bit counters for
constexpr uint32_t kSplitLocal = (kCompactMax * 2 * 8 + kCompactMax * 8) / 4;

// Lanes split the first pick of the slot's set (root positions, W <= NW <= 32
// words) and each lane runs the recursion on the root matrix with NW-word sets
// in registers. Returns the warp-uniform total.
template <int NW, bool PV>
__device__ unsigned long long split_count(const MatView M, uint32_t s, int picks, const Slot sl, unsigned &ovf_out,
                                          uint64_t dl_ns = 0, unsigned *dl_status = nullptr) {
  unsigned ovf = 0;
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  unsigned long long acc = 0;
  // per vertex with three picks: the credits go to 32-bit counters in the
  // warp's slot (the S and cs areas, 768 root positions; an entry is at most
  // C(s - 1, 2) < 2^32) and from there once to the root's counters
  MatView V = M;
  unsigned *lc = (unsigned *)sl.S;
  const bool local = PV && picks == 3 && W * 64 <= kSplitLocal;
  if (local) {
    for (uint32_t w = lane; w < W; w += 32)
      for (uint64_t b = sl.mask[w]; b; b &= b - 1) lc[w * 64 + __ffsll((long long)b) - 1] = 0u;
    __syncwarp();
    V.cnt32 = lc;
  }
  for (uint32_t r = lane; r < s; r += 32) {
    const uint32_t x = slot_select(sl, W, r);
    const uint64_t *rx = M.adj + (size_t)x * M.RS;
    uint64_t C[NW];
    int pc = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      C[w] = (uint32_t)w < W ? (sl.mask[w] & rx[w] & above_word(x, (uint32_t)w)) : 0ull;
      pc += __popcll(C[w]);
    }
    unsigned long long sub = 0;
    if (picks == 2) sub = (unsigned long long)pc;
    else if (pc >= picks - 1 && !lane_past(dl_ns, dl_status)) sub = dfs<1, NW, PV>(C, picks - 1, V, 0, ovf);
    if (PV && picks > 2) credit(V, (int)x, sub);
    acc = add_ck(acc, sub, ovf);
  }
  if (local) {
    __syncwarp();
    for (uint32_t w = lane; w < W; w += 32)
      for (uint64_t b = sl.mask[w]; b; b &= b - 1) {
        const uint32_t x = w * 64 + __ffsll((long long)b) - 1;
        atomic_add_ck(&M.cnt[x], lc[x], ovf);
      }
  }

  if (PV && picks == 2) {
    // each arc inside the set is one clique: v lies on |set & adj[v]| of them
    for (uint32_t r = lane; r < s; r += 32) {
      const uint32_t y = slot_select(sl, W, r);
      const uint64_t *cy = M.adj + (size_t)y * M.RS;
      unsigned b = 0;
      for (uint32_t w = 0; w < W; ++w) b += (unsigned)__popcll(sl.mask[w] & cy[w]);
      credit(M, (int)y, b);
    }
  }
  __syncwarp();
  { const auto ret_ = (warp_sum64_ck(acc, ovf)); ovf_out |= ovf; return ret_; }
}

// Lanes-over-words engine for roots wider than 32 words (d+ > 2048): the warp
// is one 32-lane group, lane j holding words r*32 + j of set & rowB.
template <int NW, bool PV>
__device__ unsigned long long generic_count(const MatView M, const uint64_t *rowA, uint32_t xa, const uint64_t *rowB,
                                            uint32_t xb, int picks, unsigned &ovf_out) {
  unsigned ovf = 0;
  const int j = (int)lane_id();
  uint64_t C[NW];
#pragma unroll
  for (int r = 0; r < NW; ++r) {
    const uint32_t w = (uint32_t)(r * 32 + j);
    uint64_t v = 0;
    if (w < M.W) {
      v = rowA[w] & above_word(xa, w);
      if (rowB) v &= rowB[w] & above_word(xb, w);
    }
    C[r] = v;
  }
  unsigned long long s = dfs<32, NW, PV>(C, picks, M, j, ovf);
  if (!PV) s = warp_sum64_ck(s, ovf);
  { const auto ret_ = (s); ovf_out |= ovf; return ret_; }
}

template <bool PV>
__device__ unsigned long long generic_dispatch(const MatView M, const uint64_t *rowA, uint32_t xa,
                                               const uint64_t *rowB, uint32_t xb, int picks, unsigned &ovf,
                                               unsigned *status) {
  const uint32_t nw = (M.W + 31u) / 32u;
  if (nw <= 2) return generic_count<2, PV>(M, rowA, xa, rowB, xb, picks, ovf);
  if (nw <= 4) return generic_count<4, PV>(M, rowA, xa, rowB, xb, picks, ovf);
  if (nw <= 8) return generic_count<8, PV>(M, rowA, xa, rowB, xb, picks, ovf);
  if (lane_id() == 0) atomicOr(status, ST_CAPACITY);
  return 0;
}

// Lanes-over-words for a set already in the slot (W <= 32 words).
template <bool PV>
__device__ unsigned long long wide_count(const MatView M, int picks, const Slot sl, unsigned &ovf_out) {
  unsigned ovf = 0;
  const int j = (int)lane_id();
  uint64_t C[1] = {(uint32_t)j < M.W ? sl.mask[j] : 0ull};
  unsigned long long s = dfs<32, 1, PV>(C, picks, M, j, ovf);
  if (!PV) s = warp_sum64_ck(s, ovf);
  { const auto ret_ = (s); ovf_out |= ovf; return ret_; }
}

template <bool PV>
__device__ unsigned long long split_dispatch(const MatView M, uint32_t s, int picks, const Slot sl, unsigned &ovf,
                                             uint64_t dl_ns = 0, unsigned *dl_status = nullptr) {
  if (M.W <= 2) return split_count<2, PV>(M, s, picks, sl, ovf, dl_ns, dl_status);
  if (M.W <= 4) return split_count<4, PV>(M, s, picks, sl, ovf, dl_ns, dl_status);
  if (M.W <= 8) return split_count<8, PV>(M, s, picks, sl, ovf, dl_ns, dl_status);
  if (M.W <= 12) return split_count<12, PV>(M, s, picks, sl, ovf, dl_ns, dl_status);
  return wide_count<PV>(M, picks, sl, ovf);
}

// k = 4 item of arc i (set = out-neighbours of x_i within N+(u), in the slot):
// the arcs inside the set; per vertex q lies on |set & adj[q]| of them.
template <bool PV>
__device__ unsigned long long k4_item(const MatView M, uint32_t s, const Slot sl, unsigned &ovf_out) {
  unsigned ovf = 0;
  const unsigned lane = lane_id();
  const uint32_t W = M.W;
  unsigned long long acc = 0;
  for (uint32_t r = lane; r < s; r += 32) {
    const uint32_t q = slot_select(sl, W, r);
    const uint64_t *rq = M.adj + (size_t)q * M.RS;
    unsigned x = 0, yv = 0;
    for (uint32_t z = 0; z < W; ++z) {
      const uint64_t m = sl.mask[z] & rq[z];
      x += (unsigned)__popcll(m & above_word(q, z));
      if (PV) yv += (unsigned)__popcll(m);
    }
    if (PV && yv) cnt_add(&M.cnt[q], yv);
    acc += x;
  }
  { const auto ret_ = (warp_sum64_ck(acc, ovf)); ovf_out |= ovf; return ret_; }
}

// Deadline check (batched and served passes): past the deadline, record
// ST_TIMEOUT and stop taking roots and items.
__device__ __forceinline__ uint64_t deadline_of(const CountArgs &a) {
  return a.deadline_dev ? *a.deadline_dev : a.deadline_ns;  // written before the pass started
}

__device__ __forceinline__ bool past_deadline(const CountArgs &a) {
  const uint64_t dl = deadline_of(a);
  if (dl && globaltimer_ns() > dl) {
    atomicOr(a.status, ST_TIMEOUT);
    return true;
  }
  return false;
}

// graph of vertex u in a batch (last g with goff[g] <= u), and its k
__device__ __forceinline__ uint32_t graph_of(const CountArgs &a, uint32_t u) {
  uint32_t lo = 0, hi = a.ngraphs - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (a.goff[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------- bulk-copy staging of the build
// The level-2 build reads the out-list N+(x) of every member x of N+(u)
// (Section 3.4). With bulk staging, each warp streams those out-lists into
// its own slot (idle during the build) with 1-D bulk copies
// (cp.async.bulk, completion counted by an mbarrier), two buffers deep: the
// copy of the next segment is in flight while the lanes look up the current
// one in shared memory. A copy starts and ends on 16-byte boundaries, so a
// segment is widened by up to three entries on each side (the DAG's column
// array carries 16 bytes of padding) and the lanes skip the extra entries.
constexpr int kBuildUnroll = 8;            // entries per lane per pass of the build
constexpr unsigned kWaitTries = 1u << 24;  // bound of an mbarrier wait

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits (bounded) for the phase of the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, unsigned parity) {
  for (unsigned it = 0; it < kWaitTries; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// One lane: expect `bytes` on the mbarrier and start the copy global -> shared.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

// The rows N+(L[i]) (start rb[i], length rl[i]) pulled from `next`, staged
// through the warp's slot and handed to mark(i, entries) kBuildUnroll * 32
// entries at a time (kEmpty past the segment). Called by all lanes.
template <typename Mark>
__device__ __forceinline__ void build_rows_bulk(const CountArgs &a, uint32_t d, const uint64_t *rb, const uint32_t *rl,
                                                uint8_t *slot, size_t slot_bytes, unsigned &next, Mark &mark) {
  const unsigned lane = lane_id();
  uint64_t *mb = (uint64_t *)slot;  // two mbarriers, then the two buffers
  // each buffer a multiple of 16 bytes; a segment leaves room for the widening
  const uint32_t cap = (uint32_t)(((slot_bytes - 16) / 2) / 16) * 4;
  const uint32_t seg = cap - 8;
  uint32_t *buf[2];
  buf[0] = (uint32_t *)(slot + 16);
  buf[1] = buf[0] + cap;
  const uint32_t mbar[2] = {smem_addr(&mb[0]), smem_addr(&mb[1])};
  if (lane == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar[0]) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar[1]) : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncwarp();
  unsigned parity[2] = {0u, 0u};
  uint32_t ri[2], rn[2], roff[2];  // row, entries and first-entry offset of each buffer's segment
  uint32_t cur_i = 0xffffffffu, cur_e = 0, cur_len = 0;
  uint64_t cur_xb = 0;
  // the next segment: the rest of the current row, or the next row with entries
  auto next_seg = [&](uint32_t &i, uint32_t &e0, uint32_t &ne, uint64_t &xb) -> bool {
    while (cur_i == 0xffffffffu || cur_e >= cur_len) {
      unsigned r = 0;
      if (lane == 0) r = atomicAdd(&next, 1u);
      r = __shfl_sync(0xffffffffu, r, 0);
      if (r >= d) return false;
      cur_i = r;
      cur_e = 0;
      cur_len = rl[r];
      cur_xb = rb[r];
    }
    i = cur_i;
    e0 = cur_e;
    ne = min(seg, cur_len - cur_e);
    xb = cur_xb;
    cur_e += ne;
    return true;
  };
  auto issue = [&](int b, uint32_t i, uint32_t e0, uint32_t ne, uint64_t xb) {
    const uint64_t first = xb + e0, start = first & ~3ull, end = (first + ne + 3) & ~3ull;
    ri[b] = i;
    rn[b] = ne;
    roff[b] = (uint32_t)(first - start);
    if (lane == 0) bulk_copy(smem_addr(buf[b]), a.col + start, (uint32_t)(end - start) * 4u, mbar[b]);
  };
  uint32_t i0, e0, n0;
  uint64_t x0;
  bool have = next_seg(i0, e0, n0, x0);
  if (have) issue(0, i0, e0, n0, x0);
  int b = 0;
  bool ok = true;
  while (have) {
    uint32_t i1, e1, n1;
    uint64_t x1;
    const bool have_next = next_seg(i1, e1, n1, x1);
    if (have_next) issue(1 - b, i1, e1, n1, x1);
    if (!mbar_wait(mbar[b], parity[b])) {
      ok = false;
      break;
    }
    parity[b] ^= 1u;
    const uint32_t *src = buf[b] + roff[b];
    for (uint32_t base = 0; base < rn[b]; base += 32 * kBuildUnroll) {
      uint32_t y[kBuildUnroll];
#pragma unroll
      for (int q = 0; q < kBuildUnroll; ++q) {
        const uint32_t e = base + lane + 32 * q;
        y[q] = e < rn[b] ? src[e] : kEmpty;
      }
      mark(ri[b], y);
    }
    __syncwarp();  // every lane is done with buffer b before it is refilled
    b = 1 - b;
    have = have_next;
  }
  if (!ok) {
    // a copy did not complete in time: report it, and wait (bounded) for the
    // copies still in flight before the slot is used for anything else
    if (lane == 0) atomicOr(a.status, ST_STALL);
    mbar_wait(mbar[0], parity[0]);
    mbar_wait(mbar[1], parity[1]);
  }
  __syncwarp();
  if (lane == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar[0]) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(mbar[1]) : "memory");
  }
  __syncwarp();
}

// ------------------------------------------------- dense-core lookups
// Rows of the induced subgraph read from the dense-core bit matrix (the
// members involved are all in the core; kc_core.cu). hid[i] is the core
// number of member i.

// Bits i (rows in m) of column j of the induced subgraph, hj = hid[j]:
// bit i set iff x_i -> x_j. Four loads in flight per lane.
__device__ __forceinline__ uint64_t core_column(const CountArgs &a, const uint32_t *hid, uint64_t m, uint32_t hj) {
  uint64_t c = 0;
  const unsigned long long *cb = a.core_bits + (hj >> 6);
  const uint64_t bit = 1ull << (hj & 63);
  while (m) {
    int ii[4];
    uint64_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ii[q] = m ? __ffsll((long long)m) - 1 : -1;
      m &= m - 1;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) w[q] = ii[q] >= 0 ? cb[(size_t)hid[ii[q]] * a.core_words] : 0ull;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (w[q] & bit) c |= 1ull << ii[q];
  }
  return c;
}

// Row i (core number hi) of a block root's induced subgraph: one bit per
// later member, 128 columns per pass. Other warps may set lower-triangle bits
// of the same words, hence the atomics.
template <bool PV>
__device__ __forceinline__ void core_row(const CountArgs &a, uint64_t *adj, uint32_t W, const uint32_t *hid,
                                         uint32_t i, uint32_t d, uint32_t hi) {
  const unsigned lane = lane_id();
  const unsigned long long *row = a.core_bits + (size_t)hi * a.core_words;
  for (uint32_t j0 = (i + 1) & ~63u; j0 < d; j0 += 128) {
    bool h[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint32_t j = j0 + 32 * q + lane;
      h[q] = false;
      if (j > i && j < d) {
        const uint32_t c = hid[j];
        if (c != kNoCore) h[q] = (row[c >> 6] >> (c & 63)) & 1ull;
        else atomicOr(a.status, ST_CAPACITY);  // a later member outside the core: cannot happen
      }
    }
#pragma unroll
    for (int q = 0; q < 4; q += 2) {
      const unsigned lo = __ballot_sync(0xffffffffu, h[q]), up = __ballot_sync(0xffffffffu, h[q + 1]);
      if (lane == 0 && (lo | up))
        atomicOr((unsigned long long *)&adj[(size_t)i * W + (j0 >> 6) + q / 2], ((unsigned long long)up << 32) | lo);
    }
    if (PV) {
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (h[q]) atomicOr((unsigned long long *)&adj[(size_t)(j0 + 32 * q + lane) * W + (i >> 6)], 1ull << (i & 63));
    }
  }
}

// ------------------------------------------------------- block-level root
struct BlockShared {
  unsigned long long red[kRootWarps];
  unsigned root, next, items, pad;
};

// block-wide exclusive scan of one value per thread (kRootBlock threads)
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned long long *red, unsigned *total) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  const unsigned incl = warp_incl_scan(v);
  if (lane == 31) red[warp] = incl;
  __syncthreads();
  unsigned off = 0, all = 0;
  for (int w = 0; w < kRootWarps; ++w) {
    if (w < (int)warp) off += (unsigned)red[w];
    all += (unsigned)red[w];
  }
  __syncthreads();
  *total = all;
  return off + incl - v;
}

template <bool PV, bool PA>
__device__ __forceinline__ void block_root(const CountArgs &a, uint32_t u, uint32_t oi, uint8_t *base, uint8_t *slots,
                                           unsigned long long &tsum_out, unsigned &ovf_out, BlockShared &sh) {
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  const unsigned tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
  // root rows: the DAG's out-lists, or (peeling) separate candidate rows
  // indexed like `order`, with the root's vertex id in rvert
  const uint64_t *rp_ = a.rptr ? a.rptr : a.ptr;
  const uint32_t *rc_ = a.rptr ? a.rcol : a.col;
  const uint64_t b = rp_[u];
  const uint32_t d = (uint32_t)(rp_[u + 1] - b);
  const uint32_t uv = a.rptr ? a.rvert[u] : u;
  const uint32_t W = words_of(d), T = hash_slots(d);
  const uint32_t g = a.goff ? graph_of(a, uv) : 0u;
  const int k = a.goff ? (int)a.gk[g] : a.k;
  if (k < 3 || k > KC_KMAX) {  // batches only: k = 1, 2 have closed forms, larger k is rejected
    if ((threadIdx.x & 31) == 0) atomicOr(a.status, ST_BAD_ARG);
    return;
  }
  if (d + 1 < (uint32_t)k) return;  // the root cannot hold a k-clique
  const uint32_t cmax = a.compact_max ? min(a.compact_max, (uint32_t)kCompactMax) : (uint32_t)kCompactMax;
  const uint64_t dl = deadline_of(a);
  const RootLayout lay = root_layout(d, PV, PA);
  uint32_t *L = (uint32_t *)(base + lay.L);
  uint64_t *rb = (uint64_t *)(base + lay.rb);
  uint32_t *rl = (uint32_t *)(base + lay.rl);
  unsigned long long *tab = (unsigned long long *)(base + lay.hslot);
  uint64_t *adj = (uint64_t *)(base + lay.adj);
  unsigned long long *cnt = PV ? (unsigned long long *)(base + lay.cnt) : nullptr;
  unsigned long long *asub = PA ? (unsigned long long *)(base + lay.asub) : nullptr;
  uint32_t *pre = (uint32_t *)(base + lay.pre);
  const Slot sl = carve_slot(slots + (size_t)warp * slot_layout(PV).bytes, PV);

  // N+(u) and the extents of its members' out-lists
  const uint32_t per = (d + kRootBlock - 1) / kRootBlock;
  const uint32_t c0 = min(d, tid * per), c1 = min(d, c0 + per);
  for (uint32_t i = tid; i < d; i += kRootBlock) {
    const uint32_t x = rc_[b + i];
    const uint64_t xb = a.ptr[x];
    L[i] = x;
    rb[i] = xb;
    rl[i] = (uint32_t)(a.ptr[x + 1] - xb);
    if (PV) cnt[i] = 0;
    if (PA) asub[i] = 0;
    if (a.core_bits) pre[i] = a.core_id[x];  // pre is free until the items are set up
  }
  for (uint32_t s = tid; s < T; s += kRootBlock) tab[s] = kEmptySlot;
  for (size_t w = tid; w < (size_t)d * W; w += kRootBlock) adj[w] = 0;
  if (tid == 0) sh.next = 0;
  __syncthreads();
  for (uint32_t i = tid; i < d; i += kRootBlock) pinsert(tab, T, L[i], i);
  __syncthreads();
  // the induced subgraph on N+(u): warps take whole rows (row i = N+(L[i])).
  // Out-lists are in rank order, so the hits of one row arrive in increasing
  // position and the row's bits are set with one atomic per distinct word.
  auto mark = [&](uint32_t i, const uint32_t (&y)[kBuildUnroll]) {
#pragma unroll
    for (int q = 0; q < kBuildUnroll; ++q) {
      const int t = y[q] == kEmpty ? -1 : plookup(tab, T, y[q]);
      const bool hit = t >= 0;
      const uint32_t w = hit ? ((uint32_t)t >> 6) : 0u;
      unsigned todo = __ballot_sync(0xffffffffu, hit);
      while (todo) {
        const int ld = __ffs(todo) - 1;
        const uint32_t wl = __shfl_sync(0xffffffffu, w, ld);
        const bool mine = hit && w == wl;
        const uint64_t bit = mine ? (1ull << (t & 63)) : 0ull;
        const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)bit);
        const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(bit >> 32));
        if (lane == (unsigned)ld)
          atomicOr((unsigned long long *)&adj[(size_t)i * W + wl], ((unsigned long long)hi << 32) | lo);
        todo &= ~__ballot_sync(0xffffffffu, mine);
      }
      // the lower triangle is read only by the per-vertex credits
      if (PV && hit) atomicOr((unsigned long long *)&adj[(size_t)t * W + (i >> 6)], 1ull << (i & 63));
    }
  };
  if (a.bulk_build) {
    build_rows_bulk(a, d, rb, rl, slots + (size_t)warp * slot_layout(PV).bytes, slot_layout(PV).bytes, sh.next, mark);
  } else {
    // eight loads in flight per lane
    for (;;) {
      unsigned i = 0;
      if (lane == 0) i = atomicAdd(&sh.next, 1u);
      i = __shfl_sync(0xffffffffu, i, 0);
      if (i >= d) break;
      const uint64_t xb = rb[i];
      const uint32_t len = rl[i];
      if (a.core_bits) {
        const uint32_t hi = pre[i];
        if (hi != kNoCore && (uint64_t)len >= (uint64_t)a.core_ratio * (d - 1 - i)) {
          core_row<PV>(a, adj, W, pre, i, d, hi);
          continue;
        }
      }
      for (uint32_t base = 0; base < len; base += 32 * kBuildUnroll) {
        uint32_t y[kBuildUnroll];
#pragma unroll
        for (int q = 0; q < kBuildUnroll; ++q) {
          const uint32_t e = base + lane + 32 * q;
          y[q] = e < len ? a.col[xb + e] : kEmpty;
        }
        mark(i, y);
      }
    }
  }
  __syncthreads();
  MatView M;
  M.adj = adj;
  M.cnt = cnt;
  M.cnt32 = nullptr;
  M.RS = W;
  M.W = W;
  unsigned long long rsum = 0;  // lane 0 of each warp holds its item totals
  if (k == 3) {
    for (uint32_t i = tid; i < d; i += kRootBlock) {
      unsigned c = 0, call = 0;
      for (uint32_t w = 0; w < W; ++w) {
        const uint64_t v = adj[(size_t)i * W + w];
        c += (unsigned)__popcll(v & above_word(i, w));
        if (PV) call += (unsigned)__popcll(v);
      }
      rsum = add_ck(rsum, c, ovf);
      if (PV) cnt[i] = call;  // triangles u-i-t for every neighbour t of i in N+(u)
      if (PA) asub[i] = c;
    }
  } else {
    const bool compactable = W <= (uint32_t)kCompactWords;
    uint32_t nitems = d;
    if (k >= 6 && compactable) {
      // arcs with more than kCompactMax candidates are split by their next vertex
      unsigned cl = 0;
      for (uint32_t i = c0; i < c1; ++i) {
        unsigned c = 0;
        for (uint32_t w = 0; w < W; ++w) c += (unsigned)__popcll(adj[(size_t)i * W + w] & above_word(i, w));
        c = c > cmax ? c : 0u;
        pre[i] = c;
        cl += c;
      }
      unsigned all;
      unsigned o2 = block_excl_scan(cl, sh.red, &all);
      for (uint32_t i = c0; i < c1; ++i) {
        const uint32_t c = pre[i];
        pre[i] = o2;
        o2 += c;
      }
      if (tid == 0) {
        pre[d] = all;
        sh.items = d + all;
      }
      __syncthreads();
      nitems = sh.items;
    }
    if (tid == 0) sh.next = 0;
    __syncthreads();
    for (;;) {
      unsigned t = 0;
      if (lane == 0) t = past_deadline(a) ? nitems : atomicAdd(&sh.next, 1u);
      t = __shfl_sync(0xffffffffu, t, 0);
      if (t >= nitems) break;
      unsigned long long item = 0;
      uint32_t i, av = 0xffffffffu;
      if (t < d) {
        // arc item: candidates = out-neighbours of x_i inside N+(u)
        i = t;
        const uint64_t *ri = adj + (size_t)i * W;
        if (!compactable) {
          unsigned s = 0;
          for (uint32_t w = lane; w < W; w += 32) s += (unsigned)__popcll(ri[w] & above_word(i, w));
          s = __reduce_add_sync(0xffffffffu, s);
          if (s >= (unsigned)(k - 2)) item = generic_dispatch<PV>(M, ri, i, nullptr, 0, k - 2, ovf, a.status);
        } else {
          const uint32_t s = slot_set(sl, lane < W ? (ri[lane] & above_word(i, lane)) : 0ull, W);
          if (s >= (uint32_t)(k - 2)) {
            if (k == 4) {
              item = k4_item<PV>(M, s, sl, ovf);
            } else if (k == 5 && (s > cmax || (!PV && W <= 2))) {
              // count only, rows of at most two words: compaction does not pay
              item = split_dispatch<PV>(M, s, 3, sl, ovf, dl, a.status);
            } else if (s <= cmax) {
              item = compact_count<PV>(M, s, k - 2, sl, cnt, ovf, dl, a.status);
            }  // else (k >= 6): split into pair items
          }
        }
      } else {
        // pair item: arc i and its r-th candidate av
        const uint32_t tt = t - d;
        uint32_t lo = 0, hi = d;  // last i with pre[i] <= tt
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= tt) lo = mid; else hi = mid - 1;
        }
        i = lo < d ? lo : d - 1;
        const uint64_t *ri = adj + (size_t)i * W;
        const uint64_t wv = lane < W ? (ri[lane] & above_word(i, lane)) : 0ull;
        const unsigned c = (unsigned)__popcll(wv);
        const unsigned incl = warp_incl_scan(c);
        const unsigned r = tt - pre[i];
        const unsigned hit = __ballot_sync(0xffffffffu, lane < W && r < incl && r >= incl - c);
        if (hit) {
          const int wl = __ffs(hit) - 1;
          if ((int)lane == wl) {
            uint64_t bb = wv;
            for (unsigned q = r - (incl - c); q; --q) bb &= bb - 1;
            av = lane * 64 + (uint32_t)(__ffsll((long long)bb) - 1);
          }
          av = __shfl_sync(0xffffffffu, av, wl);
          const uint64_t *rv = adj + (size_t)av * W;
          const uint64_t mw = lane < W ? (wv & rv[lane] & above_word(av, lane)) : 0ull;
          const uint32_t s0 = slot_set(sl, mw, W);
          if (s0 >= (uint32_t)(k - 3)) {
            // count only with three picks left: compaction costs as much as
            // the walk on the root rows, so the pair's set is walked in place
            if (s0 <= cmax && (PV || k != 6)) item = compact_count<PV>(M, s0, k - 3, sl, cnt, ovf, dl, a.status);
            else item = split_dispatch<PV>(M, s0, k - 3, sl, ovf, dl, a.status);
          }
        } else {
          if (lane == 0) atomicOr(a.status, ST_CAPACITY);
          av = 0xffffffffu;
        }
      }
      if (lane == 0 && item) {
        rsum = add_ck(rsum, item, ovf);
        if (PV) {
          cnt_add(&cnt[i], item);
          if (av != 0xffffffffu) cnt_add(&cnt[av], item);
        }
        if (PA) atomic_add_ck(&asub[i], item, ovf);
      }
    }
  }
  __syncthreads();
  if (PV || a.gtotal || a.rooted) {
    const unsigned long long r = warp_sum64_ck(rsum, ovf);
    if (lane == 0) sh.red[warp] = r;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < kRootWarps; ++w) t = add_ck(t, sh.red[w], ovf);
      if (PV) atomic_add_ck(&a.pv[uv], t, ovf);
      if (a.gtotal) atomic_add_ck(&a.gtotal[g], t, ovf);
      if (a.rooted) a.rooted[a.rooted_pos[oi]] = t;
    }
    if (PV)
      for (uint32_t i = tid; i < d; i += kRootBlock) atomic_add_ck(&a.pv[L[i]], cnt[i], ovf);
  }
  if (PA)
    for (uint32_t i = tid; i < d; i += kRootBlock) a.pa[b + i] = asub[i];
  tsum = add_ck(tsum, rsum, ovf);
  __syncthreads();
  ovf_out |= ovf;
  tsum_out = add_ck(tsum_out, tsum, ovf_out);
}

__device__ inline void finish_block(const CountArgs &a, unsigned long long tsum, unsigned ovf, unsigned long long *red,
                                    int nwarps) {
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  __syncthreads();
  const unsigned long long r = warp_sum64_ck(tsum, ovf);
  ovf = __reduce_or_sync(0xffffffffu, ovf);
  if (lane == 0) red[warp] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < nwarps; ++w) t = add_ck(t, red[w], ovf);
    atomic_add_ck(a.total, t, ovf);
  }
  if (lane == 0 && ovf) atomicOr(a.status, ovf);
}

// Persistent block roots: first the ones whose matrices live in global
// scratch (largest out-degrees), then the shared-memory ones, all in order of
// decreasing out-degree.
template <bool PV, bool PA>
__global__ void __launch_bounds__(kRootBlock, 1) count_block_kernel(CountArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ BlockShared sh;
  const unsigned tid = threadIdx.x;
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  uint8_t *slots = smem;
  uint8_t *root_area = smem + (size_t)kRootWarps * slot_layout(PV).bytes;
  if (blockIdx.x < a.scratch_blocks) {
    uint8_t *slab = a.scratch + (size_t)blockIdx.x * a.scratch_stride;
    for (;;) {
      if (tid == 0) sh.root = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[0], 1u);
      __syncthreads();
      const unsigned idx = sh.root;
      __syncthreads();
      if (idx >= a.n_scratch) break;
      block_root<PV, PA>(a, a.order[idx], idx, slab, slots, tsum, ovf, sh);
    }
  }
  for (;;) {
    if (tid == 0) sh.root = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[1], 1u);
    __syncthreads();
    const unsigned idx = sh.root;
    __syncthreads();
    if (idx >= a.n_big - a.n_scratch) break;
    block_root<PV, PA>(a, a.order[a.n_scratch + idx], a.n_scratch + idx, root_area, slots, tsum, ovf, sh);
  }
  finish_block(a, tsum, ovf, sh.red, kRootWarps);
}

// ------------------------------------------------------- warp-level root
// Roots with d+ <= 64: one warp, rows of one word, items over lanes (arcs for
// k = 4, triangles u->x_i->x_j for k >= 5, each lane one item).
template <bool PV, bool PA>
__device__ __forceinline__ void warp_root(const CountArgs &a, uint32_t u, uint32_t oi, uint8_t *slot,
                                          unsigned long long &tsum_out, unsigned &ovf_out, unsigned *w_next) {
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  const unsigned lane = lane_id();
  const LightLayout o = light_layout(PV, PA);
  uint32_t *L = (uint32_t *)(slot + o.L);
  uint64_t *rbeg = (uint64_t *)(slot + o.rb);
  uint32_t *hkey = (uint32_t *)(slot + o.hkey);
  uint16_t *hpos = (uint16_t *)(slot + o.hpos);
  uint64_t *adj = (uint64_t *)(slot + o.adj);
  unsigned long long *cnt = PV ? (unsigned long long *)(slot + o.cnt) : nullptr;
  unsigned long long *asub = PA ? (unsigned long long *)(slot + o.asub) : nullptr;
  uint32_t *pre = (uint32_t *)(slot + o.pre);
  uint32_t *epre = (uint32_t *)(slot + o.epre);
  // root rows: the DAG's out-lists, or (peeling) separate candidate rows
  // indexed like `order`, with the root's vertex id in rvert
  const uint64_t *rp_ = a.rptr ? a.rptr : a.ptr;
  const uint32_t *rc_ = a.rptr ? a.rcol : a.col;
  const uint64_t b = rp_[u];
  const uint32_t d = (uint32_t)(rp_[u + 1] - b);
  const uint32_t uv = a.rptr ? a.rvert[u] : u;
  const uint32_t g = a.goff ? graph_of(a, uv) : 0u;
  const int k = a.goff ? (int)a.gk[g] : a.k;
  if (k < 3 || k > KC_KMAX) {  // batches only: k = 1, 2 have closed forms, larger k is rejected
    if ((threadIdx.x & 31) == 0) atomicOr(a.status, ST_BAD_ARG);
    return;
  }
  if (d + 1 < (uint32_t)k) return;  // the root cannot hold a k-clique
  for (uint32_t i = lane; i < (uint32_t)kLightMax; i += 32) {
    adj[i] = 0;
    if (PV) cnt[i] = 0;
    if (PA) asub[i] = 0;
  }
  for (uint32_t s = lane; s < 128; s += 32) hkey[s] = kEmpty;
  uint32_t e0 = 0, e1 = 0, h0 = kNoCore, h1 = kNoCore;
  if (lane < d) {
    const uint32_t x = rc_[b + lane];
    const uint64_t xb = a.ptr[x];
    L[lane] = x;
    rbeg[lane] = xb;
    e0 = (uint32_t)(a.ptr[x + 1] - xb);
    if (a.core_bits) h0 = a.core_id[x];
  }
  if (lane + 32 < d) {
    const uint32_t x = rc_[b + lane + 32];
    const uint64_t xb = a.ptr[x];
    L[lane + 32] = x;
    rbeg[lane + 32] = xb;
    e1 = (uint32_t)(a.ptr[x + 1] - xb);
    if (a.core_bits) h1 = a.core_id[x];
  }
  // rows taken from the dense core (bits ub): members in the core whose
  // out-list holds at least core_ratio entries per later member; their
  // out-lists drop out of the scan. pre holds the core numbers until the
  // items are set up.
  uint64_t ub = 0;
  if (a.core_bits) {
    const bool b0 = h0 != kNoCore && (uint64_t)e0 >= (uint64_t)a.core_ratio * (d - 1 - lane);
    const bool b1 = h1 != kNoCore && (uint64_t)e1 >= (uint64_t)a.core_ratio * (d - 33 - lane);
    ub = (uint64_t)__ballot_sync(0xffffffffu, b0) | ((uint64_t)__ballot_sync(0xffffffffu, b1) << 32);
    if (b0) e0 = 0;
    if (b1) e1 = 0;
    pre[lane] = h0;
    pre[lane + 32] = h1;
  }
  const unsigned z0 = warp_incl_scan(e0), z1 = warp_incl_scan(e1);
  const unsigned tot0 = __shfl_sync(0xffffffffu, z0, 31), tot1 = __shfl_sync(0xffffffffu, z1, 31);
  epre[lane] = z0 - e0;
  epre[lane + 32] = tot0 + z1 - e1;
  if (lane == 0) epre[kLightMax] = tot0 + tot1;
  __syncwarp();
  for (uint32_t i = lane; i < d; i += 32) hinsert(hkey, hpos, 128, L[i], i);
  __syncwarp();
  // the concatenated rows, eight loads in flight per lane; rows past d are empty
  const uint32_t E = tot0 + tot1;
  {
    constexpr int U = 8;
    uint32_t i = 0;
    for (uint32_t base = 0; base < E; base += 32 * U) {  // warp-uniform trip count
      uint32_t y[U], row[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const uint32_t e = base + lane + 32 * q;
        y[q] = kEmpty;
        row[q] = 0;
        if (e < E) {
          while (epre[i + 1] <= e) ++i;
          row[q] = i;
          y[q] = a.col[rbeg[i] + (e - epre[i])];
        }
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int t = y[q] == kEmpty ? -1 : hlookup(hkey, hpos, 128, y[q]);
        const uint32_t r = row[q];
        warp_set_bits(adj, 1, t >= 0, r, t >= 0 ? (uint32_t)t : 0u);
        if (PV && t >= 0) atomicOr((unsigned long long *)&adj[t], 1ull << r);
      }
    }
  }
  __syncwarp();
  if (ub) {
    // columns lane and lane + 32 over the rows in ub, then rows by ballot;
    // lane t owns words t and t + 32 (upper bits from the rows, lower bits,
    // per vertex only, from the columns)
    const uint64_t m0 = ub & ((1ull << lane) - 1ull), m1 = ub & ((1ull << (lane + 32)) - 1ull);
    uint64_t c0 = 0, c1 = 0;
    if (lane < d && m0) {
      if (h0 != kNoCore) c0 = core_column(a, pre, m0, h0);
      else atomicOr(a.status, ST_CAPACITY);  // a later member outside the core: cannot happen
    }
    if (lane + 32 < d && m1) {
      if (h1 != kNoCore) c1 = core_column(a, pre, m1, h1);
      else atomicOr(a.status, ST_CAPACITY);
    }
    uint64_t r0 = 0, r1 = 0;
    for (uint64_t m = ub; m; m &= m - 1) {
      const int i = __ffsll((long long)m) - 1;
      const uint64_t row = (uint64_t)__ballot_sync(0xffffffffu, (c0 >> i) & 1ull) |
                           ((uint64_t)__ballot_sync(0xffffffffu, (c1 >> i) & 1ull) << 32);
      if (lane == (unsigned)(i & 31)) {
        if (i < 32) r0 = row;
        else r1 = row;
      }
    }
    adj[lane] |= r0 | (PV ? c0 : 0ull);
    adj[lane + 32] |= r1 | (PV ? c1 : 0ull);
    __syncwarp();
  }
  // a root with d <= 64 out-neighbours: an entry counts the root's cliques
  // through one of them, at most C(62, k - 2), below 2^32 for k <= 10
  const bool c32 = k <= 10;
  unsigned *cnt32 = (unsigned *)cnt;
  MatView V;
  V.adj = adj;
  V.cnt = cnt;
  V.cnt32 = (PV && c32) ? cnt32 : nullptr;
  V.RS = 1;
  V.W = 1;
  unsigned long long rsum = 0;
  if (k == 3) {
    for (uint32_t i = lane; i < d; i += 32) {
      const uint64_t v = adj[i];
      const unsigned c = (unsigned)__popcll(v & above_word(i, 0));
      rsum = add_ck(rsum, c, ovf);
      if (PV) cnt32[i] = (unsigned)__popcll(v);  // k = 3 uses the 32-bit counters
      if (PA) asub[i] = c;
    }
  } else {
    uint32_t nitems = d;
    if (k >= 5) {
      const uint32_t c0 = lane < d ? (uint32_t)__popcll(adj[lane] & above_word(lane, 0)) : 0u;
      const uint32_t c1 = lane + 32 < d ? (uint32_t)__popcll(adj[lane + 32] & above_word(lane + 32, 0)) : 0u;
      const unsigned y0 = warp_incl_scan(c0), y1 = warp_incl_scan(c1);
      const unsigned t0 = __shfl_sync(0xffffffffu, y0, 31), t1 = __shfl_sync(0xffffffffu, y1, 31);
      pre[lane] = y0 - c0;
      pre[lane + 32] = t0 + y1 - c1;
      if (lane == 0) pre[kLightMax] = t0 + t1;
      nitems = t0 + t1;
    }
    if (lane == 0) *w_next = 0;
    __syncwarp();
    for (;;) {
      const unsigned t = past_deadline(a) ? nitems : atomicAdd(w_next, 1u);
      if (t >= nitems) break;
      uint32_t i, jv = 0xffffffffu;
      uint64_t C[1];
      int ell;
      if (k == 4) {
        i = t;
        C[0] = adj[i] & above_word(i, 0);
        ell = 2;
      } else {
        uint32_t lo = 0, hi = d;  // last i with pre[i] <= t
        while (lo < hi) {
          const uint32_t mid = (lo + hi + 1) >> 1;
          if (pre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        i = lo;
        if (i >= d) {
          atomicOr(a.status, ST_CAPACITY);
          continue;
        }
        uint64_t w = adj[i] & above_word(i, 0);
        for (uint32_t q = t - pre[i]; q; --q) w &= w - 1;
        if (!w) {
          atomicOr(a.status, ST_CAPACITY);
          continue;
        }
        jv = (uint32_t)(__ffsll((long long)w) - 1);
        C[0] = adj[i] & adj[jv] & above_word(jv, 0);
        ell = k - 3;
      }
      if (__popcll(C[0]) < ell) continue;
      const unsigned long long s = dfs<1, 1, PV>(C, ell, V, 0, ovf);
      rsum = add_ck(rsum, s, ovf);
      if (PV) {
        credit(V, (int)i, s);
        if (jv != 0xffffffffu) credit(V, (int)jv, s);
      }
      if (PA) atomic_add_ck(&asub[i], s, ovf);
    }
  }
  __syncwarp();
  if (PV || a.gtotal || a.rooted) {
    const unsigned long long t = warp_sum64_ck(rsum, ovf);
    if (lane == 0 && PV) atomic_add_ck(&a.pv[uv], t, ovf);
    if (lane == 0 && a.gtotal) atomic_add_ck(&a.gtotal[g], t, ovf);
    if (lane == 0 && a.rooted) a.rooted[a.rooted_pos[oi]] = t;
    if (PV)
      for (uint32_t i = lane; i < d; i += 32) atomic_add_ck(&a.pv[L[i]], c32 ? cnt32[i] : cnt[i], ovf);
  }
  if (PA)
    for (uint32_t i = lane; i < d; i += 32) a.pa[b + i] = asub[i];
  tsum = add_ck(tsum, rsum, ovf);
  __syncwarp();
  ovf_out |= ovf;
  tsum_out = add_ck(tsum_out, tsum, ovf_out);
}

// Resident blocks per SM: five for the count-only variant (48 registers; its
// warp roots are latency-bound, and the batched pass of many small graphs
// runs 16% faster so), three for the others (at most 85 registers).
template <bool PV, bool PA>
__global__ void __launch_bounds__(kBlock, (PV || PA) ? 3 : 5) count_warp_kernel(CountArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  __shared__ unsigned long long red[kWarps];
  __shared__ unsigned w_next[kWarps];
  const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
  unsigned ovf = 0;
  unsigned long long tsum = 0;
  uint8_t *slot = smem + (size_t)warp * light_layout(PV, PA).bytes;
  const uint32_t chunk = a.chunk ? a.chunk : 1u;
  const uint32_t nlight = a.n_light_end - a.n_big;
  // id order walks windows of 2^16 ids; inside a window, slot s holds the id
  // with the bit-reversed offset, so the ids one warp takes are spread over
  // the window (a graph's consecutive densest roots land in different warps)
  // while all warps stay in one L2-resident window of the batch
  constexpr uint32_t kWinBits = 16;
  const unsigned long long ngroups =
      (((unsigned long long)a.n + (1ull << kWinBits) - 1) >> kWinBits) << (kWinBits - 5);
  // One call site of warp_root (its body is large). The warp-uniform cursor
  // walks the work this warp pulled: positions of the order array (out-degree
  // order) or groups of 32 id slots whose qualifying members (light_min <= d+
  // <= light_max) are taken in slot order (id order: a batch's graphs are
  // counted one id window at a time, so their out-lists stay in L2).
  uint32_t q = 0, qend = 0, base = 0;
  unsigned mask = 0;
  for (;;) {
    uint32_t u, oi = 0;  // oi: position in the order array (out-degree order only)
    if (a.light_by_id) {
      bool done = false;
      while (mask == 0) {
        if (q >= qend) {
          unsigned idx = 0;
          if (lane == 0) idx = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[2], chunk);
          idx = __shfl_sync(0xffffffffu, idx, 0);
          if ((unsigned long long)idx >= ngroups) {
            done = true;
            break;
          }
          q = idx;
          qend = (uint32_t)min(ngroups, (unsigned long long)idx + chunk);
        }
        base = q * 32u;
        ++q;
        const uint32_t slot_i = base + lane;
        const uint32_t v = (slot_i & ~((1u << kWinBits) - 1u)) | (__brev(slot_i) >> (32 - kWinBits));
        bool ok = false;
        if (v < a.n) {
          const uint32_t d = (uint32_t)(a.ptr[v + 1] - a.ptr[v]);
          ok = d >= a.light_min && d <= a.light_max;
        }
        mask = __ballot_sync(0xffffffffu, ok);
      }
      if (done) break;
      const int l = __ffs(mask) - 1;
      mask &= mask - 1;
      const uint32_t slot_l = base + (uint32_t)l;
      u = (slot_l & ~((1u << kWinBits) - 1u)) | (__brev(slot_l) >> (32 - kWinBits));
    } else {
      if (q >= qend) {
        unsigned idx = 0;
        if (lane == 0) idx = past_deadline(a) ? 0xffffffffu : atomicAdd(&a.queue[2], chunk);
        idx = __shfl_sync(0xffffffffu, idx, 0);
        if (idx >= nlight) break;
        q = idx;
        qend = min(nlight, idx + chunk);
      }
      oi = a.n_big + q;
      u = a.order[oi];
      ++q;
    }
    warp_root<PV, PA>(a, u, oi, slot, tsum, ovf, &w_next[warp]);
  }
  finish_block(a, tsum, ovf, red, kWarps);
}

template <bool PV, bool PA>
cudaError_t occupancy_variant(size_t block_smem, int *block_per_sm, int *warp_per_sm) {
  // The dynamic shared-memory limit of the block kernel is raised once to the
  // device's opt-in maximum, not to this pass's size: plans made now may be
  // launched later, after other plans (other sizes) were made.
  static std::once_flag once;
  static cudaError_t set_err = cudaSuccess;
  std::call_once(once, [] {
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    set_err = cudaGetDevice(&dev);
    if (set_err == cudaSuccess) set_err = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (set_err == cudaSuccess) set_err = cudaFuncGetAttributes(&fa, count_block_kernel<PV, PA>);
    if (set_err == cudaSuccess)
      set_err = cudaFuncSetAttribute(count_block_kernel<PV, PA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     optin - (int)fa.sharedSizeBytes);
  });
  cudaError_t e = set_err;
  if (e != cudaSuccess) return e;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(block_per_sm, count_block_kernel<PV, PA>, kRootBlock,
                                                    block_smem);
  if (e != cudaSuccess) return e;
  const size_t wsm = (size_t)kWarps * light_layout(PV, PA).bytes;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(warp_per_sm, count_warp_kernel<PV, PA>, kBlock, wsm);
}

template <bool PV, bool PA>
cudaError_t launch_variant(const CountArgs &a, int block_grid, int warp_grid, size_t block_smem, cudaStream_t s) {
  if (a.n_big > 0 && block_grid > 0) {
    count_block_kernel<PV, PA><<<block_grid, kRootBlock, block_smem, s>>>(a);
    note_launch();
  }
  if (a.n_light_end > a.n_big && warp_grid > 0) {
    const size_t wsm = (size_t)kWarps * light_layout(PV, PA).bytes;
    count_warp_kernel<PV, PA><<<warp_grid, kBlock, wsm, s>>>(a);
    note_launch();
  }
  return cudaGetLastError();
}

}  // namespace kc
