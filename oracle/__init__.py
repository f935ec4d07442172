"""CPU oracle for exact k-clique counting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never loads it and
shares no code with it (``kc_oracle.c`` is plain sequential C).

Parity status of each function (what pins it, in ``tests/test_oracle_pins.py``):

* ``count`` / ``count_per_vertex``: brute force over all k-subsets (n <= 30),
  C(n,k) on K_n, elementary symmetric polynomials on Turan graphs,
  trace(A^3)/6 and diag(A^3)/2 for triangles, additivity over disjoint unions,
  invariance over four orderings and random relabellings, sum of per-vertex
  counts = k * total, k=1 -> n, k=2 -> m, bipartite -> 0, planted disjoint
  cliques, and the 4-clique fragment of the paper's worked example
  (Appendix A, Figure 7; the figure itself is missing, so that pin is partial).
* ``count_arc``: sums over all arcs equal ``count`` (k >= 2).
* ``count_containing`` (k-cliques through one vertex, via its neighbourhood):
  equal to brute force per vertex (n <= 16), to C(n-1, k-1) on K_n, and its
  sum over the vertices is k times the total.
* ``colorful_count`` (colorful sparsification, Section 3.3): one color gives
  the exact count; over many seeds the estimate's mean and variance match
  the appendix theorem (E[Y] = X, Var[Y] from the counts s_z of clique pairs
  sharing z vertices, computed by brute force); the color generator gives
  splitmix64's well-known first output for seed 0 (0xe220a8397b1dcdaf).
* ``be_order`` (Barenboim-Elkin, Section 3.1): every out-degree is below
  12 rho~ and rho~ <= rho* <= 4 rho~ against a brute-force densest subgraph;
  a complete graph and a path worked by hand; counts equal those of every
  other orientation.
* ``peel_approx`` (arb-approx-peel, Section 4.2): K_n in one round; the
  1/(k(1+eps)) guarantee against a brute-force densest subset; at most
  log_{1+eps}(n) + 1 rounds (each round removes at least an eps/(1+eps)
  share of the remaining vertices, since the counts average k t / |S|).
* ``peel`` (arb-peel, Algorithm 2): K_n in one round at C(n,k)/n; a disjoint
  K_a + K_b in two rounds at C(b,k)/b; no k-clique -> one round at 0; the
  1/k guarantee against a brute-force densest subset (n <= 12); peeling
  rounds follow a relabelling of the vertices.
* ``orient`` (degree / degeneracy / original / gp): every ordering yields an
  acyclic orientation that keeps each edge once; the degree and GP orders
  are checked against their defining properties on hand-made graphs. The
  degeneracy (smallest-last) order is recomputed step by step from a dense
  matrix (each removed vertex has the minimum remaining degree, smallest id
  first), and its largest out-degree equals the degeneracy: 1 for trees, 2
  for cycles and grids, n - 1 for K_n, n minus the largest part for Turan
  graphs, and the brute-force maximum over all vertex subsets of the
  minimum degree on random graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkcoracle.so")
_SRC = os.path.join(_HERE, "kc_oracle.c")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ERANGE, ENOMEM = 0, 1, 2, 3


class OracleError(RuntimeError):
    pass


class OracleOverflow(OracleError):
    pass


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, i64, cint = ctypes.c_uint32, ctypes.c_int64, ctypes.c_int
            lib.or_rank_degree.argtypes = [u32, P, P]
            lib.or_rank_degeneracy.argtypes = [u32, P, P, P]
            lib.or_rank_gp.argtypes = [u32, P, P, P, P, P]
            lib.or_direct.argtypes = [u32, P, P, P, P, P]
            lib.or_direct.restype = i64
            lib.or_count.argtypes = [u32, P, P, cint, u32, u32, P, P, P]
            lib.or_count_arc.argtypes = [u32, P, P, cint, u32, u32, P, P]
            lib.or_brute.argtypes = [u32, P, cint, P, P]
            for f in (lib.or_rank_degree, lib.or_rank_degeneracy, lib.or_rank_gp, lib.or_count,
                      lib.or_count_arc, lib.or_brute):
                f.restype = cint
            _lib = lib
    return _lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int):
    if rc == ERANGE:
        raise OracleOverflow("count does not fit in uint64")
    if rc != OK:
        raise OracleError(f"oracle status {rc}")


@dataclass
class Dag:
    """Oriented graph: ``ptr`` uint64[n+1], ``adj`` uint32[m] (out-lists, ascending id)."""
    n: int
    ptr: np.ndarray
    adj: np.ndarray
    rank: np.ndarray

    @property
    def m(self) -> int:
        return int(self.ptr[-1])


def _csr_arrays(g):
    return (np.ascontiguousarray(g.row_ptr, dtype=np.uint64), np.ascontiguousarray(g.col, dtype=np.uint32))


def rank(g, method: str = "degree", perm=None) -> np.ndarray:
    """Position of every vertex in the chosen total order.

    methods: "degree" (non-decreasing degree, ties by id), "degeneracy"
    (Matula-Beck k-core order), "original" (ids), "gp" (Goodrich-Pszona,
    Algorithm 3 with epsilon = 1), "be" (Barenboim-Elkin, epsilon = 1, see
    be_order), "perm" (the given ranks).
    """
    lib = _load()
    rp, col = _csr_arrays(g)
    r = np.empty(max(g.n, 1), dtype=np.uint32)
    if method == "degree":
        _check(lib.or_rank_degree(g.n, _p(rp), _p(r)))
    elif method == "degeneracy":
        _check(lib.or_rank_degeneracy(g.n, _p(rp), _p(col), _p(r)))
    elif method == "original":
        r[:g.n] = np.arange(g.n, dtype=np.uint32)
    elif method == "gp":
        _check(lib.or_rank_gp(g.n, _p(rp), _p(col), _p(r), None, None))
    elif method == "be":
        r[:g.n] = be_order(g)[0]
    elif method == "perm":
        r[:g.n] = np.asarray(perm, dtype=np.uint32)
    else:
        raise ValueError(method)
    return r[:g.n]


def gp_rounds(g):
    """(rank, round, induced degree at removal) of the Goodrich-Pszona order."""
    lib = _load()
    rp, col = _csr_arrays(g)
    r = np.empty(max(g.n, 1), dtype=np.uint32)
    rd = np.empty(max(g.n, 1), dtype=np.uint32)
    dg = np.empty(max(g.n, 1), dtype=np.uint32)
    _check(lib.or_rank_gp(g.n, _p(rp), _p(col), _p(r), _p(rd), _p(dg)))
    return r[:g.n], rd[:g.n], dg[:g.n]


def orient(g, method: str = "degree", perm=None) -> Dag:
    """Direct every edge from the lower to the higher vertex of the order."""
    lib = _load()
    rp, col = _csr_arrays(g)
    r = np.ascontiguousarray(rank(g, method, perm), dtype=np.uint32)
    ptr = np.empty(g.n + 1, dtype=np.uint64)
    adj = np.empty(max(g.nnz // 2, 1), dtype=np.uint32)
    m = lib.or_direct(g.n, _p(rp), _p(col), _p(r), _p(ptr), _p(adj))
    return Dag(g.n, ptr, adj[:m].copy(), r)


def _count_range(dag: Dag, k: int, lo: int, hi: int, pv):
    lib = _load()
    slo = ctypes.c_uint64()
    shi = ctypes.c_uint64()
    adj = dag.adj if dag.adj.size else np.zeros(1, np.uint32)
    rc = lib.or_count(dag.n, _p(dag.ptr), _p(adj), k, lo, hi, ctypes.byref(slo), ctypes.byref(shi),
                      None if pv is None else _p(pv))
    return rc, (shi.value << 64) | slo.value


def count(dag: Dag, k: int, threads: int = 1, lo: int = 0, hi: int | None = None) -> int:
    """Number of k-cliques (Algorithm 1 from every root in [lo, hi)). Raises on uint64 overflow."""
    hi = dag.n if hi is None else hi
    if k < 1:
        raise ValueError("k must be >= 1")
    if threads <= 1:
        rc, t = _count_range(dag, k, lo, hi, None)
        _check(rc)
    else:
        bounds = np.linspace(lo, hi, threads * 8 + 1).astype(np.int64)
        with ThreadPoolExecutor(threads) as ex:
            res = list(ex.map(lambda ab: _count_range(dag, k, int(ab[0]), int(ab[1]), None),
                              zip(bounds[:-1], bounds[1:])))
        for rc, _ in res:
            _check(rc)
        t = sum(x for _, x in res)
    if t >= 1 << 64:
        raise OracleOverflow("count does not fit in uint64")
    return int(t)


def count_per_vertex(dag: Dag, k: int, threads: int = 1) -> tuple[int, np.ndarray]:
    """(total, per-vertex counts): pv[v] = number of k-cliques containing v.

    With threads > 1 the roots are split into ranges, each range summed into its
    own array, and the arrays added (the same sequential routine per range).
    """
    if threads <= 1:
        pv = np.zeros(max(dag.n, 1), dtype=np.uint64)
        rc, t = _count_range(dag, k, 0, dag.n, pv)
        _check(rc)
    else:
        bounds = np.linspace(0, dag.n, threads * 4 + 1).astype(np.int64)
        parts = [np.zeros(max(dag.n, 1), dtype=np.uint64) for _ in range(threads)]
        chunks = list(zip(bounds[:-1], bounds[1:]))

        def work(ti):
            tot = 0
            for ci in range(ti, len(chunks), threads):
                rc, x = _count_range(dag, k, int(chunks[ci][0]), int(chunks[ci][1]), parts[ti])
                _check(rc)
                tot += x
            return tot

        with ThreadPoolExecutor(threads) as ex:
            t = sum(ex.map(work, range(threads)))
        pv = parts[0]
        for q in parts[1:]:
            s = pv + q
            if np.any(s < pv):
                raise OracleOverflow("per-vertex count does not fit in uint64")
            pv = s
    if t >= 1 << 64:
        raise OracleOverflow("count does not fit in uint64")
    return int(t), pv[:dag.n]


def count_arc(dag: Dag, k: int, u: int, v: int) -> int:
    """k-cliques whose two lowest vertices in the order are the arc u->v."""
    lib = _load()
    slo = ctypes.c_uint64()
    shi = ctypes.c_uint64()
    adj = dag.adj if dag.adj.size else np.zeros(1, np.uint32)
    _check(lib.or_count_arc(dag.n, _p(dag.ptr), _p(adj), k, u, v, ctypes.byref(slo), ctypes.byref(shi)))
    t = (shi.value << 64) | slo.value
    if t >= 1 << 64:
        raise OracleOverflow("count does not fit in uint64")
    return int(t)


def neighbourhood(g, v: int):
    """The subgraph induced by N(v) (undirected neighbours of v), its vertex i
    being the i-th neighbour of v in id order."""
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    nb = np.asarray(g.col[rp[v]:rp[v + 1]], dtype=np.int64)
    src, dst = [], []
    for i, w in enumerate(nb):
        row = np.asarray(g.col[rp[w]:rp[w + 1]], dtype=np.int64)
        pos = np.searchsorted(nb, row)
        hit = pos < nb.size
        hit[hit] = nb[pos[hit]] == row[hit]
        src.append(np.full(int(hit.sum()), i, dtype=np.int64))
        dst.append(pos[hit])
    s2 = np.concatenate(src) if src else np.zeros(0, np.int64)
    d2 = np.concatenate(dst) if dst else np.zeros(0, np.int64)
    order = np.lexsort((d2, s2))
    row_ptr = np.zeros(nb.size + 1, dtype=np.uint64)
    np.cumsum(np.bincount(s2, minlength=nb.size), out=row_ptr[1:])
    return _G(int(nb.size), row_ptr, d2[order].astype(np.uint32))


def count_containing(g, k: int, v: int) -> int:
    """Number of k-cliques that contain v, from the definition: such a clique
    is v together with a (k-1)-clique of the subgraph induced by N(v). This
    is the per-vertex count of Section 3.2 computed without any per-vertex
    bookkeeping."""
    if k < 1:
        raise ValueError("k must be >= 1")
    if k == 1:
        return 1
    return count(orient(neighbourhood(g, v), "degree"), k - 1)


def brute(g, k: int) -> tuple[int, np.ndarray]:
    """Enumerate all k-subsets (the definition of a k-clique); for n <= ~30."""
    lib = _load()
    from_csr = np.zeros((g.n, g.n), dtype=np.uint8)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    from_csr[src, g.col.astype(np.int64)] = 1
    tot = ctypes.c_uint64()
    pv = np.zeros(max(g.n, 1), dtype=np.uint64)
    _check(lib.or_brute(g.n, _p(from_csr), k, ctypes.byref(tot), _p(pv)))
    return int(tot.value), pv[:g.n]


def timed_count(g, k: int, threads: int, method: str = "degree", max_seconds: float | None = None):
    """Orient + count as in the paper's timing (orientation included, load excluded).

    Returns (total, seconds, roots_done). With max_seconds the roots are taken in
    slices until the budget is spent, so the caller can scale a bounded sample.
    """
    t0 = time.perf_counter()
    dag = orient(g, method)
    if max_seconds is None:
        tot = count(dag, k, threads=threads)
        return tot, time.perf_counter() - t0, dag.n
    tot, done = 0, 0
    step = max(1, dag.n // 256)
    while done < dag.n and time.perf_counter() - t0 < max_seconds:
        hi = min(dag.n, done + step)
        tot += count(dag, k, threads=threads, lo=done, hi=hi)
        done = hi
    return tot, time.perf_counter() - t0, done


@dataclass
class PeelResult:
    rounds: int
    best_rounds: int
    best_cliques: int
    best_vertices: int
    total: int


def _induced(g, keep: np.ndarray):
    """The subgraph induced by the vertices with keep[v], relabelled 0..n'-1
    in id order (so that its vertex i is the i-th kept id)."""
    ids = np.nonzero(keep)[0]
    new = np.full(g.n, -1, dtype=np.int64)
    new[ids] = np.arange(ids.size)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    dst = g.col.astype(np.int64)
    sel = keep[src] & keep[dst]
    s2, d2 = new[src[sel]], new[dst[sel]]
    n2 = ids.size
    order = np.lexsort((d2, s2))
    s2, d2 = s2[order], d2[order]
    row_ptr = np.zeros(n2 + 1, dtype=np.uint64)
    np.cumsum(np.bincount(s2, minlength=n2), out=row_ptr[1:])
    return _G(n2, row_ptr, d2.astype(np.uint32)), ids


@dataclass
class _G:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])


def peel_approx(g, k: int, eps_num: int, eps_den: int):
    """arb-approx-peel (Section 4.2) by its definition: every round removes the
    remaining vertices whose k-clique count (in the graph induced by the
    remaining set S) is at most floor(k (1 + eps) t(S) / |S|), eps =
    eps_num / eps_den, in exact integers; counts recomputed from scratch
    each round. Returns (PeelResult, rounds int64[n]) like peel."""
    return _peel(g, k, (eps_num, eps_den))


def peel(g, k: int):
    """arb-peel (Algorithm 2) by its definition: every round removes all
    remaining vertices whose k-clique count in the graph induced by the
    remaining vertices is the minimum; the counts are recomputed from scratch
    on the remaining graph each round (the paper's Update keeps the same
    counts incrementally). The best density (k-cliques per vertex) over the
    graph itself and every remainder is kept as an exact fraction.
    Returns (PeelResult, rounds int64[n])."""
    return _peel(g, k, None)


def _peel(g, k: int, eps):
    n = g.n
    rounds = np.full(n, -1, dtype=np.int64)
    keep = np.ones(n, dtype=bool)
    total = None
    best = None
    r = 0
    while keep.any():
        sub, ids = _induced(g, keep)
        t, pv = count_per_vertex(orient(sub, "degree"), k)
        if total is None:
            total = t
            best = (t, n, 0)
        if eps is None:
            peel_now = ids[pv == pv.min()]
        else:
            thr = (k * (eps[1] + eps[0]) * t) // (ids.size * eps[1])
            peel_now = ids[pv <= thr]
        rounds[peel_now] = r
        keep[peel_now] = False
        remaining = int(keep.sum())
        if remaining:
            sub2, _ = _induced(g, keep)
            t2 = count(orient(sub2, "degree"), k)
            if t2 * best[1] > best[0] * remaining:
                best = (t2, remaining, r + 1)
        r += 1
    if total is None:
        total, best = 0, (0, 0, 0)
    return PeelResult(r, best[2], best[0], best[1], total), rounds


_MASK64 = (1 << 64) - 1


def splitmix64(state: int) -> int:
    """splitmix64 output for a given state (Steele, Lea and Flood, 2014)."""
    z = state & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def vertex_colors(n: int, colors: int, seed: int) -> np.ndarray:
    """Color of every vertex: splitmix64(seed + (v + 1) * gamma), high 32 bits
    scaled to [0, colors)."""
    gamma = 0x9E3779B97F4A7C15
    out = np.empty(n, dtype=np.int64)
    for v in range(n):
        z = splitmix64((seed + (v + 1) * gamma) & _MASK64)
        out[v] = ((z >> 32) * colors) >> 32
    return out


def colorful_count(g, k: int, colors: int, seed: int):
    """Colorful sparsification (Section 3.3): keep the edges whose endpoints
    share a color, count k-cliques exactly. Returns (C, C * colors^(k-1))."""
    col = vertex_colors(g.n, colors, seed)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    dst = g.col.astype(np.int64)
    keep = col[src] == col[dst]
    s2, d2 = src[keep], dst[keep]
    row_ptr = np.zeros(g.n + 1, dtype=np.uint64)
    np.cumsum(np.bincount(s2, minlength=g.n), out=row_ptr[1:])
    sub = _G(g.n, row_ptr, d2.astype(np.uint32))  # rows stay sorted: a filtered sorted row
    c = count(orient(sub, "degree"), k)
    return c, c * colors ** (k - 1)


def _peel_rounds(g, deg, alive, thr_of):
    """Rounds that remove every alive vertex whose induced degree is at most
    thr_of(m_S, |S|), decrementing the induced degrees of the survivors.
    Yields (selected mask, degrees at removal) per round."""
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr.astype(np.int64)))
    dst = g.col.astype(np.int64)
    while alive.any():
        S = int(alive.sum())
        mS = int(deg[alive].sum()) // 2
        sel = alive & (deg <= thr_of(mS, S))
        if not sel.any():
            raise OracleError("a removal round selected no vertex")
        at_removal = deg.copy()
        keep = alive & ~sel
        e = sel[src] & keep[dst]
        deg = deg - np.bincount(dst[e], minlength=g.n)
        alive = keep
        yield sel, at_removal, mS, S


def be_order(g):
    """Barenboim-Elkin order (Section 3.1) with epsilon = 1, as its steps read:
    first the approximate densest subgraph -- rounds removing every vertex of
    induced degree <= 2 (1 + eps) |E(S)| / |S| = 4 |E(S)| / |S|, keeping the
    largest |E(S)| / |S| seen, rho~ -- then alpha~ = 2 (1 + eps) rho~ = 4 rho~
    and rounds removing every vertex of induced degree < (2 + eps) alpha~ =
    12 rho~ (integer division keeps both thresholds exact). Vertices are
    ordered by (round, induced degree at removal, id).
    Returns (rank, round, degree at removal, (rho~ numerator, denominator))."""
    deg0 = np.diff(g.row_ptr.astype(np.int64))
    best = (0, 1)
    for _, _, mS, S in _peel_rounds(g, deg0.copy(), np.ones(g.n, dtype=bool), lambda m, s: (4 * m) // s):
        if mS * best[1] > best[0] * S:
            best = (mS, S)
    thr = 0 if best[0] == 0 else (12 * best[0] - 1) // best[1]
    rnd = np.zeros(g.n, dtype=np.int64)
    dge = np.zeros(g.n, dtype=np.int64)
    for r, (sel, at, _, _) in enumerate(_peel_rounds(g, deg0.copy(), np.ones(g.n, dtype=bool), lambda m, s: thr)):
        rnd[sel] = r
        dge[sel] = at[sel]
    order = np.lexsort((np.arange(g.n), dge, rnd))
    rank = np.empty(g.n, dtype=np.uint32)
    rank[order] = np.arange(g.n, dtype=np.uint32)
    return rank, rnd, dge, best
