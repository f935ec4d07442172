"""Seeded synthetic graph generators (input side only).

This module is shared by the CUDA path's tests and bench and by the CPU
oracle's tests. It holds none of the clique-counting arithmetic: it only
draws edge lists (Erdos-Renyi, R-MAT, Barabasi-Albert, Chung-Lu with planted
cliques) and builds a simple undirected CSR (symmetric, rows sorted, no
self-loops, no duplicates), which is the input the paper's method assumes
(Section 2, "Graph Notation" and "Graph Storage").

The heavy loops live in ``graphgen.c`` (compiled on first use with gcc); the
structural fixtures used by the pins (complete graphs, Turan graphs, disjoint
unions, relabellings) are plain numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(os.path.dirname(_HERE), "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_SRC = os.path.join(_HERE, "graphgen.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared object (no contraction: same graph on any host)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            u32, u64, i64, dbl, cint = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                        ctypes.c_double, ctypes.c_int)
            lib.gg_er.argtypes = [u32, dbl, u64, P, P, i64]
            lib.gg_er.restype = i64
            lib.gg_rmat.argtypes = [cint, u64, dbl, dbl, dbl, u64, cint, P, P, cint]
            lib.gg_rmat.restype = cint
            lib.gg_ba.argtypes = [u32, u32, u64, P, P]
            lib.gg_ba.restype = i64
            lib.gg_chung_lu.argtypes = [u32, dbl, dbl, dbl, u64, u64, P, P, P, cint]
            lib.gg_chung_lu.restype = cint
            lib.gg_planted_sets.argtypes = [u32, u32, u32, u32, u64, P, P]
            lib.gg_planted_sets.restype = i64
            lib.gg_csr.argtypes = [u32, u64, P, P, P, P]
            lib.gg_csr.restype = i64
            lib.gg_permutation.argtypes = [u32, u64, u64, P]
            lib.gg_permutation.restype = None
            lib.gg_dlog.argtypes = [dbl]
            lib.gg_dlog.restype = dbl
            lib.gg_dexp.argtypes = [dbl]
            lib.gg_dexp.restype = dbl
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Csr:
    """Simple undirected graph in CSR form: ``row_ptr`` uint64[n+1], ``col`` uint32[2m]."""
    n: int
    row_ptr: np.ndarray
    col: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]

    def edges(self) -> tuple[np.ndarray, np.ndarray]:
        """Each undirected edge once, as (u, v) with u < v."""
        src = np.repeat(np.arange(self.n, dtype=np.uint32), np.diff(self.row_ptr).astype(np.int64))
        keep = src < self.col
        return src[keep], self.col[keep]


def from_edges(n: int, eu, ev) -> Csr:
    """CSR of the simple graph spanned by the pairs (eu[i], ev[i]) (loops and repeats dropped)."""
    eu = np.ascontiguousarray(eu, dtype=np.uint32)
    ev = np.ascontiguousarray(ev, dtype=np.uint32)
    assert eu.shape == ev.shape
    if eu.size and (int(eu.max()) >= n or int(ev.max()) >= n):
        raise ValueError("vertex id out of range")
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    col = np.empty(max(2 * eu.size, 1), dtype=np.uint32)
    nnz = _load().gg_csr(n, eu.size, _ptr(eu), _ptr(ev), _ptr(row_ptr), _ptr(col))
    if nnz < 0:
        raise MemoryError("gg_csr failed")
    return Csr(n, row_ptr, col[:nnz].copy())


# ----------------------------------------------------------- random families
def erdos_renyi_edges(n: int, p: float, seed: int):
    lib = _load()
    mean = p * n * (n - 1) / 2
    cap = int(mean + 12 * np.sqrt(mean + 1) + 64)
    while True:
        eu = np.empty(cap, dtype=np.uint32)
        ev = np.empty(cap, dtype=np.uint32)
        cnt = lib.gg_er(n, p, seed, _ptr(eu), _ptr(ev), cap)
        if cnt >= 0:
            return eu[:cnt], ev[:cnt]
        cap = -cnt


def erdos_renyi(n: int, p: float, seed: int) -> Csr:
    """G(n, p): every one of the n(n-1)/2 pairs independently with probability p."""
    eu, ev = erdos_renyi_edges(n, p, seed)
    return from_edges(n, eu, ev)


def rmat_edges(scale: int, nedges: int, a: float, b: float, c: float, seed: int,
               permute: bool = True, threads: int | None = None):
    eu = np.empty(nedges, dtype=np.uint32)
    ev = np.empty(nedges, dtype=np.uint32)
    th = threads or min(16, os.cpu_count() or 1)
    rc = _load().gg_rmat(scale, nedges, a, b, c, seed, int(permute), _ptr(eu), _ptr(ev), th)
    if rc != 0:
        raise ValueError(f"gg_rmat failed ({rc})")
    return eu, ev


def rmat(scale: int, edge_factor: int, a=0.57, b=0.19, c=0.19, seed: int = 0,
         permute: bool = True) -> Csr:
    """R-MAT with 2^scale vertices and edge_factor * 2^scale sampled pairs, symmetrised."""
    eu, ev = rmat_edges(scale, edge_factor << scale, a, b, c, seed, permute)
    return from_edges(1 << scale, eu, ev)


def barabasi_albert_edges(n: int, m0: int, seed: int):
    m0 = max(1, int(m0))
    core = min(m0 + 1, n)
    cap = core * (core - 1) // 2 + max(0, n - core) * m0
    eu = np.empty(max(cap, 1), dtype=np.uint32)
    ev = np.empty(max(cap, 1), dtype=np.uint32)
    cnt = _load().gg_ba(n, m0, seed, _ptr(eu), _ptr(ev))
    if cnt < 0:
        raise MemoryError("gg_ba failed")
    return eu[:cnt], ev[:cnt]


def barabasi_albert(n: int, m0: int, seed: int) -> Csr:
    """Preferential attachment: a seed clique on m0+1 vertices, then m0 distinct edges per vertex."""
    eu, ev = barabasi_albert_edges(n, m0, seed)
    return from_edges(n, eu, ev)


def chung_lu_edges(n: int, gamma: float, mean_deg: float, seed: int, i0: float = 1.0,
                   npairs: int | None = None, threads: int | None = None):
    if npairs is None:
        npairs = int(round(mean_deg * n / 2))
    eu = np.empty(npairs, dtype=np.uint32)
    ev = np.empty(npairs, dtype=np.uint32)
    w = np.empty(n, dtype=np.float64)
    th = threads or min(16, os.cpu_count() or 1)
    rc = _load().gg_chung_lu(n, gamma, mean_deg, i0, seed, npairs, _ptr(eu), _ptr(ev), _ptr(w), th)
    if rc != 0:
        raise MemoryError("gg_chung_lu failed")
    return eu, ev, w


def planted_sets(n: int, count: int, smin: int, smax: int, seed: int):
    """`count` random vertex sets with sizes uniform in [smin, smax] (members distinct per set)."""
    sizes = np.empty(count, dtype=np.uint32)
    members = np.empty(max(count * smax, 1), dtype=np.uint32)
    tot = _load().gg_planted_sets(n, count, smin, smax, seed, _ptr(sizes), _ptr(members))
    out, off = [], 0
    for s in sizes.tolist():
        out.append(members[off:off + s].copy())
        off += s
    assert off == tot
    return out


def clique_pairs(sets):
    """All pairs inside each vertex set (the edges of cliques planted on those sets)."""
    us, vs = [], []
    for s in sets:
        s = np.asarray(s, dtype=np.uint32)
        i, j = np.triu_indices(s.size, 1)
        us.append(s[i])
        vs.append(s[j])
    if not us:
        return np.empty(0, np.uint32), np.empty(0, np.uint32)
    return np.concatenate(us), np.concatenate(vs)


def permutation(n: int, seed: int, stream: int = 7) -> np.ndarray:
    perm = np.empty(max(n, 1), dtype=np.uint32)
    _load().gg_permutation(n, seed, stream, _ptr(perm))
    return perm[:n]


def uniform_ints(seed: int, stream: int, count: int, lo: int, hi: int) -> np.ndarray:
    """`count` integers uniform in [lo, hi], from the same counter-based stream as the C side."""
    # a permutation-free draw: reuse the Fisher-Yates stream with bound hi-lo+1 per index
    span = hi - lo + 1
    out = np.empty(count, dtype=np.int64)
    key = _stream_key(seed, stream)
    for i in range(count):
        out[i] = lo + _rnd_below(key, i, span)
    return out


_M64 = (1 << 64) - 1


def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _stream_key(seed: int, stream: int) -> int:
    a = _mix64((seed + 0x9E3779B97F4A7C15) & _M64)
    b = (stream * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _M64
    return _mix64(a ^ b)


def _rnd(key: int, ctr: int) -> int:
    return _mix64((key + (ctr + 1) * 0x9E3779B97F4A7C15) & _M64)


def _rnd_below(key: int, ctr: int, bound: int) -> int:
    return (_rnd(key, ctr) * bound) >> 64


def _rnd_unit(key: int, ctr: int) -> float:
    return ((_rnd(key, ctr) >> 11) + 1) / 9007199254740992.0


# ------------------------------------------------------ structural fixtures
def empty(n: int) -> Csr:
    return Csr(n, np.zeros(n + 1, dtype=np.uint64), np.empty(0, dtype=np.uint32))


def complete(n: int) -> Csr:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j)


def turan(parts) -> Csr:
    """Complete multipartite graph with the given part sizes (Turan graph when balanced)."""
    parts = [int(p) for p in parts]
    n = sum(parts)
    label = np.repeat(np.arange(len(parts)), parts)
    i, j = np.triu_indices(n, 1)
    keep = label[i] != label[j]
    return from_edges(n, i[keep], j[keep])


def random_bipartite(n1: int, n2: int, p: float, seed: int) -> Csr:
    key = _stream_key(seed, 11)
    us, vs = [], []
    ctr = 0
    for a in range(n1):
        for b in range(n2):
            if _rnd_unit(key, ctr) <= p:
                us.append(a)
                vs.append(n1 + b)
            ctr += 1
    return from_edges(n1 + n2, np.array(us, np.uint32), np.array(vs, np.uint32))


def disjoint_union(graphs) -> Csr:
    us, vs, off = [], [], 0
    for g in graphs:
        eu, ev = g.edges()
        us.append(eu.astype(np.int64) + off)
        vs.append(ev.astype(np.int64) + off)
        off += g.n
    if not us:
        return empty(0)
    return from_edges(off, np.concatenate(us), np.concatenate(vs))


def concat_csr(graphs) -> tuple[Csr, np.ndarray]:
    """Disjoint union by concatenating CSRs: graph g's ids shift by off[g].
    Rows stay sorted, so this equals disjoint_union without re-sorting.
    Returns (union, off uint64[len(graphs)+1])."""
    ns = np.array([g.n for g in graphs], dtype=np.int64)
    off = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(ns, out=off[1:])
    nnz = np.array([g.nnz for g in graphs], dtype=np.int64)
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(nnz, out=eoff[1:])
    col = np.empty(int(eoff[-1]), dtype=np.uint32)
    row_ptr = np.empty(int(off[-1]) + 1, dtype=np.int64)
    row_ptr[-1] = eoff[-1]
    for i, g in enumerate(graphs):
        np.add(g.col, np.uint32(off[i]), out=col[eoff[i]:eoff[i + 1]], casting="unsafe")
        np.add(g.row_ptr[:-1].astype(np.int64, copy=False), eoff[i], out=row_ptr[off[i]:off[i + 1]])
    return Csr(int(off[-1]), row_ptr.view(np.uint64), col), off.astype(np.uint64)


def relabel(g: Csr, perm) -> Csr:
    """Graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    eu, ev = g.edges()
    return from_edges(g.n, perm[eu.astype(np.int64)], perm[ev.astype(np.int64)])


def dense_adjacency(g: Csr) -> np.ndarray:
    a = np.zeros((g.n, g.n), dtype=np.uint8)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    a[src, g.col.astype(np.int64)] = 1
    return a


# ------------------------------------------------------- workload recipes
def config_er_2000() -> Csr:
    """Erdos-Renyi G(n=2000, p=0.01), seed 1."""
    return erdos_renyi(2000, 0.01, 1)


def config_rmat20() -> Csr:
    """R-MAT scale 20, edge factor 16, (a,b,c,d) = (0.57,0.19,0.19,0.05), seed 2, ids permuted."""
    return rmat(20, 16, 0.57, 0.19, 0.19, seed=2, permute=True)


def chung_lu_planted_edges(n: int = 50_000_000, gamma: float = 2.1, mean_deg: float = 36.0, cliques: int = 1000,
                           smin: int = 20, smax: int = 200, seed: int = 4, i0: float = 1.0):
    """The endpoint pairs (before deduplication) of chung_lu_planted."""
    eu, ev, _ = chung_lu_edges(n, gamma, mean_deg, seed, i0=i0)
    sets = planted_sets(n, cliques, smin, smax, seed)
    cu, cv = clique_pairs(sets)
    return np.concatenate([eu, cu]), np.concatenate([ev, cv]), sets


def csr_from_edges_on_device(n: int, eu, ev, device="cuda"):
    """(row_ptr int64[n+1], col int32[nnz]) on `device` of the simple graph
    spanned by the pairs: the same CSR as from_edges, built with torch sorts on
    the device (for edge lists too large to sort quickly on the host). Input
    preparation only: nothing of the counting method runs here."""
    import torch
    u = torch.from_numpy(np.ascontiguousarray(eu, dtype=np.uint32).view(np.int32)).to(device).to(torch.int64)
    v = torch.from_numpy(np.ascontiguousarray(ev, dtype=np.uint32).view(np.int32)).to(device).to(torch.int64)
    u &= 0xFFFFFFFF
    v &= 0xFFFFFFFF
    keep = u != v
    u, v = u[keep], v[keep]
    keys = torch.cat([(u << 32) | v, (v << 32) | u])
    del u, v, keep
    keys = torch.unique(keys, sorted=True)
    rows = keys >> 32
    col = (keys & 0xFFFFFFFF).to(torch.int32)
    del keys
    counts = torch.bincount(rows, minlength=n)
    del rows
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=row_ptr[1:])
    return row_ptr, col


def chung_lu_planted(n: int = 50_000_000, gamma: float = 2.1, mean_deg: float = 36.0, cliques: int = 1000,
                     smin: int = 20, smax: int = 200, seed: int = 4, i0: float = 1.0) -> Csr:
    """Chung-Lu power-law graph (weights (i + i0)^(-1/(gamma-1)) scaled to the mean
    degree and capped at sqrt(sum w); sum(w)/2 endpoint pairs drawn in proportion
    to the weights, then deduplicated) plus `cliques` cliques of sizes uniform in
    [smin, smax] planted on uniformly random vertex sets. The full-size default is
    the 50M-vertex workload (about 0.9e9 edges)."""
    eu, ev, _ = chung_lu_planted_edges(n, gamma, mean_deg, cliques, smin, smax, seed, i0)
    return from_edges(n, eu, ev)


@dataclass
class BatchSpec:
    kind: str  # "er" or "ba"
    n: int
    avg_deg: int
    k: int
    seed: int


def batch_specs(count: int = 4096, seed: int = 3, n_lo: int = 50, n_hi: int = 20000,
                d_lo: int = 4, d_hi: int = 64, k_lo: int = 3, k_hi: int = 8) -> list[BatchSpec]:
    """Per-graph parameters of the mixed batch: ER or BA (50/50), n, average degree and k uniform."""
    key = _stream_key(seed, 21)
    specs = []
    for g in range(count):
        base = 8 * g
        kind = "er" if _rnd_below(key, base, 2) == 0 else "ba"
        n = n_lo + _rnd_below(key, base + 1, n_hi - n_lo + 1)
        d = d_lo + _rnd_below(key, base + 2, d_hi - d_lo + 1)
        k = k_lo + _rnd_below(key, base + 3, k_hi - k_lo + 1)
        specs.append(BatchSpec(kind, int(n), int(d), int(k), int(_rnd(key, base + 4) & 0x7FFFFFFF)))
    return specs


def graph_from_spec(sp: BatchSpec) -> Csr:
    if sp.kind == "er":
        p = min(1.0, sp.avg_deg / max(1, sp.n - 1))
        return erdos_renyi(sp.n, p, sp.seed)
    return barabasi_albert(sp.n, max(1, int(round(sp.avg_deg / 2))), sp.seed)


def build_batch(specs, threads: int | None = None) -> list[Csr]:
    th = threads or min(16, os.cpu_count() or 1)
    with ThreadPoolExecutor(th) as ex:
        return list(ex.map(graph_from_spec, specs))
