"""Pins for the CPU oracle: facts fixed by the paper and by mathematics, not by the oracle itself.

Every test here runs on the CPU. A plausible slip in the oracle (a dropped
term, a wrong arc direction, a missed per-vertex credit, an off-by-one level)
breaks at least one of them.
"""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2002_10047_gb300 import graphgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- helpers
def py_brute(g, k):
    """Definition of a k-clique, enumerated with itertools (independent of the C code)."""
    adj = gg.dense_adjacency(g).astype(bool)
    tot, pv = 0, np.zeros(g.n, dtype=np.int64)
    for s in itertools.combinations(range(g.n), k):
        if all(adj[a, b] for a, b in itertools.combinations(s, 2)):
            tot += 1
            pv[list(s)] += 1
    return tot, pv


def elem_sym(vals, k):
    """e_k(vals) by the standard product expansion prod (1 + a x)."""
    e = [1] + [0] * k
    for a in vals:
        for j in range(k, 0, -1):
            e[j] += e[j - 1] * a
    return e[k]


ORDERS = ["degree", "degeneracy", "original", "gp", "be"]


def small_graphs():
    out = []
    for n, p, seed in [(8, 0.5, 1), (12, 0.6, 2), (14, 0.45, 3), (16, 0.7, 4), (10, 1.0, 5), (9, 0.0, 6)]:
        out.append((f"er{n}_{p}", gg.erdos_renyi(n, p, seed)))
    out.append(("ba15", gg.barabasi_albert(15, 3, 7)))
    return out


# --------------------------------------------------- brute force (pin i)
@pytest.mark.parametrize("name,g", small_graphs())
def test_brute_force_python(name, g):
    for order in ORDERS:
        dag = oracle.orient(g, order)
        for k in range(1, 8):
            want, want_pv = py_brute(g, k)
            tot, pv = oracle.count_per_vertex(dag, k)
            assert tot == want, (name, order, k)
            assert oracle.count(dag, k) == want
            np.testing.assert_array_equal(pv.astype(np.int64), want_pv)


def test_brute_force_c_n30():
    for seed, p in [(11, 0.5), (12, 0.7), (13, 0.85)]:
        g = gg.erdos_renyi(30, p, seed)
        dag = oracle.orient(g, "degree")
        for k in range(1, 9):
            want, want_pv = oracle.brute(g, k)
            tot, pv = oracle.count_per_vertex(dag, k)
            assert tot == want
            np.testing.assert_array_equal(pv, want_pv)


def test_c_brute_matches_python_brute():
    g = gg.erdos_renyi(13, 0.55, 21)
    for k in range(1, 7):
        a, apv = oracle.brute(g, k)
        b, bpv = py_brute(g, k)
        assert a == b
        np.testing.assert_array_equal(apv.astype(np.int64), bpv)


# ------------------------------------------------- closed forms (ii, iii)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 17, 33, 40])
def test_complete_graph(n):
    g = gg.complete(n)
    for order in ("degree", "gp"):
        dag = oracle.orient(g, order)
        for k in range(1, 9):
            tot, pv = oracle.count_per_vertex(dag, k)
            assert tot == math.comb(n, k)
            assert np.all(pv == math.comb(n - 1, k - 1))


@pytest.mark.parametrize("parts", [[3, 3, 3], [1, 2, 3, 4], [5, 5, 5, 5, 5], [2, 7, 1, 6, 3, 4]])
def test_turan_graph(parts):
    g = gg.turan(parts)
    dag = oracle.orient(g, "degeneracy")
    label = np.repeat(np.arange(len(parts)), parts)
    for k in range(1, 8):
        tot, pv = oracle.count_per_vertex(dag, k)
        assert tot == elem_sym(parts, k)
        for j, a in enumerate(parts):
            rest = parts[:j] + parts[j + 1:]
            assert np.all(pv[label == j] == elem_sym(rest, k - 1))


# ---------------------------------------------------------- triangles (iv)
@pytest.mark.parametrize("which", ["er2000", "rmat12", "ba3000"])
def test_triangles_trace(which):
    if which == "er2000":
        g = gg.config_er_2000()
    elif which == "rmat12":
        g = gg.rmat(12, 16, seed=9)
    else:
        g = gg.barabasi_albert(3000, 8, 3)
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    a = sp.csr_matrix((np.ones(g.nnz, dtype=np.int64), (src, g.col.astype(np.int64))), shape=(g.n, g.n))
    diag = np.asarray((a @ a).multiply(a).sum(axis=1)).ravel()  # diag(A^3)_i
    dag = oracle.orient(g, "degree")
    tot, pv = oracle.count_per_vertex(dag, 3)
    assert 6 * tot == int(diag.sum())
    np.testing.assert_array_equal(2 * pv.astype(np.int64), diag)


# ------------------------------------------------------ invariants (v-ix)
def test_additivity_disjoint_union():
    parts = [gg.erdos_renyi(40, 0.3, 31), gg.complete(9), gg.barabasi_albert(60, 4, 32), gg.turan([3, 4, 5])]
    u = gg.disjoint_union(parts)
    for k in range(1, 7):
        tot, pv = oracle.count_per_vertex(oracle.orient(u, "degree"), k)
        sums, pvs = 0, []
        for p in parts:
            t, q = oracle.count_per_vertex(oracle.orient(p, "gp"), k)
            sums += t
            pvs.append(q)
        assert tot == sums
        np.testing.assert_array_equal(pv, np.concatenate(pvs))


def test_orientation_and_relabel_invariance():
    g = gg.rmat(10, 12, seed=41)
    perm = gg.permutation(g.n, 42)
    h = gg.relabel(g, perm)
    rnd_rank = gg.permutation(g.n, 43)
    for k in range(1, 7):
        ref, ref_pv = oracle.count_per_vertex(oracle.orient(g, "degree"), k)
        for order in ORDERS:
            t, pv = oracle.count_per_vertex(oracle.orient(g, order), k)
            assert t == ref
            np.testing.assert_array_equal(pv, ref_pv)
        t, pv = oracle.count_per_vertex(oracle.orient(g, "perm", rnd_rank), k)
        assert t == ref
        np.testing.assert_array_equal(pv, ref_pv)
        t, pv = oracle.count_per_vertex(oracle.orient(h, "degeneracy"), k)
        assert t == ref
        np.testing.assert_array_equal(pv[perm.astype(np.int64)], ref_pv)


def test_sum_per_vertex_and_small_k():
    g = gg.erdos_renyi(300, 0.08, 51)
    dag = oracle.orient(g, "degree")
    deg = g.degrees()
    t1, pv1 = oracle.count_per_vertex(dag, 1)
    assert t1 == g.n and np.all(pv1 == 1)
    t2, pv2 = oracle.count_per_vertex(dag, 2)
    assert t2 == g.m
    np.testing.assert_array_equal(pv2.astype(np.int64), deg)
    for k in range(3, 7):
        t, pv = oracle.count_per_vertex(dag, k)
        assert int(pv.sum()) == k * t


def test_bipartite_and_planted():
    b = gg.random_bipartite(20, 25, 0.5, 61)
    dag = oracle.orient(b, "degree")
    assert oracle.count(dag, 2) == b.m
    for k in range(3, 7):
        assert oracle.count(dag, k) == 0
    n = 400
    perm = gg.permutation(n, 62)
    sizes = [3, 5, 8, 13, 21, 30]
    sets, off = [], 0
    for s in sizes:
        sets.append(perm[off:off + s])
        off += s
    eu, ev = gg.clique_pairs(sets)
    g = gg.from_edges(n, eu, ev)
    dag = oracle.orient(g, "gp")
    for k in range(1, 9):
        want = sum(math.comb(s, k) for s in sizes) + (n - off if k == 1 else 0)
        assert oracle.count(dag, k) == want


def test_count_arc_sums_to_total():
    g = gg.erdos_renyi(60, 0.35, 71)
    dag = oracle.orient(g, "degree")
    src = np.repeat(np.arange(dag.n), np.diff(dag.ptr).astype(np.int64))
    for k in range(2, 7):
        s = sum(oracle.count_arc(dag, k, int(u), int(v)) for u, v in zip(src, dag.adj))
        assert s == oracle.count(dag, k)


def test_count_containing_is_the_per_vertex_definition():
    """k-cliques through v = (k-1)-cliques of N(v): against brute force per
    vertex, C(n-1, k-1) on K_n, and sum over v = k * total."""
    for name, g in small_graphs():
        for k in (1, 2, 3, 4, 5):
            _, want_pv = py_brute(g, k)
            got = [oracle.count_containing(g, k, v) for v in range(g.n)]
            assert got == want_pv.tolist(), (name, k)
    K = gg.complete(12)
    assert oracle.count_containing(K, 5, 3) == math.comb(11, 4)
    g = gg.rmat(9, 8, seed=4)
    for k in (3, 4):
        tot = oracle.count(oracle.orient(g, "degree"), k)
        assert sum(oracle.count_containing(g, k, v) for v in range(g.n)) == k * tot


def test_empty_and_out_of_range_k():
    g = gg.empty(5)
    dag = oracle.orient(g, "degree")
    assert oracle.count(dag, 1) == 5
    assert oracle.count(dag, 2) == 0
    assert oracle.count(oracle.orient(gg.complete(4), "degree"), 5) == 0
    with pytest.raises(ValueError):
        oracle.count(dag, 0)


def test_root_range_split():
    g = gg.barabasi_albert(500, 6, 81)
    dag = oracle.orient(g, "degree")
    for k in (3, 4, 5):
        whole = oracle.count(dag, k)
        assert oracle.count(dag, k, threads=4) == whole
        assert oracle.count(dag, k, lo=0, hi=200) + oracle.count(dag, k, lo=200) == whole


# ----------------------------------------------------- orderings (own pins)
def test_orientations_are_acyclic_and_complete():
    g = gg.rmat(9, 10, seed=91)
    deg = g.degrees()
    for order in ORDERS:
        dag = oracle.orient(g, order)
        assert dag.m == g.m
        src = np.repeat(np.arange(dag.n), np.diff(dag.ptr).astype(np.int64))
        r = dag.rank.astype(np.int64)
        assert np.all(r[src] < r[dag.adj.astype(np.int64)])
        assert np.array_equal(np.sort(r), np.arange(g.n))
        for v in range(g.n):  # out-lists ascending by id
            row = dag.adj[dag.ptr[v]:dag.ptr[v + 1]]
            assert np.all(np.diff(row.astype(np.int64)) > 0)
        if order == "degree":
            key = deg * (1 << 32) + np.arange(g.n)
            assert np.all(key[src] < key[dag.adj.astype(np.int64)])


def _degeneracy_brute(g):
    """max over all vertex subsets S of the minimum degree in G[S] (the
    definition of degeneracy); for n <= ~16."""
    A = gg.dense_adjacency(g).astype(np.int64)
    best = 0
    for mask in range(1, 1 << g.n):
        idx = [i for i in range(g.n) if mask >> i & 1]
        best = max(best, int(A[np.ix_(idx, idx)].sum(1).min()))
    return best


def _max_out(dag):
    return int(np.diff(dag.ptr.astype(np.int64)).max()) if dag.n else 0


def _degeneracy_graphs():
    rng = np.random.default_rng(33)
    out = [("rmat9", gg.rmat(9, 10, seed=91)), ("ba300", gg.barabasi_albert(300, 4, 5)),
           ("er400", gg.erdos_renyi(400, 0.03, 6)), ("turan", gg.turan([7, 5, 5, 2])),
           ("planted", gg.disjoint_union([gg.complete(9), gg.erdos_renyi(60, 0.1, 8), gg.complete(4)]))]
    n = 200  # R-MAT-like skew plus a planted clique on random ids
    g = gg.rmat(8, 6, seed=12)
    ids = rng.choice(g.n, 12, replace=False)
    eu, ev = g.edges()
    pu, pv = zip(*itertools.combinations(ids.tolist(), 2))
    out.append(("rmat8_planted", gg.from_edges(g.n, np.r_[eu, pu], np.r_[ev, pv])))
    return out


@pytest.mark.parametrize("name,g", _degeneracy_graphs())
def test_degeneracy_order_removes_a_minimum_degree_vertex(name, g):
    """Smallest-last (Matula-Beck), the k-core order of Section 5: each vertex,
    when its rank comes, has the minimum degree in the graph induced by the
    vertices not yet removed, and is the smallest id among those of that
    degree; recomputed here from a dense matrix, step by step. The largest
    out-degree of the orientation is the largest such minimum degree."""
    r = oracle.rank(g, "degeneracy").astype(np.int64)
    order = np.argsort(r)
    assert np.array_equal(r[order], np.arange(g.n))
    A = gg.dense_adjacency(g).astype(np.int64)
    deg = A.sum(1)
    alive = np.ones(g.n, dtype=bool)
    dmax = 0
    for v in order:
        cand = np.nonzero(alive)[0]
        want = cand[np.lexsort((cand, deg[cand]))[0]]
        assert v == want, (name, int(v), int(want))
        dmax = max(dmax, int(deg[v]))
        alive[v] = False
        deg -= A[v]
    assert _max_out(oracle.orient(g, "degeneracy")) == dmax


def test_degeneracy_closed_forms():
    """The largest out-degree of the degeneracy orientation equals the
    degeneracy: 1 for a tree, 2 for a cycle and a grid, n - 1 for K_n, n minus
    the largest part for a complete multipartite (Turan) graph, s - 1 for
    disjoint cliques of size up to s, 0 with no edge; and the brute-force
    maximum of the minimum degree over all vertex subsets on random graphs."""
    rng = np.random.default_rng(5)
    n = 300
    parent = np.array([int(rng.integers(0, i)) for i in range(1, n)], dtype=np.uint32)
    tree = gg.from_edges(n, np.arange(1, n, dtype=np.uint32), parent)
    cyc = gg.from_edges(50, np.arange(50, dtype=np.uint32), (np.arange(50, dtype=np.uint32) + 1) % 50)
    R, C = 9, 13
    v = np.arange(R * C).reshape(R, C)
    grid = gg.from_edges(R * C, np.r_[v[:, :-1].ravel(), v[:-1, :].ravel()],
                         np.r_[v[:, 1:].ravel(), v[1:, :].ravel()])
    cases = [(tree, 1), (cyc, 2), (grid, 2), (gg.complete(23), 22), (gg.empty(7), 0),
             (gg.turan([6, 4, 4, 3]), 17 - 6), (gg.turan([9, 1]), 1),
             (gg.disjoint_union([gg.complete(5), gg.complete(11), gg.complete(3)]), 10)]
    for g, want in cases:
        assert _max_out(oracle.orient(g, "degeneracy")) == want
    for seed in range(6):
        g = gg.erdos_renyi(13, 0.25 + 0.1 * seed, 40 + seed)
        assert _max_out(oracle.orient(g, "degeneracy")) == _degeneracy_brute(g)
    # the degree order can be worse than the degeneracy, never better
    g = gg.rmat(9, 10, seed=91)
    assert _max_out(oracle.orient(g, "degree")) >= _max_out(oracle.orient(g, "degeneracy"))


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_gp_star_by_hand():
    rows = {r[0]: r[1:] for r in _read_golden("gp_star_order.txt")}
    g = gg.from_edges(6, [0] * 5, [1, 2, 3, 4, 5])
    rank, rounds, _ = oracle.gp_rounds(g)
    order = [int(x) for x in rows["order"]]
    assert [int(v) for v in np.argsort(rank)] == order
    assert [int(x) for x in rounds] == [int(x) for x in rows["rounds"]]


def test_gp_round_sizes_and_selection():
    g = gg.barabasi_albert(1000, 5, 101)
    rank, rounds, dg = oracle.gp_rounds(g)
    n_left = g.n
    for r in range(int(rounds.max()) + 1):
        sel = rounds == r
        assert sel.sum() == (n_left + 2) // 3
        n_left -= int(sel.sum())
    assert n_left == 0
    # induced degree at removal never exceeds the induced degree of a vertex still left
    # (checked by recomputing induced degrees round by round with numpy)
    alive = np.ones(g.n, dtype=bool)
    deg = g.degrees().copy()
    src = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    for r in range(int(rounds.max()) + 1):
        sel = rounds == r
        np.testing.assert_array_equal(dg[sel], deg[sel])
        key = deg.astype(np.int64) * (1 << 32) + np.arange(g.n)
        assert key[sel].max() < key[alive & ~sel].min() if (alive & ~sel).any() else True
        alive &= ~sel
        hit = sel[src] & alive[g.col]
        np.subtract.at(deg, g.col[hit].astype(np.int64), 1)
        deg[~alive] = 0


def test_paper_example_fragment():
    """Appendix A, Figure 7 fragments (partial pin: the figure is missing)."""
    rows = _read_golden("paper_example_fragment.txt")
    names = rows[0][1:]
    idx = {nm: i for i, nm in enumerate(names)}
    eu = [idx[r[1]] for r in rows if r[0] == "edge"]
    ev = [idx[r[2]] for r in rows if r[0] == "edge"]
    g = gg.from_edges(len(names), eu, ev)
    dag = oracle.orient(g, "original")  # ids are the order positions
    for r in rows:
        if r[0] == "out":
            v = idx[r[1]]
            got = sorted(int(x) for x in dag.adj[dag.ptr[v]:dag.ptr[v + 1]])
            assert got == sorted(idx[x] for x in r[2:])
    for r in rows:
        if r[0] == "sink_within":  # x has no out-neighbour inside N+(root)
            root, x = idx[r[1]], idx[r[2]]
            nroot = set(int(y) for y in dag.adj[dag.ptr[root]:dag.ptr[root + 1]])
            assert x in nroot
            assert not nroot & set(int(y) for y in dag.adj[dag.ptr[x]:dag.ptr[x + 1]])
    # N+(w2) ∩ N+(u2) = {x2}: one triangle on the arc u2 -> w2
    assert oracle.count_arc(dag, 3, idx["u2"], idx["w2"]) == 1
    for r in rows:
        if r[0] == "clique_from":
            root = idx[r[1]]
            members = sorted(idx[x] for x in r[2:])
            assert min(members) == root
            a = gg.dense_adjacency(g)
            assert all(a[x, y] for x, y in itertools.combinations(members, 2))
            assert oracle.count(dag, 4, lo=root, hi=root + 1) >= 1
    assert oracle.count(dag, 4, lo=idx["v"], hi=idx["v"] + 1) == 1
