"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit-exact.

Counts are integers, so the tolerance is zero everywhere: totals, per-vertex
and per-arc counts must be identical. Graph sizes are chosen so the oracle
finishes in seconds while the device path still exercises all three root
classes (warp roots with out-degree <= 64, block roots with the bit matrix in
shared memory, and block roots with the matrix in global scratch).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_10047_gb300 import build, kclique
    build.build()
    return kclique


def gpu_orient(kc, g, method="degree", sym=False):
    rp, col = kc.csr_to_device(g)
    return kc.orient(rp, col, g.n, method=method, validate_symmetry=sym)


def rank_ordered(od):
    """The oracle's out-lists re-sorted into its total order (the library's export order)."""
    src = np.repeat(np.arange(od.n), np.diff(od.ptr.astype(np.int64)))
    order = np.lexsort((od.rank[od.adj.astype(np.int64)], src))
    return od.adj[order]


def exported_arcs(dag):
    """(src, dst) of every arc of the device DAG, in export order."""
    ptr, col = dag.export()
    ptr = ptr.cpu().numpy().view(np.uint64)
    col = col.cpu().numpy().view(np.uint32)
    src = np.repeat(np.arange(len(ptr) - 1), np.diff(ptr.astype(np.int64)))
    return ptr, col, src


def planted_graph(n=3000, p=0.004, sizes=(40, 70, 100), seed=17):
    eu, ev = gg.erdos_renyi_edges(n, p, seed)
    sets = gg.planted_sets(n, len(sizes), min(sizes), max(sizes), seed + 1)
    # force the requested sizes exactly
    perm = gg.permutation(n, seed + 2)
    sets, off = [], 0
    for s in sizes:
        sets.append(perm[off:off + s])
        off += s
    cu, cv = gg.clique_pairs(sets)
    return gg.from_edges(n, np.concatenate([eu, cu]), np.concatenate([ev, cv]))


GRAPHS = {
    "er2000": (gg.config_er_2000, range(1, 9)),
    "rmat12": (lambda: gg.rmat(12, 16, seed=3), range(1, 8)),
    "rmat14": (lambda: gg.rmat(14, 16, seed=5), range(3, 6)),
    "ba5000": (lambda: gg.barabasi_albert(5000, 24, 7), range(2, 8)),
    "planted": (planted_graph, range(3, 6)),
    "turan": (lambda: gg.turan([17, 23, 31, 9, 40]), range(1, 7)),
    "rmat10_dense": (lambda: gg.rmat(10, 48, seed=11), range(3, 8)),
}


@pytest.fixture(scope="module")
def graphs():
    return {name: f() for name, (f, _) in GRAPHS.items()}


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("method", ["degree", "gp", "be"])
def test_orientation_bit_exact(kc, graphs, name, method):
    g = graphs[name]
    dag = gpu_orient(kc, g, method)
    od = oracle.orient(g, method)
    ptr, col = dag.export()
    assert dag.n == g.n and dag.m == g.m
    np.testing.assert_array_equal(ptr.cpu().numpy().view(np.uint64), od.ptr)
    np.testing.assert_array_equal(col.cpu().numpy().view(np.uint32), rank_ordered(od))
    assert dag.max_out_degree == int(np.diff(od.ptr.astype(np.int64)).max(initial=0))


@pytest.mark.parametrize("name", list(GRAPHS))
def test_counts_bit_exact(kc, graphs, name):
    g = graphs[name]
    ks = GRAPHS[name][1]
    dag = gpu_orient(kc, g, "degree")
    odag = oracle.orient(g, "degree")
    for k in ks:
        want, want_pv = oracle.count_per_vertex(odag, k, threads=8)
        assert kc.count(dag, k) == want, (name, k)
        tot, pv = kc.count_per_vertex(dag, k)
        assert tot == want, (name, k)
        np.testing.assert_array_equal(kc.as_uint64(pv), want_pv, err_msg=f"{name} k={k}")


@pytest.mark.parametrize("name", ["er2000", "rmat12", "planted", "turan"])
def test_per_arc_bit_exact(kc, graphs, name):
    g = graphs[name]
    dag = gpu_orient(kc, g, "degree")
    odag = oracle.orient(g, "degree")
    _, col, src = exported_arcs(dag)
    rng = np.random.default_rng(5)
    pick = rng.choice(odag.m, size=min(400, odag.m), replace=False)
    for k in (2, 3, 4, 5):
        tot, pa = kc.count_per_arc(dag, k)
        pa = kc.as_uint64(pa)
        assert int(pa.sum()) == tot == oracle.count(odag, k, threads=8)
        for e in pick:
            assert int(pa[e]) == oracle.count_arc(odag, k, int(src[e]), int(col[e])), (name, k, e)


@pytest.mark.parametrize("name", ["rmat12", "planted", "turan", "rmat10_dense"])
def test_rooted_counts_bit_exact(kc, graphs, name):
    """kc_count_roots: every root's count against the oracle's top call for
    that root alone (Algorithm 1 from one vertex), on a shuffled root list
    covering warp, shared-memory and (rmat10_dense at d+ > 64) block roots."""
    g = graphs[name]
    dag = gpu_orient(kc, g, "degree")
    odag = oracle.orient(g, "degree")
    rng = np.random.default_rng(9)
    roots = rng.permutation(g.n)[: min(g.n, 1500)]
    r = torch.from_numpy(roots.astype(np.int32)).cuda()
    for k in GRAPHS[name][1]:
        tot, out = kc.count_roots(dag, k, r)
        want = np.array([oracle.count(odag, k, lo=int(u), hi=int(u) + 1) for u in roots], dtype=np.uint64)
        np.testing.assert_array_equal(kc.as_uint64(out), want, err_msg=f"{name} k={k}")
        assert tot == int(want.astype(object).sum())


def test_rooted_counts_edges(kc):
    """All roots sum to the total (including roots in global scratch, K_2100);
    an empty list; repeated or out-of-range ids are rejected."""
    g = gg.complete(2100)
    dag = gpu_orient(kc, g, "degree")
    every = torch.arange(g.n, dtype=torch.int32, device="cuda")
    for k in (1, 2, 3, 4):
        tot, out = kc.count_roots(dag, k, every)
        out = kc.as_uint64(out)
        assert tot == math.comb(2100, k) == int(out.astype(object).sum())
        # the vertex of rank i roots C(2099 - i, k - 1) cliques
        ptr, _, _ = exported_arcs(dag)
        dplus = np.diff(ptr.astype(np.int64))
        assert all(int(out[v]) == math.comb(int(dplus[v]), k - 1) for v in range(0, g.n, 97))
    tot, out = kc.count_roots(dag, 4, torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert tot == 0 and out.numel() == 0
    with pytest.raises(kc.KcError):
        kc.count_roots(dag, 4, torch.tensor([3, 5, 3], dtype=torch.int32, device="cuda"))
    with pytest.raises(kc.KcError):
        kc.count_roots(dag, 4, torch.tensor([3, 2100], dtype=torch.int32, device="cuda"))


def test_build_staging_modes_agree(kc, graphs):
    """The level-2 build staged with bulk copies and read with ordinary loads
    (the default) give the same counts, per vertex too, on graphs with
    shared-memory and global-scratch block roots (K_2100)."""
    cases = [(graphs["rmat10_dense"], (3, 4, 5, 6)), (graphs["rmat14"], (3, 4, 5)), (gg.complete(2100), (3, 4))]
    try:
        for g, ks in cases:
            dag = gpu_orient(kc, g, "degree")
            for k in ks:
                kc.kc_set_bulk_build(True)
                t1, p1 = kc.count_per_vertex(dag, k)
                c1 = kc.count(dag, k)
                kc.kc_set_bulk_build(False)
                t2, p2 = kc.count_per_vertex(dag, k)
                c2 = kc.count(dag, k)
                assert t1 == t2 == c1 == c2, (g.n, k)
                np.testing.assert_array_equal(kc.as_uint64(p1), kc.as_uint64(p2))
    finally:
        kc.kc_set_bulk_build(False)


def test_dag_stats(kc, graphs):
    for name in ("rmat12", "planted", "turan"):
        g = graphs[name]
        dag = gpu_orient(kc, g, "degree")
        st = kc.dag_stats(dag)
        ptr, col, src = exported_arcs(dag)
        dout = np.diff(ptr.astype(np.int64))
        assert st["max_out"] == int(dout.max(initial=0))
        assert st["sum_out_sq"] == int((dout * dout).sum())
        assert st["sum_arc_head"] == int(dout[col.astype(np.int64)].sum())
        assert st["triangles"] == oracle.count(oracle.orient(g, "degree"), 3)


def test_gp_orientation_counts(kc, graphs):
    for name in ("rmat12", "planted", "ba5000"):
        g = graphs[name]
        dag = gpu_orient(kc, g, "gp")
        odag = oracle.orient(g, "gp")
        for k in (3, 4, 5):
            want, want_pv = oracle.count_per_vertex(odag, k, threads=8)
            tot, pv = kc.count_per_vertex(dag, k)
            assert tot == want
            np.testing.assert_array_equal(kc.as_uint64(pv), want_pv)


@pytest.mark.parametrize("n,ks", [(66, range(1, 9)), (130, range(3, 7)), (600, (3, 4, 5)), (1100, (3, 4)),
                                  (2100, (3, 4)), (4200, (3,))])
def test_complete_graphs_closed_form(kc, n, ks):
    """K_n: C(n,k) in total and C(n-1,k-1) per vertex; large n drives roots into
    global-scratch matrices with several words per lane."""
    g = gg.complete(n)
    dag = gpu_orient(kc, g, "degree")
    assert dag.max_out_degree == n - 1
    for k in ks:
        assert kc.count(dag, k) == math.comb(n, k)
        tot, pv = kc.count_per_vertex(dag, k)
        assert tot == math.comb(n, k)
        pv = kc.as_uint64(pv)
        assert np.all(pv == math.comb(n - 1, k - 1))


def test_deep_k(kc):
    """Deep recursion up to k = KC_KMAX = 32 (the search is pruned hard near k = n)."""
    g = gg.complete(24)
    dag = gpu_orient(kc, g, "degree")
    for k in (12, 23, 24):
        assert kc.count(dag, k) == math.comb(24, k)
        tot, pv = kc.count_per_vertex(dag, k)
        assert np.all(kc.as_uint64(pv) == math.comb(23, k - 1))
    g = gg.complete(33)
    dag = gpu_orient(kc, g, "gp")
    for k in (31, 32):
        assert kc.count(dag, k) == math.comb(33, k)
        tot, pv = kc.count_per_vertex(dag, k)
        assert np.all(kc.as_uint64(pv) == math.comb(32, k - 1))
    assert kc.count(dag, 32) == 33
    with pytest.raises(kc.KcError):
        kc.count(dag, 33)
    with pytest.raises(kc.KcError):
        kc.count(dag, 0)


def test_empty_and_tiny(kc):
    for g in (gg.empty(0), gg.empty(7), gg.from_edges(2, [0], [1]), gg.complete(3)):
        dag = gpu_orient(kc, g, "degree")
        for k in range(1, 6):
            want = math.comb(g.n, k) if g.m == g.n * (g.n - 1) // 2 else (g.n if k == 1 else (g.m if k == 2 else 0))
            assert kc.count(dag, k) == want
            if g.n:
                tot, pv = kc.count_per_vertex(dag, k)
                assert tot == want
                assert int(kc.as_uint64(pv).sum()) == k * want


def test_malformed_csr_rejected(kc):
    good = gg.complete(6)
    rp, col = good.row_ptr.copy(), good.col.copy()

    def attempt(rp_, col_, n=6, sym=False):
        r = torch.from_numpy(rp_.astype(np.int64)).cuda()
        c = torch.from_numpy(col_.view(np.int32) if col_.dtype == np.uint32 else col_.astype(np.int32)).cuda()
        return kc.orient(r, c, n, validate_symmetry=sym)

    attempt(rp, col)  # sanity
    bad = col.copy()
    bad[1], bad[2] = bad[2], bad[1]  # unsorted row
    with pytest.raises(kc.KcError):
        attempt(rp, bad)
    bad = col.copy()
    bad[0] = 0  # self-loop in row 0
    with pytest.raises(kc.KcError):
        attempt(rp, bad)
    bad = col.copy()
    bad[-1] = 9  # id out of range
    with pytest.raises(kc.KcError):
        attempt(rp, bad)
    bad_rp = rp.copy()
    bad_rp[-1] += 2  # offsets disagree with nnz
    with pytest.raises(kc.KcError):
        attempt(bad_rp, col)
    # asymmetric: drop one arc of an edge and add an unmatched one elsewhere
    g = gg.from_edges(6, [0, 1, 2], [1, 2, 3])
    rp2, col2 = g.row_ptr.copy(), g.col.copy()
    col2[0] = 2  # row 0 now {2} although 2 does not list 0
    with pytest.raises(kc.KcError):
        attempt(rp2, col2, sym=True)


def test_config_er2000_full(kc):
    """G(2000, 0.01), seed 1: exact 4-clique total and per-vertex counts (and k = 3)."""
    g = gg.config_er_2000()
    dag = gpu_orient(kc, g, "degree")
    odag = oracle.orient(g, "degree")
    for k in (3, 4):
        want, want_pv = oracle.count_per_vertex(odag, k)
        tot, pv = kc.count_per_vertex(dag, k)
        assert tot == want
        np.testing.assert_array_equal(kc.as_uint64(pv), want_pv)
