"""GPU parity with the dense-core bit matrix (kc_orient's KC_CORE_BITS): rows
of the induced subgraphs read from the core's bits instead of scans of the
members' out-lists give the oracle's counts bit-exact, in total, per vertex,
per arc, per root and in arb-peel. The lookup rule is driven to both ends
(ratio 0: every member in the core takes the lookup path; a core of every
vertex; a core of an eighth of the vertices) and to its default, on warp
roots, shared-memory block roots and global-scratch block roots (K_2100)."""
import math

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DEFAULT = (131072, 1)


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_10047_gb300 import build, kclique
    build.build()
    yield kclique
    kclique.kc_set_core_policy(*DEFAULT)


def planted_graph(n=3000, p=0.004, sizes=(40, 70, 100), seed=17):
    eu, ev = gg.erdos_renyi_edges(n, p, seed)
    perm = gg.permutation(n, seed + 2)
    sets, off = [], 0
    for s in sizes:
        sets.append(perm[off:off + s])
        off += s
    cu, cv = gg.clique_pairs(sets)
    return gg.from_edges(n, np.concatenate([eu, cu]), np.concatenate([ev, cv]))


def chung_lu_small():
    """A skewed graph of the Chung-Lu family (exponent 2.1, mean degree 36)
    with planted cliques: light roots whose out-neighbours are the heavy head."""
    return gg.chung_lu_planted(n=40_000, cliques=20, smin=20, smax=60, seed=4)


GRAPHS = {
    "er2000": (gg.config_er_2000, (3, 4, 5)),
    "rmat12": (lambda: gg.rmat(12, 16, seed=3), (3, 4, 5, 6)),
    "ba5000": (lambda: gg.barabasi_albert(5000, 24, 7), (3, 4, 5)),
    "planted": (planted_graph, (3, 4, 5, 6)),
    "rmat10_dense": (lambda: gg.rmat(10, 48, seed=11), (3, 4, 5, 6)),
    "chung_lu_40k": (chung_lu_small, (3, 4, 5)),
}


@pytest.fixture(scope="module")
def graphs():
    return {name: f() for name, (f, _) in GRAPHS.items()}


@pytest.fixture(scope="module")
def want(graphs):
    out = {}
    for name, (_, ks) in GRAPHS.items():
        od = oracle.orient(graphs[name], "degree")
        out[name] = (od, {k: oracle.count_per_vertex(od, k, threads=8) for k in ks})
    return out


def policies(n):
    """(max_vertices, ratio): every vertex in the core and every member in it
    looked up, an eighth of them looked up, the default rule, and a rule that
    mixes lookups and scans inside one root (ratio 4)."""
    return [(n, 0), (max(64, n // 8), 0), DEFAULT, (max(64, n // 8), 4)]


@pytest.mark.parametrize("name", list(GRAPHS))
def test_core_counts_bit_exact(kc, graphs, want, name):
    g = graphs[name]
    od, per_k = want[name]
    rp, col = kc.csr_to_device(g)
    for maxv, ratio in policies(g.n):
        kc.kc_set_core_policy(maxv, ratio)
        dag = kc.orient(rp, col, g.n, core=True)
        assert 0 < dag.core_vertices <= min(maxv, g.n), (name, maxv)
        for k, (tot_w, pv_w) in per_k.items():
            assert kc.count(dag, k) == tot_w, (name, maxv, ratio, k)
            tot, pv = kc.count_per_vertex(dag, k)
            assert tot == tot_w, (name, maxv, ratio, k)
            np.testing.assert_array_equal(kc.as_uint64(pv), pv_w, err_msg=f"{name} {maxv} {ratio} k={k}")
        dag.free()
    kc.kc_set_core_policy(*DEFAULT)


@pytest.mark.parametrize("name", ["rmat12", "planted", "chung_lu_40k"])
def test_core_per_arc_and_rooted(kc, graphs, want, name):
    g = graphs[name]
    od, per_k = want[name]
    rp, col = kc.csr_to_device(g)
    kc.kc_set_core_policy(max(64, g.n // 8), 0)
    try:
        dag = kc.orient(rp, col, g.n, core=True)
        ptr, dcol = dag.export()
        ptr = ptr.cpu().numpy().view(np.uint64)
        dcol = dcol.cpu().numpy().view(np.uint32)
        src = np.repeat(np.arange(g.n), np.diff(ptr.astype(np.int64)))
        rng = np.random.default_rng(3)
        pick = rng.choice(od.m, size=min(300, od.m), replace=False)
        for k in (3, 4):
            tot, pa = kc.count_per_arc(dag, k)
            pa = kc.as_uint64(pa)
            assert int(pa.sum()) == tot == per_k[k][0]
            for e in pick:
                assert int(pa[e]) == oracle.count_arc(od, k, int(src[e]), int(dcol[e])), (name, k, e)
        roots = rng.permutation(g.n)[: min(g.n, 1000)]
        r = torch.from_numpy(roots.astype(np.int32)).cuda()
        for k in (4, 5):
            tot, out = kc.count_roots(dag, k, r)
            w = np.array([oracle.count(od, k, lo=int(u), hi=int(u) + 1) for u in roots], dtype=np.uint64)
            np.testing.assert_array_equal(kc.as_uint64(out), w, err_msg=f"{name} k={k}")
    finally:
        kc.kc_set_core_policy(*DEFAULT)


def test_core_switches(kc, graphs, want):
    """core=False builds none; the automatic rule builds one on the skewed
    graph and none on the Erdos-Renyi graph; a count told not to use the
    core (ratio 2^32 - 1) gives the same counts."""
    g = graphs["chung_lu_40k"]
    rp, col = kc.csr_to_device(g)
    plain = kc.orient(rp, col, g.n, core=False)
    assert plain.core_vertices == 0
    st = kc.dag_stats(plain)
    # the automatic rule: largest out-degree >= 128 and builds reading >= 16
    # out-list entries per arc; this graph is skewed enough for it
    assert st["max_out"] >= 128 and st["sum_arc_head"] >= 16 * plain.m
    dag = kc.orient(rp, col, g.n)
    assert dag.core_vertices > 0
    # the build split under the default rule: fewer out-list entries scanned
    # than the plain build volume, and some rows looked up instead
    sc = kc.dag_stats(dag)
    assert sc["core_vertices"] == dag.core_vertices
    assert st["core_vertices"] == 0 and st["build_lookups"] == 0 and st["build_scanned"] == st["sum_arc_head"]
    assert sc["sum_arc_head"] == st["sum_arc_head"] and 0 < sc["build_scanned"] < st["sum_arc_head"]
    assert sc["build_lookups"] > 0
    ge = graphs["er2000"]
    rpe, cole = kc.csr_to_device(ge)
    assert kc.orient(rpe, cole, ge.n).core_vertices == 0
    od, per_k = want["chung_lu_40k"]
    try:
        kc.kc_set_core_policy(DEFAULT[0], 0xFFFFFFFF)
        assert kc.count(dag, 4) == per_k[4][0]
    finally:
        kc.kc_set_core_policy(*DEFAULT)
    assert kc.count(dag, 4) == per_k[4][0]
    kc.kc_set_core_policy(0, 1)  # no core at all
    try:
        assert kc.orient(rp, col, g.n, core=True).core_vertices == 0
    finally:
        kc.kc_set_core_policy(*DEFAULT)


@pytest.mark.parametrize("n,ks", [(130, (3, 4, 5, 6)), (600, (3, 4, 5)), (1100, (3, 4)), (2100, (3, 4))])
def test_core_complete_graphs(kc, n, ks):
    """K_n with every vertex in the core and every row looked up: closed forms,
    on warp, shared-memory and global-scratch roots."""
    g = gg.complete(n)
    rp, col = kc.csr_to_device(g)
    kc.kc_set_core_policy(n, 0)
    try:
        dag = kc.orient(rp, col, g.n, core=True)
        assert dag.core_vertices == n
        st = kc.dag_stats(dag)
        # every member looked up: one bit per pair of N+(u), sum over u of
        # C(d+(u), 2) = C(n, 3), and nothing scanned
        assert st["build_scanned"] == 0 and st["build_lookups"] == math.comb(n, 3)
        for k in ks:
            assert kc.count(dag, k) == math.comb(n, k)
            tot, pv = kc.count_per_vertex(dag, k)
            assert tot == math.comb(n, k)
            assert np.all(kc.as_uint64(pv) == math.comb(n - 1, k - 1))
    finally:
        kc.kc_set_core_policy(*DEFAULT)


def test_core_peel(kc, graphs):
    """arb-peel's candidate rows take the same core lookups."""
    g = graphs["planted"]
    rp, col = kc.csr_to_device(g)
    kc.kc_set_core_policy(max(64, g.n // 4), 0)
    try:
        dag = kc.orient(rp, col, g.n, core=True)
        assert dag.core_vertices > 0
        for k in (3, 4):
            w, w_rounds = oracle.peel(g, k)
            res, rounds = kc.peel(rp, col, dag, k)
            assert np.array_equal(rounds.cpu().numpy().astype(np.int64), w_rounds), k
            assert res["rounds"] == w.rounds and res["total"] == w.total, k
            assert (res["best_cliques"], res["best_vertices"], res["best_rounds"]) == \
                (w.best_cliques, w.best_vertices, w.best_rounds), k
    finally:
        kc.kc_set_core_policy(*DEFAULT)


def test_core_threshold_digits(kc, graphs, want):
    """The core threshold is found digit by digit over the 64-bit keys: a
    boundary key above 2^9 (degrees 519 / 599 / 699, the core being the K_700
    whose 700 vertices outrank the rest) and Goodrich-Pszona keys (round in
    the high word) give the same counts."""
    g = gg.disjoint_union([gg.complete(520), gg.complete(600), gg.complete(700)])
    rp, col = kc.csr_to_device(g)
    kc.kc_set_core_policy(800, 0)
    try:
        dag = kc.orient(rp, col, g.n, core=True)
        assert dag.core_vertices == 700
        for k in (3, 4):
            want_k = math.comb(520, k) + math.comb(600, k) + math.comb(700, k)
            assert kc.count(dag, k) == want_k
            tot, pv = kc.count_per_vertex(dag, k)
            assert tot == want_k
        for name in ("rmat12", "planted", "chung_lu_40k"):
            h = graphs[name]
            od, per_k = want[name]
            rph, colh = kc.csr_to_device(h)
            kc.kc_set_core_policy(max(64, h.n // 8), 0)
            dag = kc.orient(rph, colh, h.n, method="gp", core=True)
            assert dag.core_vertices > 0, name
            for k in (3, 4):
                tot, pv = kc.count_per_vertex(dag, k)
                assert tot == per_k[k][0], (name, k)
                np.testing.assert_array_equal(kc.as_uint64(pv), per_k[k][1], err_msg=f"{name} gp k={k}")
    finally:
        kc.kc_set_core_policy(*DEFAULT)

