"""GPU parity of arb-peel (Algorithm 2) and arb-approx-peel (Section 4.2)
through the C ABI: the round in which
every vertex is removed, the number of rounds and the best density (an exact
fraction) equal the oracle's peel, for both orientations (the result does
not depend on the orientation)."""
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


def planted(n=400, p=0.02, sizes=(12, 20, 35), seed=31):
    eu, ev = gg.erdos_renyi_edges(n, p, seed)
    perm = gg.permutation(n, seed + 1)
    sets, off = [], 0
    for s in sizes:
        sets.append(perm[off:off + s])
        off += s
    cu, cv = gg.clique_pairs(sets)
    return gg.from_edges(n, np.concatenate([eu, cu]), np.concatenate([ev, cv]))


CASES = {
    "er300": (lambda: gg.erdos_renyi(300, 0.06, 3), (3, 4)),
    "ba500": (lambda: gg.barabasi_albert(500, 6, 4), (3, 4, 5)),
    "rmat9": (lambda: gg.rmat(9, 8, seed=5), (3, 4, 5)),
    "planted": (planted, (3, 4, 6)),
    "turan": (lambda: gg.turan([6, 9, 4, 11]), (3, 4)),
    "k40_plus_er": (lambda: gg.disjoint_union([gg.complete(40), gg.erdos_renyi(200, 0.05, 8)]), (3, 5)),
    "two_cliques": (lambda: gg.disjoint_union([gg.complete(7), gg.complete(11)]), (4,)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_peel_matches_oracle(kc, name):
    make, ks = CASES[name]
    g = make()
    rp, col = kc.csr_to_device(g)
    for k in ks:
        want, want_rounds = oracle.peel(g, k)
        for method in ("degree", "gp"):
            dag = kc.orient(rp, col, g.n, method=method)
            res, rounds = kc.peel(rp, col, dag, k)
            got_rounds = rounds.cpu().numpy().astype(np.int64)
            assert np.array_equal(got_rounds, want_rounds), (name, k, method)
            assert res["rounds"] == want.rounds and res["total"] == want.total, (name, k, method)
            assert (res["best_cliques"], res["best_vertices"], res["best_rounds"]) == \
                (want.best_cliques, want.best_vertices, want.best_rounds), (name, k, method)


def test_peel_edge_cases(kc):
    for g, k in ((gg.empty(6), 3), (gg.random_bipartite(30, 40, 0.2, 2), 3), (gg.complete(50), 4)):
        rp, col = kc.csr_to_device(g)
        dag = kc.orient(rp, col, g.n)
        want, want_rounds = oracle.peel(g, k)
        res, rounds = kc.peel(rp, col, dag, k)
        assert np.array_equal(rounds.cpu().numpy().astype(np.int64), want_rounds)
        assert (res["rounds"], res["best_cliques"], res["best_vertices"]) == \
            (want.rounds, want.best_cliques, want.best_vertices)
    g = gg.complete(10)
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    other = gg.complete(11)
    orp, ocol = kc.csr_to_device(other)
    with pytest.raises(kc.KcError):
        kc.peel(orp, ocol, dag, 3)  # the CSR is not the one the DAG came from
    with pytest.raises(kc.KcError):
        kc.peel(rp, col, dag, 2)


def test_peel_larger_graph_invariants(kc):
    """R-MAT scale 13: the rounds partition the vertices, counts removed add up
    to the total, and degree and GP orientations agree on every vertex."""
    g = gg.rmat(13, 12, seed=7)
    rp, col = kc.csr_to_device(g)
    out = {}
    for method in ("degree", "gp"):
        dag = kc.orient(rp, col, g.n, method=method)
        res, rounds = kc.peel(rp, col, dag, 4)
        out[method] = (res, rounds.cpu().numpy())
        r = out[method][1]
        assert r.min() == 0 and r.max() == res["rounds"] - 1
        assert res["total"] == kc.count(dag, 4)
        assert res["best_cliques"] * g.n >= res["total"] * res["best_vertices"]
    assert out["degree"][0] == out["gp"][0]
    assert np.array_equal(out["degree"][1], out["gp"][1])


@pytest.mark.parametrize("name", ["er300", "ba500", "rmat9", "planted", "k40_plus_er"])
def test_approx_peel_matches_oracle(kc, name):
    from fractions import Fraction
    make, ks = CASES[name]
    g = make()
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    for k in ks:
        for eps in (Fraction(1, 10), Fraction(1, 2), Fraction(2, 1), Fraction(0)):
            want, want_rounds = oracle.peel_approx(g, k, eps.numerator, eps.denominator)
            res, rounds = kc.peel(rp, col, dag, k, epsilon=eps)
            assert np.array_equal(rounds.cpu().numpy().astype(np.int64), want_rounds), (name, k, eps)
            assert (res["rounds"], res["best_cliques"], res["best_vertices"], res["best_rounds"]) == \
                (want.rounds, want.best_cliques, want.best_vertices, want.best_rounds), (name, k, eps)
