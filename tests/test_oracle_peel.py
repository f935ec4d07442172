"""Pins of the oracle's arb-peel (Algorithm 2) and arb-approx-peel (Section
4.2), on the CPU.

The peel is pinned by cases whose rounds and densities follow from closed
forms (complete graphs, disjoint unions of two complete graphs, graphs
without k-cliques), by a small graph worked by hand, by the 1/k guarantee
(Section 4.1) against a brute-force densest subset, and by relabelling; the
approximate peel by complete graphs, its 1/(k(1+eps)) guarantee and its
logarithmic round bound."""
import itertools
import math
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg


@pytest.mark.parametrize("n,k", [(5, 3), (8, 4), (12, 5), (7, 7)])
def test_complete_graph_one_round(n, k):
    res, rounds = oracle.peel(gg.complete(n), k)
    assert res.rounds == 1 and res.best_rounds == 0
    assert (res.best_cliques, res.best_vertices) == (comb(n, k), n)
    assert res.total == comb(n, k) and (rounds == 0).all()


@pytest.mark.parametrize("a,b,k", [(5, 9, 3), (6, 9, 4), (7, 12, 5)])
def test_two_complete_graphs(a, b, k):
    g = gg.disjoint_union([gg.complete(a), gg.complete(b)])
    res, rounds = oracle.peel(g, k)
    # the smaller clique's vertices have fewer k-cliques: it goes first
    assert res.rounds == 2
    assert (rounds[:a] == 0).all() and (rounds[a:] == 1).all()
    whole = Fraction(comb(a, k) + comb(b, k), a + b)
    big = Fraction(comb(b, k), b)
    assert big > whole
    assert (res.best_cliques, res.best_vertices, res.best_rounds) == (comb(b, k), b, 1)


def test_no_k_cliques_one_round():
    g = gg.random_bipartite(20, 25, 0.3, 5)
    res, rounds = oracle.peel(g, 3)
    assert res.rounds == 1 and res.total == 0 and (rounds == 0).all()
    assert (res.best_cliques, res.best_vertices, res.best_rounds) == (0, g.n, 0)


def test_triangle_with_pendant_by_hand():
    # triangle 0-1-2 plus vertex 3 attached to 0, k = 3: counts 1,1,1,0.
    # round 0 removes 3 (count 0); the triangle (1 clique, 3 vertices) is
    # denser than the whole graph (1/4); round 1 removes 0, 1, 2.
    g = gg.from_edges(4, [0, 0, 1, 0], [1, 2, 2, 3])
    res, rounds = oracle.peel(g, 3)
    assert rounds.tolist() == [1, 1, 1, 0]
    assert (res.rounds, res.best_rounds, res.best_cliques, res.best_vertices, res.total) == (2, 1, 1, 3, 1)


def _densest_brute(g, k):
    """max over non-empty vertex sets S of (k-cliques inside S) / |S|."""
    a = gg.dense_adjacency(g).astype(bool)
    cl = []
    for c in itertools.combinations(range(g.n), k):
        if all(a[x, y] for x, y in itertools.combinations(c, 2)):
            cl.append(sum(1 << v for v in c))
    cl = np.array(cl, dtype=np.int64)
    best = Fraction(0)
    for S in range(1, 1 << g.n):
        cnt = int(np.count_nonzero((cl & S) == cl)) if cl.size else 0
        best = max(best, Fraction(cnt, bin(S).count("1")))
    return best


@pytest.mark.parametrize("seed,k", [(1, 3), (2, 3), (3, 4), (4, 4), (5, 3)])
def test_one_over_k_guarantee(seed, k):
    g = gg.erdos_renyi(12, 0.55, seed)
    res, _ = oracle.peel(g, k)
    dstar = Fraction(res.best_cliques, res.best_vertices)
    opt = _densest_brute(g, k)
    assert dstar <= opt  # the peel's best is the density of an actual subset
    assert dstar >= opt / k


def test_relabelling_moves_rounds_with_the_vertices():
    g = gg.barabasi_albert(150, 4, 11)
    perm = gg.permutation(g.n, 12)
    res, rounds = oracle.peel(g, 3)
    res2, rounds2 = oracle.peel(gg.relabel(g, perm), 3)
    assert res == res2
    assert np.array_equal(rounds2[perm.astype(np.int64)], rounds)


@pytest.mark.parametrize("n,k", [(6, 3), (9, 4)])
def test_approx_complete_graph_one_round(n, k):
    res, rounds = oracle.peel_approx(gg.complete(n), k, 1, 2)
    assert res.rounds == 1 and (rounds == 0).all()
    assert (res.best_cliques, res.best_vertices) == (comb(n, k), n)


@pytest.mark.parametrize("seed,k,eps", [(1, 3, (1, 2)), (3, 4, (1, 4)), (5, 3, (1, 1)), (2, 3, (0, 1))])
def test_approx_guarantee(seed, k, eps):
    g = gg.erdos_renyi(12, 0.55, seed)
    res, _ = oracle.peel_approx(g, k, *eps)
    dstar = Fraction(res.best_cliques, res.best_vertices)
    opt = _densest_brute(g, k)
    assert dstar <= opt
    assert dstar >= opt / (k * (1 + Fraction(*eps)))


@pytest.mark.parametrize("eps", [(1, 10), (1, 2), (2, 1)])
def test_approx_round_bound(eps):
    g = gg.rmat(10, 12, seed=3)
    res, rounds = oracle.peel_approx(g, 4, *eps)
    e = eps[0] / eps[1]
    assert res.rounds <= math.ceil(math.log(g.n) / math.log1p(e)) + 1
    assert rounds.min() == 0 and rounds.max() == res.rounds - 1
