"""Pins of the oracle's Barenboim-Elkin order (Section 3.1, epsilon = 1)."""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg


def test_complete_graph_one_round_id_order():
    # K_n: rho(S) = (n-1)/2, every degree n-1 <= 4 rho = 2(n-1): one densest
    # round; then n-1 < 12 rho: one round, all at degree n-1, so id order
    g = gg.complete(9)
    rank, rnd, dge, best = oracle.be_order(g)
    assert (rnd == 0).all() and (dge == 8).all()
    assert Fraction(*best) == Fraction(8, 2)
    assert rank.tolist() == list(range(9))


def test_path_by_hand():
    # path 0-1-2-3-4: |E| = 4, |S| = 5, threshold 4*4//5 = 3 removes all in
    # round 0 (rho~ = 4/5); then 12 rho~ = 9.6: all removed in round 0 at
    # their degrees 1,2,2,2,1 -> order 0, 4, 1, 2, 3
    g = gg.from_edges(5, [0, 1, 2, 3], [1, 2, 3, 4])
    rank, rnd, dge, best = oracle.be_order(g)
    assert best == (4, 5) and (rnd == 0).all()
    assert np.argsort(rank).tolist() == [0, 4, 1, 2, 3]


def _densest(g):
    a = gg.dense_adjacency(g).astype(bool)
    best = Fraction(0)
    for r in range(1, g.n + 1):
        for S in itertools.combinations(range(g.n), r):
            m = int(a[np.ix_(S, S)].sum()) // 2
            best = max(best, Fraction(m, r))
    return best


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_density_bound_and_out_degree(seed):
    g = gg.erdos_renyi(11, 0.45, seed)
    rank, rnd, dge, best = oracle.be_order(g)
    rho = Fraction(*best)
    rho_star = _densest(g)
    assert rho <= rho_star <= 4 * rho  # the approximate densest subgraph's guarantee
    od = oracle.orient(g, "be")
    outdeg = np.diff(od.ptr.astype(np.int64))
    assert (outdeg < 12 * rho).all() if rho > 0 else (outdeg == 0).all()


def test_rounds_logarithmic_and_counts_invariant():
    g = gg.rmat(12, 16, seed=3)
    _, rnd, _, _ = oracle.be_order(g)
    assert rnd.max() + 1 <= int(np.ceil(np.log(g.n) / np.log(1.5))) + 1
    for k in (3, 4, 5):
        assert oracle.count(oracle.orient(g, "be"), k) == oracle.count(oracle.orient(g, "degree"), k)
