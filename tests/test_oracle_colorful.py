"""Pins of the oracle's colorful sparsification (Section 3.3; the estimator
theorem of Appendix B), on the CPU."""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg


def test_splitmix64_first_output():
    # splitmix64 seeded with 0: the first output is 0xe220a8397b1dcdaf
    assert oracle.splitmix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    cols = oracle.vertex_colors(5, 1 << 32, 0)
    assert int(cols[0]) == 0xE220A8397B1DCDAF >> 32


@pytest.mark.parametrize("k", [3, 4, 5])
def test_one_color_is_exact(k):
    g = gg.erdos_renyi(200, 0.12, 4)
    c, est = oracle.colorful_count(g, k, 1, 123)
    assert c == est == oracle.count(oracle.orient(g), k)


def test_colors_uniform_and_deterministic():
    cols = oracle.vertex_colors(20000, 7, 99)
    assert np.array_equal(cols, oracle.vertex_colors(20000, 7, 99))
    counts = np.bincount(cols, minlength=7)
    assert counts.min() > 20000 / 7 * 0.9 and counts.max() < 20000 / 7 * 1.1


def _cliques(g, k):
    a = gg.dense_adjacency(g).astype(bool)
    return [c for c in itertools.combinations(range(g.n), k)
            if all(a[x, y] for x, y in itertools.combinations(c, 2))]


def _theorem_variance(g, k, colors):
    """Var[Y] of the appendix theorem with p = 1/colors; s_z counts the ordered
    pairs of distinct k-cliques sharing z vertices (the sum over i != j of
    Cov(C_i, C_j) in Var[sum C_i])."""
    cl = [frozenset(c) for c in _cliques(g, k)]
    X = len(cl)
    s = [0] * (k + 1)
    for i in range(X):
        for j in range(X):
            if i != j:
                s[len(cl[i] & cl[j])] += 1
    p = 1.0 / colors
    q = p ** (k - 1)
    var = X * (q - q * q) + sum(s[z] * (p ** (2 * (k - 1) - z + 1) - q * q) for z in range(2, k))
    return X, var / (q * q)


@pytest.mark.parametrize("k,colors", [(3, 2), (4, 2), (3, 3)])
def test_unbiased_with_theorem_variance(k, colors):
    g = gg.erdos_renyi(26, 0.5, 6)
    X, var = _theorem_variance(g, k, colors)
    S = 400
    ys = np.array([oracle.colorful_count(g, k, colors, seed)[1] for seed in range(S)], dtype=np.float64)
    assert X == oracle.count(oracle.orient(g), k)
    # the mean is within four standard errors of the exact count
    assert abs(ys.mean() - X) <= 4.0 * math.sqrt(var / S)
    # and the sample variance agrees with the theorem's (its relative
    # sampling error at S = 400 is ~0.1 here)
    ratio = ys.var(ddof=1) / var
    assert 0.7 < ratio < 1.4, ratio
