"""GPU parity of colorful sparsification (Section 3.3) through the C ABI: the
exact count of the monochromatic subgraph equals the oracle's for the same
colors (both sides draw them from splitmix64 by its definition), and the
estimate is that count times colors^(k-1)."""
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


GRAPHS = {
    "er": lambda: gg.erdos_renyi(3000, 0.01, 2),
    "rmat12": lambda: gg.rmat(12, 16, seed=9),
    "ba": lambda: gg.barabasi_albert(4000, 12, 3),
    "k60": lambda: gg.complete(60),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_colorful_matches_oracle(kc, name):
    g = GRAPHS[name]()
    rp, col = kc.csr_to_device(g)
    for k in (3, 4, 5):
        for colors, seed in ((1, 0), (2, 1), (3, 77), (8, (1 << 63) + 5)):
            want, want_est = oracle.colorful_count(g, k, colors, seed)
            for method in ("degree", "gp"):
                c, est = kc.count_colorful(rp, col, k, colors, seed, method=method)
                assert c == want, (name, k, colors, seed, method)
                assert est == float(want) * float(colors) ** (k - 1)


def test_colorful_one_color_is_exact_count(kc):
    g = gg.rmat(14, 16, seed=5)
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    for k in (3, 4, 6):
        assert kc.count_colorful(rp, col, k, 1, 42)[0] == kc.count(dag, k)


def test_colorful_rejects_bad_arguments(kc):
    g = gg.complete(10)
    rp, col = kc.csr_to_device(g)
    with pytest.raises(kc.KcError):
        kc.count_colorful(rp, col, 3, 0, 1)
    with pytest.raises(kc.KcError):
        kc.count_colorful(rp, col, 33, 2, 1)
