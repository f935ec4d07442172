"""The 50M-vertex Chung-Lu workload with 1000 planted cliques (about 0.9e9
edges) at full size, through the C ABI in the configuration the benchmark
times. The oracle cannot count the whole graph in test time (the dense head
of the power law makes single roots take seconds), so parity is sampled: the
rooted counts (cliques whose lowest vertex is u) of seeded random roots and of
planted-clique members, from the per-arc pass, against the oracle one root at
a time, bit-exact; plus invariants at full size (degree and Goodrich-Pszona
orientations give the same totals; per-vertex counts sum to k times the
total)."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2002_10047_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

N = 50_000_000


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_10047_gb300 import build, kclique
    build.build()
    return kclique


@pytest.fixture(scope="module")
def workload(kc):
    eu, ev, sets = gg.chung_lu_planted_edges(n=N)
    rp, col = gg.csr_from_edges_on_device(N, eu, ev)
    del eu, ev
    host = gg.Csr(N, rp.cpu().numpy().view(np.uint64), col.cpu().numpy().view(np.uint32))
    return rp, col, host, sets


def rooted_from_arcs(dag, per_arc):
    """Rooted count of every vertex: the sum of its out-arcs' counts."""
    ptr, _ = dag.export()
    c = torch.zeros(per_arc.numel() + 1, dtype=torch.int64, device=per_arc.device)
    torch.cumsum(per_arc, 0, out=c[1:])  # int64 wrap-around is exact modulo 2^64
    return (c[ptr[1:]] - c[ptr[:-1]]).cpu().numpy().view(np.uint64)


def test_chunglu_full_size_sampled_parity(kc, workload):
    rp, col, host, sets = workload
    dag = kc.orient(rp, col, N, method="degree")
    assert dag.m == host.m
    total, per_arc = kc.count_per_arc(dag, 4)
    rooted = rooted_from_arcs(dag, per_arc)
    assert int(rooted.astype(object).sum()) == total
    od = oracle.orient(host, "degree")
    rng = np.random.default_rng(4)
    sample = set(rng.choice(N, 3000, replace=False).tolist())
    members = np.concatenate(sets)
    sample |= set(rng.choice(members, 200, replace=False).tolist())
    sample = sorted(sample)

    def one(u):
        return oracle.count(od, 4, lo=int(u), hi=int(u) + 1)

    with ThreadPoolExecutor(min(16, os.cpu_count() or 1)) as ex:
        want = np.array(list(ex.map(one, sample)), dtype=np.uint64)
    got = rooted[np.array(sample)]
    assert np.array_equal(got, want), [(u, int(a), int(b)) for u, a, b in zip(sample, got, want) if a != b][:5]
    assert want.sum() > 0


def test_chunglu_full_size_invariants(kc, workload):
    rp, col, _, _ = workload
    d_deg = kc.orient(rp, col, N, method="degree")
    d_gp = kc.orient(rp, col, N, method="gp")
    for k in (3, 4):
        assert kc.count(d_deg, k) == kc.count(d_gp, k)
    tot, pv = kc.count_per_vertex(d_deg, 4)
    s = int(kc.as_uint64(pv).astype(object).sum())
    assert s == 4 * tot
