"""Host-side logic without a GPU: the batch recipe and the CSR concatenation
that builds a batch's union graph."""
import numpy as np

import oracle
from paper_2002_10047_gb300 import graphgen as gg


def test_concat_csr_equals_disjoint_union():
    specs = gg.batch_specs(40, seed=3, n_hi=600)
    graphs = gg.build_batch(specs) + [gg.empty(0), gg.complete(7), gg.empty(2)]
    u, off = gg.concat_csr(graphs)
    ref = gg.disjoint_union(graphs)
    assert u.n == ref.n == int(off[-1])
    assert u.row_ptr.dtype == np.uint64 and u.col.dtype == np.uint32
    assert np.array_equal(u.row_ptr, ref.row_ptr) and np.array_equal(u.col, ref.col)
    assert np.array_equal(np.diff(off.astype(np.int64)), [g.n for g in graphs])


def test_union_counts_are_per_graph_sums():
    """Counting the union graph g by g (roots restricted to each vertex range)
    gives each graph's own count: the property the batched pass relies on."""
    specs = gg.batch_specs(12, seed=5, n_hi=400)
    graphs = gg.build_batch(specs)
    u, off = gg.concat_csr(graphs)
    for k in (3, 4, 5):
        dag = oracle.orient(u, "degree")
        total = 0
        for i, g in enumerate(graphs):
            want = oracle.count(oracle.orient(g, "degree"), k)
            # the union's roots in graph i's id range (its out-lists stay inside it)
            assert oracle.count(dag, k, lo=int(off[i]), hi=int(off[i + 1])) == want
            total += want
        assert oracle.count(dag, k) == total


def test_batch_recipe_ranges():
    specs = gg.batch_specs(4096, seed=3)
    kinds = [s.kind for s in specs]
    assert 1900 < kinds.count("er") < 2200
    assert min(s.n for s in specs) >= 50 and max(s.n for s in specs) <= 20000
    assert min(s.avg_deg for s in specs) >= 4 and max(s.avg_deg for s in specs) <= 64
    assert {s.k for s in specs} == set(range(3, 9))
    assert gg.batch_specs(8, seed=3) == specs[:8]  # counter-based: a prefix is stable


def test_device_csr_builder_equals_host_csr():
    """The torch-sort CSR builder (input preparation for the 50M-vertex
    workload) gives the same CSR as the host builder; run on the CPU here."""
    import pytest
    torch = pytest.importorskip("torch")
    eu, ev, _ = gg.chung_lu_planted_edges(n=200000, cliques=20)
    g = gg.from_edges(200000, eu, ev)
    rp, col = gg.csr_from_edges_on_device(200000, eu, ev, device="cpu")
    assert np.array_equal(rp.numpy().view(np.uint64), g.row_ptr)
    assert np.array_equal(col.numpy().view(np.uint32), g.col)
    del torch


def test_bench_build_bytes_model():
    """The bench's algorithmic bytes of a counting pass: without a dense core
    the builds scan sum over arcs u->x of d+(x) entries (4 bytes each); with
    one, the scanned entries plus one 64-bit word per core lookup plus the
    members' core numbers (4 bytes per arc)."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_model", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    n, m, head = 1000, 9000, 250000
    plain = {"build_scanned": head, "build_lookups": 0, "core_vertices": 0}
    assert bench.build_bytes(n, m, plain) == 8 * (n + 1) + 4 * n + 4 * m + 8 * m + 4 * head
    core = {"build_scanned": 40000, "build_lookups": 3000, "core_vertices": 128}
    assert bench.build_bytes(n, m, core) == 8 * (n + 1) + 4 * n + 4 * m + 8 * m + 4 * 40000 + 8 * 3000 + 4 * m
