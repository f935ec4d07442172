"""GPU parity of the batched pass: many disjoint graphs with their own k in one
oriented union, counted by one pass of the persistent kernels, against the
CPU oracle per graph (bit-exact) and against one library call per graph.

The mixed batch follows the batch recipe (Erdos-Renyi or Barabasi-Albert
50/50, n, average degree and k uniform); the small cases cap n so that the
oracle finishes in seconds, and the full 4096-graph batch is checked graph by
graph as well (about 3e9 cliques in total; the oracle runs on all host cores).
"""
import ctypes
import os
from concurrent.futures import ThreadPoolExecutor

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


def oracle_totals(graphs, ks, threads=None):
    th = threads or min(16, os.cpu_count() or 1)

    def one(gk):
        g, k = gk
        return oracle.count(oracle.orient(g, "degree"), int(k))

    with ThreadPoolExecutor(th) as ex:
        return np.array(list(ex.map(one, zip(graphs, ks))), dtype=np.uint64)


def device_batch(kc, graphs, ks, method="degree"):
    u, off = gg.concat_csr(graphs)
    rp, col = kc.csr_to_device(u)
    dag = kc.orient(rp, col, u.n, method=method)
    offs = torch.from_numpy(off.view(np.int64)).cuda()
    kt = torch.tensor(np.asarray(ks, dtype=np.uint8), dtype=torch.uint8, device="cuda")
    return dag, kc.Batch(offs, kt)


@pytest.fixture(scope="module")
def small_batch():
    specs = gg.batch_specs(96, seed=3, n_hi=1500)
    graphs = gg.build_batch(specs)
    # a few special members: empty, single vertex, a complete graph, a dense ER
    graphs += [gg.empty(0), gg.empty(1), gg.complete(40), gg.erdos_renyi(300, 0.3, 9), gg.empty(0)]
    ks = [s.k for s in specs] + [3, 4, 8, 5, 6]
    return graphs, ks, oracle_totals(graphs, ks)


def test_batch_small_mixed_bit_exact(kc, small_batch):
    graphs, ks, want = small_batch
    for method in ("degree", "gp"):
        dag, b = device_batch(kc, graphs, ks, method)
        tot, out = kc.count_batched(dag, b)
        got = kc.as_uint64(out)
        assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]
        assert tot == int(want.sum())


def test_batch_matches_one_call_per_graph(kc, small_batch):
    graphs, ks, _ = small_batch
    dag, b = device_batch(kc, graphs, ks)
    _, out = kc.count_batched(dag, b)
    got = kc.as_uint64(out)
    for i, (g, k) in enumerate(zip(graphs, ks)):
        if g.n == 0:
            assert got[i] == 0
            continue
        rp, col = kc.csr_to_device(g)
        assert kc.count(kc.orient(rp, col, g.n), k) == int(got[i]), i


@pytest.mark.parametrize("params", [
    (2, 1, 1, 2), (32, 64, 4, 1), (64, 128, 16, 2), (17, 100, 7, 1), (48, 0, 0, 0), (0, 64, 0, 2),
    (0, 0, 32, 1), (3, 128, 1, 2), (64, 64, 100, 2),
])
def test_batch_params_give_same_counts(kc, small_batch, params):
    graphs, ks, want = small_batch
    dag, b = device_batch(kc, graphs, ks)
    _, out = kc.count_batched(dag, b, params=params)
    assert np.array_equal(kc.as_uint64(out), want)


def test_batch_params_single_graph_all_root_classes(kc):
    """The tunables on one graph whose roots span warp, shared-memory block and
    global-scratch block roots, against the oracle, k = 3..7."""
    g = gg.rmat(13, 24, seed=21)
    od = oracle.orient(g, "degree")
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    offs = torch.tensor([0, g.n], dtype=torch.int64, device="cuda")
    for k in range(3, 8):
        want = oracle.count(od, k, threads=8)
        b = kc.Batch(offs, torch.tensor([k], dtype=torch.uint8, device="cuda"))
        for params in ((2, 1, 1, 1), (32, 64, 16, 2), (64, 128, 4, 1), (64, 128, 1, 2), (0, 0, 0, 0)):
            tot, out = kc.count_batched(dag, b, params=params)
            assert tot == want and int(kc.as_uint64(out)[0]) == want, (k, params)


def test_batch_plan_graph_capture_replay(kc, small_batch):
    graphs, ks, want = small_batch
    dag, b = device_batch(kc, graphs, ks)
    plan = kc.Plan(dag, b, params=(32, 128, 4, 2))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # one eager launch before capture
        plan.launch()
    torch.cuda.current_stream().wait_stream(side)
    assert plan.result() == int(want.sum())
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        plan.launch()
    for _ in range(3):
        plan.out.fill_(12345)
        cg.replay()
        assert plan.result() == int(want.sum())
        assert np.array_equal(kc.as_uint64(plan.out), want)
    plan.free()


def test_batch_autotune(kc, small_batch):
    graphs, ks, want = small_batch
    dag, b = device_batch(kc, graphs, ks)
    params, ms = kc.autotune_batched(dag, b)
    assert params["light_max"] in (32, 48, 64) and params["compact_max"] in (64, 128)
    assert params["chunk"] in (1, 4, 16) and params["light_order"] in (1, 2) and ms > 0
    _, out = kc.count_batched(dag, b, params=params)
    assert np.array_equal(kc.as_uint64(out), want)


def test_batch_rejects_bad_arguments(kc):
    g = gg.complete(12)
    dag, b = device_batch(kc, [g, g], [4, 5])
    with pytest.raises(ValueError):
        kc.Batch(b.offsets, b.ks[:1])
    # a per-graph k outside [3, KC_KMAX] that the host cannot see (k_min is the
    # caller's claim): the device reports it as KC_EINVAL
    bad = kc.Batch(b.offsets, torch.tensor([4, 40], dtype=torch.uint8, device="cuda"))
    with pytest.raises(kc.KcError) as e:
        kc.count_batched(dag, bad)
    assert e.value.status == kc.KC_EINVAL
    lib = kc._load()
    out = torch.empty(2, dtype=torch.int64, device="cuda")
    t = ctypes.c_uint64()
    for k_min in (2, 33):
        cb = kc._Batch(2, b.offsets.data_ptr(), b.ks.data_ptr(), k_min)
        rc = lib.kc_count_batched(dag.handle, ctypes.byref(cb), None, out.data_ptr(), ctypes.byref(t), 0)
        assert rc == kc.KC_EINVAL
    # a batch with all graphs below their k (no roots qualify): zeros
    dag2, b2 = device_batch(kc, [gg.complete(3), gg.complete(4)], [5, 6])
    tot, out2 = kc.count_batched(dag2, b2)
    assert tot == 0 and not kc.as_uint64(out2).any()


def test_batch_full_4096_bit_exact(kc):
    """The full mixed batch (4096 graphs, seed 3; 41.3M vertices, 0.70B edges):
    every graph's total against the oracle."""
    specs = gg.batch_specs(4096, seed=3)
    graphs = gg.build_batch(specs)
    ks = [s.k for s in specs]
    want = oracle_totals(graphs, ks)
    dag, b = device_batch(kc, graphs, ks)
    del graphs
    for params in (None, (0, 0, 16, kc.KC_LIGHT_BY_ID)):
        tot, out = kc.count_batched(dag, b, params=params)
        got = kc.as_uint64(out)
        assert np.array_equal(got, want), (params, np.nonzero(got != want)[0][:10])
        assert tot == int(want.sum())
