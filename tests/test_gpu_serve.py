"""The serving loop (kc_server): requests of different sizes and k on a pool of
device-resident graphs, admitted by memory footprint and run concurrently.
Every result must be identical to the same request run alone (and, per
distinct graph and k, to the CPU oracle); counts are integers, so the
tolerance is zero."""
import threading

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


POOL = [
    lambda: gg.rmat(10, 16, seed=51),
    lambda: gg.rmat(11, 8, seed=52),
    lambda: gg.rmat(12, 12, seed=53),
    lambda: gg.erdos_renyi(2000, 0.01, 54),
    lambda: gg.erdos_renyi(30000, 0.0008, 55),
    lambda: gg.barabasi_albert(3000, 8, 56),
    lambda: gg.complete(40),
    lambda: gg.turan([9, 12, 15, 7, 11, 10, 8]),
    lambda: gg.empty(5),
]


@pytest.fixture(scope="module")
def pool(kc):
    graphs = [f() for f in POOL]
    dags = []
    for g in graphs:
        rp, col = kc.csr_to_device(g)
        dags.append(kc.orient(rp, col, g.n))
    return graphs, dags


def requests(count, seed=5):
    key = seed
    gi = gg.uniform_ints(key, 1, count, 0, len(POOL) - 1)
    ks = gg.uniform_ints(key, 2, count, 3, 9)
    pv = gg.uniform_ints(key, 3, count, 0, 1)
    return [(int(a), int(b), bool(c)) for a, b, c in zip(gi, ks, pv)]


@pytest.fixture(scope="module")
def alone(kc, pool):
    """Each distinct (graph, k) run alone through the one-shot entry points, and
    checked against the oracle."""
    graphs, dags = pool
    res = {}
    for gi, k, _ in requests(160):
        if (gi, k) in res:
            continue
        tot, pv = kc.count_per_vertex(dags[gi], k)
        pvh = kc.as_uint64(pv).copy()
        assert kc.count(dags[gi], k) == tot
        want, want_pv = oracle.count_per_vertex(oracle.orient(graphs[gi], "degree"), k, threads=8)
        assert tot == want and np.array_equal(pvh, want_pv), (gi, k)
        res[(gi, k)] = (tot, pvh)
    return res


def run_mix(kc, dags, reqs, server, threads=2):
    ids = [None] * len(reqs)

    def submitter(part):
        for i in part:
            gi, k, pv = reqs[i]
            ids[i] = server.submit(dags[gi], k, per_vertex=pv)

    parts = [range(t, len(reqs), threads) for t in range(threads)]
    ths = [threading.Thread(target=submitter, args=(p,)) for p in parts]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    out = []
    for i, (gi, k, pv) in enumerate(reqs):
        r = server.wait(ids[i])
        vec = None
        if pv:
            buf = torch.empty(dags[gi].n, dtype=torch.int64)
            vec = server.fetch_per_vertex(ids[i], buf).numpy().view(np.uint64).copy()
            server.release(ids[i])
        else:
            server.forget(ids[i])
        out.append((r, vec))
    return out


def test_serve_mix_equals_alone(kc, pool, alone):
    graphs, dags = pool
    reqs = requests(160)
    srv = kc.Server(slots=8, hbm_budget=256 << 20, grid_share_pct=25)
    try:
        out = run_mix(kc, dags, reqs, srv)
        st = srv.stats()
    finally:
        srv.close()
    for (gi, k, pv), (r, vec) in zip(reqs, out):
        assert r["status"] == kc.KC_OK
        want, want_pv = alone[(gi, k)]
        assert r["total"] == want, (gi, k)
        if pv:
            assert np.array_equal(vec, want_pv), (gi, k)
        assert r["latency_s"] >= r["run_s"] >= 0
    assert st["submitted"] == st["completed"] == len(reqs)
    assert st["peak_in_flight"] >= 2  # requests overlapped on the GPU
    assert st["bytes_in_use"] == 0 and st["queued"] == 0


def test_serve_budget_serialises(kc, pool, alone):
    """A budget smaller than any footprint admits one request at a time."""
    graphs, dags = pool
    reqs = requests(40, seed=6)
    srv = kc.Server(slots=8, hbm_budget=1)
    try:
        out = run_mix(kc, dags, reqs, srv, threads=1)
        st = srv.stats()
    finally:
        srv.close()
    for (gi, k, pv), (r, vec) in zip(reqs, out):
        want, want_pv = alone.get((gi, k)) or (kc.count(dags[gi], k), None)
        assert r["total"] == want
        if pv and want_pv is not None:
            assert np.array_equal(vec, want_pv)
    assert st["peak_in_flight"] == 1
    assert st["completed"] == len(reqs)


def test_serve_grid_cap_and_device_fetch(kc, pool, alone):
    graphs, dags = pool
    srv = kc.Server(slots=3, hbm_budget=64 << 20, grid_share_pct=1)
    try:
        ids = [srv.submit(dags[gi], k, per_vertex=True) for gi, k in ((2, 5), (0, 4), (6, 9), (8, 3))]
        for rid, (gi, k) in zip(ids, ((2, 5), (0, 4), (6, 9), (8, 3))):
            r = srv.wait(rid, timeout_ms=60000)
            assert r["status"] == kc.KC_OK
            d = torch.empty(max(dags[gi].n, 1), dtype=torch.int64, device="cuda")[:dags[gi].n]
            srv.fetch_per_vertex(rid, d)
            srv.release(rid)
            if (gi, k) in alone:
                assert r["total"] == alone[(gi, k)][0]
                assert np.array_equal(kc.as_uint64(d), alone[(gi, k)][1])
            else:
                assert r["total"] == kc.count(dags[gi], k)
        with pytest.raises(kc.KcError):
            srv.wait(123456789)
        with pytest.raises(kc.KcError):
            srv.wait(ids[0])  # released
        with pytest.raises(kc.KcError):
            srv.submit(dags[0], 2)
    finally:
        srv.close()


def test_serve_request_time_budget(kc, pool):
    """A request whose time budget runs out completes with KC_ETIMEDOUT (the
    counting kernels stop taking roots); every root is short, so the pass is
    bounded either way. The same request without a budget completes."""
    g = gg.erdos_renyi(1 << 20, 40.0 / (1 << 20), 57)
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    want = kc.count(dag, 4)
    srv = kc.Server(slots=2, hbm_budget=1 << 30)
    try:
        rid = srv.submit(dag, 4, timeout_us=1)
        r = srv.wait(rid, timeout_ms=60000)
        assert r["status"] == kc.KC_ETIMEDOUT
        rid = srv.submit(dag, 4)
        r = srv.wait(rid, timeout_ms=60000)
        assert r["status"] == kc.KC_OK and r["total"] == want
    finally:
        srv.close()
