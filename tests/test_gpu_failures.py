"""Failure handling on the GPU without faulting it: time budgets that run out
(the kernels give up and report KC_ETIMEDOUT; the context stays usable) and
device allocations that fail, injected on the host (kc_debug_fail_allocations_after):
every entry point reports KC_ENOMEM, releases what it had allocated, and the
next call succeeds."""
import ctypes

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


def pool_used():
    """Bytes in use in the current device's default memory pool, where the
    library's stream-ordered allocations live (driver API via ctypes)."""
    cu = ctypes.CDLL("libcuda.so.1")
    dev = ctypes.c_int()
    assert cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
    pool = ctypes.c_void_p()
    assert cu.cuDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    v = ctypes.c_uint64()
    torch.cuda.synchronize()
    assert cu.cuMemPoolGetAttribute(pool, 7, ctypes.byref(v)) == 0  # CU_MEMPOOL_ATTR_USED_MEM_CURRENT
    return v.value


def test_budget_runs_out_then_completes(kc):
    g = gg.rmat(14, 16, seed=5)
    rp, col = kc.csr_to_device(g)
    dag = kc.orient(rp, col, g.n)
    want = oracle.count_per_vertex(oracle.orient(g, "degree"), 6)
    for per_vertex in (False, True):
        out = torch.empty(g.n, dtype=torch.int64, device="cuda") if per_vertex else None
        with pytest.raises(kc.KcTimeout):
            kc.count_budget(dag, 6, 1, out=out)  # 1 microsecond: past it before the first roots finish
        got = kc.count_budget(dag, 6, 60_000_000, out=out)  # a minute: completes
        assert got == want[0]
        if per_vertex:
            np.testing.assert_array_equal(kc.as_uint64(out), want[1])
    assert kc.count(dag, 6) == want[0]  # the context is still usable
    with pytest.raises(kc.KcError):
        kc.count_budget(dag, 6, 0)  # a zero budget is rejected


def test_injected_allocation_failures(kc):
    g = gg.rmat(12, 16, seed=3)
    rp, col = kc.csr_to_device(g)
    od = oracle.orient(g, "degree")
    want4, want4_pv = oracle.count_per_vertex(od, 4)
    dag = kc.orient(rp, col, g.n)
    base = pool_used()
    calls = {
        "orient": lambda: kc.orient(rp, col, g.n).free(),
        "orient_gp": lambda: kc.orient(rp, col, g.n, method="gp").free(),
        "orient_core": lambda: kc.orient(rp, col, g.n, core=True).free(),
        "count": lambda: kc.count(dag, 4),
        "count_per_vertex": lambda: kc.count_per_vertex(dag, 4),
        "count_roots": lambda: kc.count_roots(dag, 4, torch.arange(100, dtype=torch.int32, device="cuda")),
        "count_budget": lambda: kc.count_budget(dag, 4, 10_000_000),
    }
    for name, call in calls.items():
        failed = 0
        for after in range(0, 16):
            kc.kc_debug_fail_allocations_after(after)
            try:
                call()
            except kc.KcError as e:
                assert e.status == kc.KC_ENOMEM, (name, after, e.status)
                failed += 1
            finally:
                kc.kc_debug_fail_allocations_after(-1)
            assert pool_used() == base, (name, after)  # nothing left allocated
        assert failed >= 1, name
    # clean calls afterwards
    assert kc.count(dag, 4) == want4
    tot, pv = kc.count_per_vertex(dag, 4)
    assert tot == want4
    np.testing.assert_array_equal(kc.as_uint64(pv), want4_pv)


def test_automatic_core_is_optional_under_allocation_failure(kc):
    """The dense core that kc_orient builds by default (here: R-MAT 14, largest
    out-degree 144) is optional: when one of its allocations fails the handle
    comes back without a core and counts the same; failures before it still
    give KC_ENOMEM, and nothing stays allocated either way."""
    g = gg.rmat(14, 16, seed=5)
    rp, col = kc.csr_to_device(g)
    want = oracle.count(oracle.orient(g, "degree"), 4, threads=8)
    full = kc.orient(rp, col, g.n)
    assert full.core_vertices > 0
    full.free()
    base = pool_used()
    coreless = 0
    for after in range(0, 24):
        kc.kc_debug_fail_allocations_after(after)
        try:
            dag = kc.orient(rp, col, g.n)
        except kc.KcError as e:
            assert e.status == kc.KC_ENOMEM, (after, e.status)
            dag = None
        finally:
            kc.kc_debug_fail_allocations_after(-1)
        if dag is not None:
            coreless += dag.core_vertices == 0
            assert kc.count(dag, 4) == want, after
            dag.free()
        assert pool_used() == base, after
    assert coreless >= 1
