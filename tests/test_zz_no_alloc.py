"""kc_count_noalloc: the count taken without any device allocation.

Some callers cannot call cudaMalloc where they count (code under a fixed memory
budget or behind a custom allocator that owns the device memory, paths that
must not take allocator locks). This entry point uses one static device array
as its scratch. The test calls it through the C ABI and checks it against
kc_count, twice in a row (the array keeps the previous call's contents), on a
graph whose roots all fit shared memory and on one whose largest roots use the
array's per-block matrices; checks that the device's default memory pool, from
which kc_count allocates, sees no allocation during the calls (while a
kc_count call does raise its high-water mark); and checks that a graph too
large for the array is refused.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_2002_10047_gb300 import graphgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_10047_gb300 import build, kclique
    build.build()
    lib = kclique._load()
    lib.kc_count_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), ctypes.c_void_p]
    lib.kc_count_noalloc.restype = ctypes.c_int
    return kclique


def noalloc(kc, dag, k):
    t = ctypes.c_uint64()
    rc = kc._load().kc_count_noalloc(dag.handle, k, ctypes.byref(t), int(torch.cuda.current_stream().cuda_stream))
    return rc, int(t.value)


class DefaultPool:
    """The current device's default stream-ordered memory pool (driver API via
    ctypes): kc_count's work block and slabs come from it."""
    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8  # CUmemPool_attribute

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        assert self.cu.cuInit(0) == 0
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return v.value

    def reset_high(self):
        zero = ctypes.c_uint64(0)  # resets the high-water mark to the current use
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def orient(kc, g):
    rp, col = kc.csr_to_device(g)
    return kc.orient(rp, col, g.n)


def test_noalloc_matches_kc_count_twice(kc):
    for g, ks in ((gg.rmat(13, 16, seed=3), (1, 2, 3, 4, 5, 6)), (gg.complete(2100), (3, 4))):
        dag = orient(kc, g)
        for k in ks:
            want = kc.count(dag, k)
            for _ in range(2):
                rc, got = noalloc(kc, dag, k)
                assert rc == kc.KC_OK
                assert got == want
        if g.n == 2100:
            assert want == math.comb(2100, 4)


def test_noalloc_draws_nothing_from_the_memory_pool(kc):
    pool = DefaultPool()
    for g, k in ((gg.rmat(13, 16, seed=3), 5), (gg.complete(2100), 3)):  # the second uses the slabs
        dag = orient(kc, g)
        want = kc.count(dag, k)
        torch.cuda.synchronize()
        pool.reset_high()
        base = pool.get(pool.USED_MEM_CURRENT)
        for _ in range(3):
            rc, got = noalloc(kc, dag, k)
            assert rc == kc.KC_OK and got == want
        torch.cuda.synchronize()
        assert pool.get(pool.USED_MEM_HIGH) == base
        assert pool.get(pool.USED_MEM_CURRENT) == base
        assert kc.count(dag, k) == want  # control: kc_count allocates from this pool
        torch.cuda.synchronize()
        assert pool.get(pool.USED_MEM_HIGH) > base


def test_noalloc_refuses_oversized_roots(kc):
    g = gg.complete(8300)  # largest out-degree 8299: one root matrix exceeds the static array
    dag = orient(kc, g)
    rc, _ = noalloc(kc, dag, 3)
    assert rc == kc.KC_ECAPACITY
