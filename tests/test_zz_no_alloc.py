"""kc_count_noalloc: the count taken without any device allocation.

Some callers cannot call cudaMalloc where they count (code captured into a CUDA
graph, code under a fixed memory budget or a custom allocator, paths that must
not take allocator locks). This entry point uses one static device array as its
scratch. The test calls it through the C ABI and checks it against kc_count,
twice in a row (the array keeps the previous call's contents), on a graph whose
roots all fit shared memory and on one whose largest roots use the array's
per-block matrices, and checks that a graph too large for the array is refused.
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


def test_noalloc_refuses_oversized_roots(kc):
    g = gg.complete(8300)  # largest out-degree 8299: one root matrix exceeds the static array
    dag = orient(kc, g)
    rc, _ = noalloc(kc, dag, 3)
    assert rc == kc.KC_ECAPACITY
