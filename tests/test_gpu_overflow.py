"""The overflow path of the count reductions: the counting kernels' checked
64-bit reduction (thread sums and the block epilogue the counting kernels end
with), driven through kc_checked_sum with sums that fit exactly and sums one
past 2^64 - 1 (in a thread, inside a warp, between the warps of one block,
and across blocks), which must raise instead of wrapping."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def kc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2002_10047_gb300 import build, kclique
    build.build()
    return kclique


def dev(vals):
    return torch.from_numpy(np.asarray(vals, dtype=np.uint64).view(np.int64)).cuda()


def test_sums_that_fit_are_exact(kc):
    rng = np.random.default_rng(1)
    v = rng.integers(0, 1 << 40, size=1 << 20, dtype=np.uint64)
    assert kc.kc_checked_sum(dev(v)) == int(v.astype(object).sum())
    assert kc.kc_checked_sum(dev([])) == 0
    top = (1 << 64) - 1
    assert kc.kc_checked_sum(dev([top])) == top
    assert kc.kc_checked_sum(dev([top - 5, 2, 3])) == top
    # 2^21 - 1 values of 2^43: 2^64 - 2^43, spread over many warps and blocks
    assert kc.kc_checked_sum(dev(np.full((1 << 21) - 1, 1 << 43, dtype=np.uint64))) == (1 << 64) - (1 << 43)


@pytest.mark.parametrize("vals", [
    [1 << 63, 1 << 63],                                  # two lanes of one warp
    [(1 << 64) - 1, 1],
    [(1 << 62)] * 4,                                     # exactly 2^64
    [1 << 63] + [0] * 31 + [1 << 63],                    # lane 0 of warps 0 and 1 of block 0
])
def test_small_overflows_raise(kc, vals):
    with pytest.raises(kc.KcOverflow):
        kc.kc_checked_sum(dev(vals))


def test_overflow_across_warps_and_blocks_raises(kc):
    # 2^21 values of 2^43 sum to exactly 2^64: no single thread, warp or block
    # wraps, the wrap happens in the per-block atomic accumulation
    with pytest.raises(kc.KcOverflow):
        kc.kc_checked_sum(dev(np.full(1 << 21, 1 << 43, dtype=np.uint64)))
