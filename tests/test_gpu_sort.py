"""GPU batch sort (cpma_sort_batch) against its plain definition: the keys in
non-decreasing order, each tag travelling with its key, equal keys in input
order (a stable sort: numpy's stable argsort).  The sizes and key shapes
cover the single-tile sorts (a sorting network for untagged batches, a
stable rank sort for tagged ones), the buckets by the 8 highest varying bits
(batches of up to 1.25M keys), buckets too large for one block's shared
memory (sorted through global memory by that block), the digit passes
(larger batches), 34-bit uniform and skewed keys, and keys that vary in one
digit only, in all eight, in fewer than 8 bits, or not at all."""
import numpy as np
import pytest
import torch

from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    g = cp.CPMA(torch.arange(1, 100, dtype=torch.int64, device="cuda"))
    yield g
    torch.cuda.synchronize()


def check(g, keys, tagged=True):
    keys = np.ascontiguousarray(keys, dtype=np.uint64)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    tags = np.arange(keys.size, dtype=np.uint32) * np.uint32(2654435761)
    dt = torch.from_numpy(tags.view(np.int32)).cuda() if tagged else None
    sk, st = cp.cpma_sort_batch(g.handle, dk, dt)
    order = np.argsort(keys, kind="stable")
    assert np.array_equal(sk.cpu().numpy().view(np.uint64), keys[order])
    if tagged:
        assert np.array_equal(st.cpu().numpy().view(np.uint32), tags[order])


@pytest.mark.parametrize("k", [4096, 4097, 100_000, 1_000_000, 1_310_720, 1_400_000])
def test_sort_uniform_40bit(handle, k):
    check(handle, W.uniform_keys(31 + k, k, bits=40))


def test_sort_keys_only(handle):
    check(handle, W.uniform_keys(7, 600_000, bits=40), tagged=False)


def test_sort_bucket_overflow(handle):
    # 40% of the keys share one value: its bucket far exceeds one block's
    # shared memory (an oversized bucket with nothing to sort inside)
    k = 1_000_000
    keys = W.uniform_keys(11, k, bits=40)
    keys[W.permuted_indices(k, 400_000, 12)] = np.uint64(0x12_3456_789A)
    check(handle, keys)
    # an oversized bucket whose keys differ: a narrow band of values takes
    # a quarter of the batch (sorted through global memory, several digits)
    band = W.uniform_keys(17, 250_000, bits=30) + np.uint64(0x55_0000_0000)
    keys[:250_000] = band
    check(handle, keys)


@pytest.mark.parametrize("k", [20_000, 100_000, 1_000_000])
def test_sort_34bit_uniform_and_zipf(handle, k):
    check(handle, W.uniform_keys(41 + k, k, bits=34))
    check(handle, W.zipf_keys(42 + k, k, bits=34))


def test_sort_few_varying_bits(handle):
    check(handle, W.uniform_keys(18, 50_000, bits=5) << np.uint64(20))   # fewer than 8 bits
    check(handle, np.arange(70_000, dtype=np.uint64)[::-1].copy())       # dense, reversed


def test_sort_one_varying_digit(handle):
    check(handle, W.uniform_keys(13, 100_000, bits=8))                       # lowest digit
    check(handle, W.uniform_keys(14, 200_000, bits=8) << np.uint64(56))      # highest digit


def test_sort_all_digits_and_equal_keys(handle):
    check(handle, W.full_range_keys(15, 300_000))
    check(handle, np.full(50_000, 0xABCDEF, dtype=np.uint64))
    check(handle, W.zipf_keys(16, 1_000_000))


@pytest.mark.parametrize("k", [1, 2, 3, 255, 1000, 2048, 2049, 4096])
def test_sort_small_keys_only(handle, k):
    # untagged batches of at most 4096 keys: the one-block sorting network,
    # padded to a power of two (repeats and the maximum key included)
    keys = W.uniform_keys(61 + k, k, bits=40)
    if k > 8:
        keys[: k // 8] = keys[k // 2]
        keys[-1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    check(handle, keys, tagged=False)
