"""The update calls' memory contract and bounded wait, through the C ABI.

An update reserves every byte it can need before it changes anything, so a
failed allocation -- from the caller's allocator or the memory budget --
leaves the set exactly as it was, and so does a sort that gives up waiting
(CPMA_ETIMEOUT).  Failures are made on the host: an allocator that refuses
its N-th request, a budget just above what the handle holds, a sort or
routing tile told (through the test hook) never to publish its counts, with
a short poll limit.  Nothing here faults or hangs the GPU: the wait is bounded and the
kernels check the error flag before they change a leaf."""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.uint64)).view(np.int64)).cuda()


def snapshot(g):
    data, used, heads = g.layout()
    torch.cuda.synchronize()
    return (g.leaves(), g.leaf_bytes(), g.size(), g.bytes(), data.cpu().numpy().tobytes(),
            used.cpu().numpy().tobytes(), heads.cpu().numpy().tobytes())


def same_as_oracle(g, o):
    data, used, heads = g.layout()
    od, ou, oh = o.layout()
    assert g.leaves() == o.leaves() and g.leaf_bytes() == o.leaf_bytes()
    assert np.array_equal(data.cpu().numpy(), od)
    assert np.array_equal(used.cpu().numpy().view(np.uint32), ou)
    assert np.array_equal(cp.to_u64(heads), oh)
    assert g.size() == o.size() and g.bytes() == o.bytes()


def raw_update(g, keys, delete=False):
    k = T(keys)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    fn = cp.lib().cpma_delete_batch if delete else cp.lib().cpma_insert_batch
    rc = fn(g.handle, C.c_void_p(k.data_ptr()), k.numel(), 0, C.c_void_p(out.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, int(out.item())


class CountingAllocator:
    """Device memory from torch's caching allocator; from request fail_at on
    (until fail_at is cleared) it refuses every request, as a device that has
    run out of memory would."""

    def __init__(self):
        self.calls = 0
        self.fail_at = None
        self.held = {}
        self.alloc_fn = cp.ALLOC_FN(self._alloc)
        self.free_fn = cp.FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        self.calls += 1
        if self.fail_at is not None and self.calls >= self.fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes))
        self.held[p] = int(nbytes)
        return p

    def _free(self, p, stream, ctx):
        self.held.pop(p)
        torch.cuda.caching_allocator_delete(p)


@pytest.mark.parametrize("delete", [False, True])
def test_allocator_failing_at_every_request_leaves_the_set_unchanged(delete):
    base = W.uniform_keys(501, 20000, bits=40)
    if delete:
        keys = W.sample_present(np.unique(base), 502, 15000)   # shrinks the array
    else:
        keys = W.uniform_keys(503, 40000, bits=40)             # grows it
    o_after = oracle.SeqCPMA(base, leaf_bytes=256)
    (o_after.delete_batch if delete else o_after.insert_batch)(keys)
    failed = 0
    for N in range(1, 200):
        A = CountingAllocator()
        g = cp.CPMA(T(base), leaf_bytes=256, alloc=A.alloc_fn, free=A.free_fn)
        assert A.held and g.mem_held() == sum(A.held.values())
        before = snapshot(g)
        A.fail_at = A.calls + N
        rc, _ = raw_update(g, keys, delete)
        if rc == cp.CPMA_OK:
            same_as_oracle(g, o_after)
            break
        assert rc == cp.CPMA_ENOMEM, rc
        failed += 1
        assert snapshot(g) == before, "request %d refused: the set changed" % N
        A.fail_at = None                       # the handle still works
        rc, _ = raw_update(g, keys, delete)
        assert rc == cp.CPMA_OK
        same_as_oracle(g, o_after)
        del g
        assert not A.held                      # everything given back
    else:
        raise AssertionError("the update never succeeded")
    assert failed >= 3, failed


def test_budget_refuses_before_changing_anything():
    base = W.uniform_keys(511, 30000, bits=40)
    keys = W.uniform_keys(512, 60000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=256)
    o = oracle.SeqCPMA(base, leaf_bytes=256)
    held = g.mem_held()
    assert held >= g.bytes()
    g.set_mem_budget(held + 4096)
    before = snapshot(g)
    rc, _ = raw_update(g, keys)
    assert rc == cp.CPMA_ENOMEM
    assert snapshot(g) == before
    assert g.mem_held() <= held + 4096
    g.set_mem_budget(0)
    rc, added = raw_update(g, keys)
    assert rc == cp.CPMA_OK and added == o.insert_batch(keys)
    same_as_oracle(g, o)
    # at a cap of exactly what the handle holds, a batch whose reservation
    # is already held (a delete of fewer keys: no buffer has to grow, a
    # shrink is done in place) goes through
    held = g.mem_held()
    g.set_mem_budget(held)
    gone = W.sample_present(oracle.PlainSet(np.concatenate([base, keys])).S, 513, 1000)
    rc, removed = raw_update(g, gone, delete=True)
    assert rc == cp.CPMA_OK and removed == o.delete_batch(gone)
    same_as_oracle(g, o)
    assert g.mem_held() <= held


@pytest.mark.parametrize("silent", [0, 1, 3])
def test_sort_wait_gives_up_with_etimeout(silent):
    base = W.uniform_keys(521, 50000, bits=40)
    keys = W.uniform_keys(522, 20000, bits=40)   # five 4096-key sort tiles
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    before = snapshot(g)
    cp.cpma_test_sort_stall(g.handle, 2000, silent)
    rc, _ = raw_update(g, keys)
    assert rc == cp.CPMA_ETIMEOUT
    assert snapshot(g) == before
    rc, _ = raw_update(g, keys, delete=True)
    assert rc == cp.CPMA_ETIMEOUT
    assert snapshot(g) == before
    cp.cpma_test_sort_stall(g.handle, 0, -1)
    rc, added = raw_update(g, keys)
    assert rc == cp.CPMA_OK and added == o.insert_batch(keys)
    same_as_oracle(g, o)


def raw_sorted_update(g, keys, delete=False):
    k = T(np.sort(np.asarray(keys, np.uint64)))
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    fn = cp.lib().cpma_delete_batch if delete else cp.lib().cpma_insert_batch
    rc = fn(g.handle, C.c_void_p(k.data_ptr()), k.numel(), 1, C.c_void_p(out.data_ptr()),
            C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, int(out.item())


@pytest.mark.parametrize("silent", [0, 1, 5])
def test_route_wait_gives_up_with_etimeout(silent):
    # a batch given sorted skips the sort: the routing's look-back is the
    # wait that runs out (20000 keys: 79 tiles of 256 keys)
    base = W.uniform_keys(531, 50000, bits=40)
    keys = W.uniform_keys(532, 20000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    before = snapshot(g)
    cp.cpma_test_sort_stall(g.handle, 2000, silent)
    rc, _ = raw_sorted_update(g, keys)
    assert rc == cp.CPMA_ETIMEOUT
    assert snapshot(g) == before
    rc, _ = raw_sorted_update(g, keys, delete=True)
    assert rc == cp.CPMA_ETIMEOUT
    assert snapshot(g) == before
    cp.cpma_test_sort_stall(g.handle, 0, -1)
    rc, added = raw_sorted_update(g, keys)
    assert rc == cp.CPMA_OK and added == o.insert_batch(keys)
    same_as_oracle(g, o)
