"""GPU parity of the point path (Sec. 4: a batch much smaller than the set is
applied as point updates).  Inserts and deletes of up to 16384 keys whose
touched leaves all change in place, and batches that some leaf cannot take
(more than 32 keys -- 4 for a delete -- in one leaf, a leaf pushed over its
own bound or past 512 bytes, a leaf emptied) and that the batch algorithm
then finishes, give the same counts, set and byte layout as the sequential
oracle.  The point path is checked to have run, both ways, and turning it
off changes nothing."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu
M64 = (1 << 64) - 1


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    cp.lib()
    yield
    torch.cuda.synchronize()


def T(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.uint64))
    return torch.from_numpy(a.view(np.int64)).cuda()


def same_layout(g, o):
    assert g.leaves() == o.leaves()
    data, used, heads = g.layout()
    od, ou, oh = o.layout()
    assert np.array_equal(used.cpu().numpy().view(np.uint32), ou)
    assert np.array_equal(cp.to_u64(heads), oh)
    gd = data.cpu().numpy()
    if not np.array_equal(gd, od):
        bad = np.unique(np.nonzero(gd != od)[0] // g.leaf_bytes())[:10]
        raise AssertionError("leaf bytes differ in leaves %s" % bad)
    assert g.size() == o.size() and g.bytes() == o.bytes()


def batches(seed, p, heads, n_rounds):
    """Small insert batches of the kinds the point path distinguishes: fresh
    keys, neighbours of present keys (hits and split gaps), keys around leaf
    heads (new heads), keys past the last element, repeats, and runs of 20
    to 40 keys into one gap (over 32 keys: the batch algorithm's)."""
    rng = np.random.default_rng(seed)
    sizes = [1, 2, 7, 33, 100, 1000, 4096, 9000]
    for r in range(n_rounds):
        S = p.S
        k = sizes[r % len(sizes)]
        kind = r % 6
        pick = S[rng.integers(0, S.size, size=k)].astype(np.int64)
        if kind == 0:
            keys = W.uniform_keys(seed * 100 + r, k, bits=40).astype(np.int64)
        elif kind == 1:
            keys = pick + rng.integers(-2, 3, size=k)
        elif kind == 2:
            hd = heads().astype(np.int64)
            keys = hd[rng.integers(0, hd.size, size=k)] + rng.integers(-3, 2, size=k)
        elif kind == 3:
            keys = np.int64(S[-1]) + rng.integers(1, 1 << 20, size=k)
        elif kind == 4:
            keys = np.concatenate([pick, pick[: max(1, k // 3)]])
        else:
            span = int(rng.integers(20, 41))
            keys = np.concatenate([pick[:1] + 1 + np.arange(span), pick[1:]])
        yield r, np.clip(keys, 0, None).astype(np.uint64)


@pytest.mark.parametrize("LB", [256, 512])
def test_point_path_matches_oracle(LB):
    base = W.uniform_keys(601 + LB, 60000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB)
    o = oracle.SeqCPMA(base, leaf_bytes=LB)
    p = oracle.PlainSet(base)
    heads = lambda: cp.to_u64(g.layout()[2])
    n_ins = 0
    for r, keys in batches(LB, p, heads, 42):
        if r % 7 == 3:  # deletes keep the leaves uneven
            gone = W.sample_present(p.S, 700 + r, 300)
            assert int(g.delete_batch(T(gone)).item()) == o.delete_batch(gone) == p.delete_batch(gone)
            n_ins += 1
        elif r % 5 == 4:
            srt = np.sort(keys)
            assert int(g.insert_batch(T(srt), sorted=True).item()) == o.insert_batch(srt) == p.insert_batch(srt)
            n_ins += keys.size <= 16384
        else:
            assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
            n_ins += keys.size <= 16384
        same_layout(g, o)
    st = g.point_stats()
    assert st["calls"] == n_ins, st
    assert 0 < st["batch"] < st["calls"], st   # both outcomes taken


@pytest.mark.parametrize("LB", [256, 512])
def test_point_deletes_match_oracle(LB):
    """Small deletes (the point path takes up to 4096 keys): present and
    absent keys, leaf heads (a new head), the last element, repeats, whole
    runs of neighbours (a leaf emptied or pushed under its bound: the batch
    algorithm), with inserts between."""
    rng = np.random.default_rng(LB + 3)
    base = W.uniform_keys(651 + LB, 50000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB)
    o = oracle.SeqCPMA(base, leaf_bytes=LB)
    p = oracle.PlainSet(base)
    sizes = [1, 3, 30, 300, 1000, 4096]
    n_del = 0
    for r in range(36):
        S = p.S
        k = sizes[r % len(sizes)]
        kind = r % 5
        if kind == 0:
            keys = W.sample_present(S, 660 + r, k)
        elif kind == 1:
            keys = np.concatenate([W.sample_present(S, 660 + r, k // 2 + 1),
                                   W.uniform_keys(670 + r, k // 2 + 1, bits=40)])
        elif kind == 2:
            hd = cp.to_u64(g.layout()[2])
            keys = np.concatenate([hd[rng.integers(0, hd.size, size=k)], S[-1:]])
        elif kind == 3:
            keys = W.sample_present(S, 660 + r, k)
            keys = np.concatenate([keys, keys[: k // 2 + 1]])
        else:
            at = int(rng.integers(0, S.size - 200))
            keys = S[at: at + int(rng.integers(2, 120))]  # a run of neighbours
        keys = np.asarray(keys, dtype=np.uint64)
        if r % 4 == 3:
            srt = np.sort(keys)
            got = int(g.delete_batch(T(srt), sorted=True).item())
        else:
            got = int(g.delete_batch(T(keys)).item())
        assert got == o.delete_batch(keys) == p.delete_batch(keys)
        n_del += keys.size <= 4096
        same_layout(g, o)
        if r % 6 == 5:
            ins = W.uniform_keys(680 + r, 2000, bits=40)
            assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins) == p.insert_batch(ins)
            n_del += 1
            same_layout(g, o)
    st = g.point_stats()
    assert st["calls"] == n_del, st
    assert 0 < st["batch"] < st["calls"], st


def test_point_path_fills_a_leaf_past_its_bound():
    """Runs of 32 one-byte codes into the same leaf, batch after batch: the
    point path takes them until the leaf would pass its bound or 512 bytes,
    then the batch algorithm redistributes; the layout stays the oracle's."""
    base = W.uniform_keys(611, 30000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    x0 = int(np.sort(base)[15000])
    for r in range(24):
        keys = np.uint64(x0) + np.uint64(1000 * r + 1) + np.arange(32, dtype=np.uint64)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys)
        same_layout(g, o)
    st = g.point_stats()
    assert st["calls"] == 24 and st["batch"] >= 1, st


def test_point_path_off_changes_nothing():
    base = W.uniform_keys(621, 40000, bits=40)
    a = cp.CPMA(T(base), leaf_bytes=512)
    b = cp.CPMA(T(base), leaf_bytes=512)
    b.set_point_max(0)
    p = oracle.PlainSet(base)
    heads = lambda: cp.to_u64(a.layout()[2])
    calls = 0
    for r, keys in batches(5, p, heads, 14):
        na, nb = int(a.insert_batch(T(keys)).item()), int(b.insert_batch(T(keys)).item())
        assert na == nb == p.insert_batch(keys)
        gone = W.sample_present(p.S, 690 + r, keys.size)
        na, nb = int(a.delete_batch(T(gone)).item()), int(b.delete_batch(T(gone)).item())
        assert na == nb == p.delete_batch(gone)
        calls += (keys.size <= 16384) + (gone.size <= 4096)
        for x, y in zip(a.layout(), b.layout()):
            assert torch.equal(x, y)
    assert b.point_stats() == {"calls": 0, "batch": 0}
    assert a.point_stats()["calls"] == calls


def test_point_path_extreme_keys_and_limits():
    """Keys 0 and 2^64-1 (routed by the head array's last entry), batches of
    4096 keys (the largest ranked in the routing kernel), 4097 and 16384
    (sorted by the batch sort first; 16384 is the largest the point path
    takes) and 16385 (the batch algorithm's), and the point limit lowered
    below a batch's size."""
    base = np.concatenate([W.uniform_keys(631, 20000, bits=64), np.array([5, M64 - 5], np.uint64)])
    g = cp.CPMA(T(base), leaf_bytes=256)
    o = oracle.SeqCPMA(base, leaf_bytes=256)
    p = oracle.PlainSet(base)
    for keys in ([0], [M64], [M64, 0, M64 - 1, 1], W.uniform_keys(632, 4096, bits=64),
                 W.uniform_keys(633, 4097, bits=64), W.uniform_keys(635, 16384, bits=64),
                 W.uniform_keys(636, 16385, bits=64)):
        keys = np.asarray(keys, dtype=np.uint64)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    assert g.point_stats()["calls"] == 6
    g.set_point_max(10)
    keys = W.uniform_keys(634, 11, bits=64)
    assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys)
    same_layout(g, o)
    assert g.point_stats()["calls"] == 6


def test_point_path_rejects_an_unsorted_batch_unchanged():
    base = W.uniform_keys(641, 20000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    before = [t.cpu().clone() for t in g.layout()]
    for k in (2, 100, 4096, 9000):
        keys = np.sort(W.uniform_keys(642 + k, k, bits=40))[::-1].copy()  # descending
        with pytest.raises(cp.CPMAError) as e:
            g.insert_batch(T(keys), sorted=True)
        assert e.value.code == cp.CPMA_EINVAL
        assert all(torch.equal(a, b.cpu()) for a, b in zip(before, g.layout()))
    assert g.size() == len(oracle.PlainSet(base))


def test_point_path_with_profiling_and_graphs():
    """Profiling and graph mode on: small updates still take the point path,
    their phases are recorded (routing and the warp-per-leaf phase), and the
    layout stays the oracle's."""
    base = W.uniform_keys(661, 1 << 20, bits=40)  # about 0.4 keys per leaf at 4096
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    g.use_graphs(1 << 20)
    g.reserve(5000)
    g.profile(True)
    for r, k in enumerate([1, 40, 1000, 4096]):
        keys = W.uniform_keys(662 + r, k, bits=40)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys)
        gone = W.sample_present(np.unique(keys), 670 + r, max(1, k // 3))
        assert int(g.delete_batch(T(gone)).item()) == o.delete_batch(gone)
        same_layout(g, o)
    prof = g.profile_read()
    g.profile(False)
    assert g.point_stats() == {"calls": 8, "batch": 0}
    assert g.graph_stats()["launches"] == 0  # no batch went to the batch algorithm
    for ph in ("route", "merge_lane"):
        assert prof[ph]["calls"] == 8 and prof[ph]["ms"] > 0, (ph, prof[ph])
