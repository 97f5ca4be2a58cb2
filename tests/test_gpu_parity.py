"""GPU parity: every C-ABI call against the CPU oracle on the same seeded
inputs, bit for bit (all of this work is integer).  Set-level answers are
compared with the plain definition (PlainSet); the byte layout (leaf bytes,
used counts, head index, leaf count, get_size) with the sequential CPMA."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import workloads as W
from setops import sorted_unique, union

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
    assert g.leaf_bytes() == o.leaf_bytes()
    data, used, heads = g.layout()
    od, ou, oh = o.layout()
    gu = used.cpu().numpy().view(np.uint32)
    gh = cp.to_u64(heads)
    if not np.array_equal(gu, ou):
        bad = np.nonzero(gu != ou)[0][:10]
        raise AssertionError("used differs at leaves %s: gpu %s oracle %s" % (bad, gu[bad], ou[bad]))
    assert np.array_equal(gh, oh), np.nonzero(gh != oh)[0][:10]
    gd = data.cpu().numpy()
    if not np.array_equal(gd, od):
        LB = g.leaf_bytes()
        bad = np.unique(np.nonzero(gd != od)[0] // LB)[:10]
        raise AssertionError("leaf bytes differ in leaves %s" % bad)
    assert g.size() == o.size()
    assert g.bytes() == o.bytes()


def same_queries(g, p, seed, nq=400):
    S = p.S
    q = np.concatenate([W.uniform_keys(seed, nq, bits=40), S[:: max(1, S.size // nq)][:nq],
                        np.array([0, 1, M64, M64 - 1], np.uint64)])
    assert np.array_equal(g.has_batch(T(q)).cpu().numpy(), p.has_batch(q))
    lo, hi = W.range_queries_fixed_width(seed + 1, nq, 1 << 28)
    if S.size:
        lo2, hi2, _ = W.range_queries_by_rank(S, seed + 2, nq, 1, max(2, S.size // 3))
        lo, hi = np.concatenate([lo, lo2]), np.concatenate([hi, hi2])
    lo = np.concatenate([lo, np.array([0, 5, M64, 0, 7], np.uint64)])
    hi = np.concatenate([hi, np.array([M64, 5, M64, 1, 3], np.uint64)])
    s, c = g.range_map(T(lo), T(hi))
    ws, wc = p.range_map(lo, hi)
    assert np.array_equal(cp.to_u64(c), wc)
    assert np.array_equal(cp.to_u64(s), ws)
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == p.sum() and int(c.item()) == len(p)


@pytest.mark.parametrize("LB", [256, 512, 1024, 2048])
@pytest.mark.parametrize("n,bits", [(0, 40), (1, 40), (7, 64), (5000, 40), (70000, 40),
                                    (70000, 64), (4096, 40), (4097, 40)])
def test_build_layout(LB, n, bits):
    keys = W.uniform_keys(11 + n, n, bits=bits) if bits < 64 else W.full_range_keys(11 + n, n)
    keys = np.concatenate([keys, keys[: n // 5]])  # repeats
    g = cp.CPMA(T(keys) if keys.size else None, leaf_bytes=LB)
    o = oracle.SeqCPMA(keys, leaf_bytes=LB)
    same_layout(g, o)
    same_queries(g, oracle.PlainSet(keys), 5 + n)


@pytest.mark.parametrize("LB", [256, 512, 2048])
def test_update_sequence(LB):
    rng = np.random.default_rng(LB)
    base = W.uniform_keys(21, 30000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB)
    o = oracle.SeqCPMA(base, leaf_bytes=LB)
    p = oracle.PlainSet(base)
    for r in range(24):
        kind = r % 6
        if kind == 0:
            keys = W.uniform_keys(100 + r, int(rng.choice([1, 50, 3000, 20000])), bits=40)
            keys = np.concatenate([keys, keys[: keys.size // 3]])
        elif kind == 1:
            keys = W.zipf_keys(200 + r, 20000, bits=34)          # hot leaves, huge slices
        elif kind == 2:
            keys = np.sort(W.uniform_keys(300 + r, 5000, bits=40))  # pre-sorted
        elif kind == 3:
            keys = np.concatenate([W.sample_present(p.S, 400 + r, 4000),
                                   W.uniform_keys(500 + r, 1000, bits=40)])
        elif kind == 4:
            keys = W.sample_present(p.S, 600 + r, len(p) // 2)   # big delete: shrink
        else:
            keys = W.full_range_keys(700 + r, 3000)
        is_del = kind in (3, 4)
        srt = kind == 2
        if is_del:
            got = int(g.delete_batch(T(keys), sorted=srt).item())
            assert got == o.delete_batch(keys) == p.delete_batch(keys)
        else:
            got = int(g.insert_batch(T(keys), sorted=srt).item())
            assert got == o.insert_batch(keys) == p.insert_batch(keys)
        assert o.check() == 0
        same_layout(g, o)
        if r % 4 == 3:
            same_queries(g, p, 900 + r, 200)


@pytest.mark.parametrize("num,den", [(11, 10), (3, 2), (2, 1)])
def test_growing_factors_grow_and_shrink(num, den):
    # App. C: growing factors 1.1 ... 2 (R9 with g = num/den).  The set grows
    # from 2000 keys by batches that force several resizes, then big deletes
    # shrink it; layout parity after every batch, and both directions seen.
    cfg = dict(leaf_bytes=256, grow_num=num, grow_den=den)
    base = W.uniform_keys(31, 2000, bits=40)
    g = cp.CPMA(T(base), **cfg)
    o = oracle.SeqCPMA(base, **cfg)
    p = oracle.PlainSet(base)
    same_layout(g, o)
    Ls = [g.leaves()]
    for r in range(8):
        keys = W.uniform_keys(800 + r, 1500 * (r + 1), bits=40)
        if r % 3 == 2:
            keys = np.concatenate([keys, W.zipf_keys(850 + r, 3000, bits=34)])
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
        Ls.append(g.leaves())
    same_queries(g, p, 860)
    for r in range(6):
        keys = W.sample_present(p.S, 870 + r, (len(p) * 3) // 5)
        assert int(g.delete_batch(T(keys)).item()) == o.delete_batch(keys) == p.delete_batch(keys)
        assert o.check() == 0
        same_layout(g, o)
        Ls.append(g.leaves())
    same_queries(g, p, 880)
    assert max(Ls) > Ls[0] and Ls[-1] < max(Ls), Ls


@pytest.mark.parametrize("growth", [16, 40])
def test_leaf_size_growing_with_n(growth):
    # R13 (Sec. 5: leaves of Theta(log n)): every build and resize sets the
    # leaf size for the key count it will hold; layout parity after every
    # batch while the set grows from 3000 to ~3e5 keys and back, and the leaf
    # size must have moved both ways.
    cfg = dict(leaf_bytes=256, leaf_growth=growth)
    base = W.uniform_keys(41, 3000, bits=40)
    g = cp.CPMA(T(base), **cfg)
    o = oracle.SeqCPMA(base, **cfg)
    p = oracle.PlainSet(base)
    same_layout(g, o)
    assert g.leaf_bytes() == o.leaf_bytes()
    sizes = [g.leaf_bytes()]
    for r in range(7):
        keys = W.uniform_keys(950 + r, 4000 * 2 ** r, bits=40)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
        sizes.append(g.leaf_bytes())
    same_queries(g, p, 960)
    for r in range(5):
        keys = W.sample_present(p.S, 970 + r, (len(p) * 3) // 4)
        assert int(g.delete_batch(T(keys)).item()) == o.delete_batch(keys) == p.delete_batch(keys)
        assert o.check() == 0
        same_layout(g, o)
        sizes.append(g.leaf_bytes())
    same_queries(g, p, 980)
    assert max(sizes) > sizes[0] and sizes[-1] < max(sizes), sizes


def test_grow_from_empty_and_delete_everything():
    g = cp.CPMA(None, leaf_bytes=256)
    o = oracle.SeqCPMA([], leaf_bytes=256)
    p = oracle.PlainSet([])
    same_layout(g, o)
    for r in range(6):
        keys = W.uniform_keys(40 + r, 3000 * (r + 1), bits=40)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    same_queries(g, p, 77)
    allk = p.S.copy()
    assert int(g.delete_batch(T(allk)).item()) == o.delete_batch(allk) == p.delete_batch(allk)
    same_layout(g, o)
    assert g.size() == 0 and g.leaves() == 1
    same_queries(g, p, 78)


def test_extreme_keys():
    g = cp.CPMA(None, leaf_bytes=256)
    o = oracle.SeqCPMA([], leaf_bytes=256)
    p = oracle.PlainSet([])
    for keys in ([M64, 0, M64], [1, M64 - 1, 1 << 63], list(range(2, 600)),
                 [M64 - i for i in range(2, 400)]):
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
        same_queries(g, p, 3)
    keys = [0, M64, 5, 7]
    assert int(g.delete_batch(T(keys)).item()) == o.delete_batch(keys) == p.delete_batch(keys)
    same_layout(g, o)
    same_queries(g, p, 4)


def test_single_key_batches_and_duplicates():
    base = W.uniform_keys(31, 8000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    for i in range(20):
        k = [int(W.uniform_keys(1000 + i, 1, bits=40)[0])]
        assert int(g.insert_batch(T(k)).item()) == o.insert_batch(k)
        k = [int(base[i * 7])] * 9000                  # one key repeated: sort copy path
        assert int(g.delete_batch(T(k)).item()) == o.delete_batch(k)
    same_layout(g, o)


def test_sorted_flag_rejects_unsorted_batch():
    base = W.uniform_keys(41, 5000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    before = [t.cpu().clone() for t in g.layout()]
    keys = W.uniform_keys(42, 3000, bits=40)             # not sorted
    with pytest.raises(cp.CPMAError) as e:
        g.insert_batch(T(keys), sorted=True)
    assert e.value.code == cp.CPMA_EINVAL
    after = [t.cpu() for t in g.layout()]
    assert all(torch.equal(a, b) for a, b in zip(before, after))
    assert g.size() == len(oracle.PlainSet(base))


def test_clone_is_independent():
    base = W.uniform_keys(51, 20000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    h = g.clone()
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    ins = W.uniform_keys(52, 5000, bits=40)
    h.insert_batch(T(ins))
    same_layout(g, o)
    o.insert_batch(ins)
    same_layout(h, o)


def test_config_plain_cpma():
    """uint64 keys uniform in [0, 2^40) from seed 1: build from 2^20 keys, one
    batch insert of 10^4 keys, one batch delete of 10^3 existing keys, then
    1000 range_map sums over [lo, lo + 2^24) with lo uniform."""
    base = W.uniform_keys(1, 1 << 20, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    p = oracle.PlainSet(base)
    same_layout(g, o)
    ins = W.uniform_keys(2, 10 ** 4, bits=40)
    assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins) == p.insert_batch(ins)
    same_layout(g, o)
    dele = W.sample_present(p.S, 3, 10 ** 3)
    assert int(g.delete_batch(T(dele)).item()) == o.delete_batch(dele) == p.delete_batch(dele)
    same_layout(g, o)
    lo, hi = W.range_queries_fixed_width(4, 1000, 1 << 24)
    s, c = g.range_map(T(lo), T(hi))
    ws, wc = p.range_map(lo, hi)
    assert np.array_equal(cp.to_u64(s), ws) and np.array_equal(cp.to_u64(c), wc)
    os_, oc = o.range_map(lo, hi)
    assert np.array_equal(os_, ws) and np.array_equal(oc, wc)
    same_queries(g, p, 9)


def test_many_uneven_ranges_one_launch():
    base = W.uniform_keys(61, 300000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    p = oracle.PlainSet(base)
    lo, hi, _ = W.range_queries_by_rank(p.S, 62, 20000, 1, 200000)
    s, c = g.range_map(T(lo), T(hi))
    ws, wc = p.range_map(lo, hi)
    assert np.array_equal(cp.to_u64(c), wc)
    assert np.array_equal(cp.to_u64(s), ws)


@pytest.mark.parametrize("point", [True, False])
@pytest.mark.parametrize("LB", [256, 512, 1024])
def test_small_batches_hit_every_splice_case(LB, point):
    """Many batches of 1..40 keys: keys just below / equal to / just above
    existing keys and heads, runs in one gap, keys past the last element,
    repeats and deletes of neighbours -- the splice paths' edge cases, with
    inserts taking the point path when it applies and with it off."""
    rng = np.random.default_rng(LB + 7)
    base = np.unique(W.uniform_keys(81, 6000, bits=30))
    g = cp.CPMA(T(base), leaf_bytes=LB)
    if not point:
        g.set_point_max(0)
    o = oracle.SeqCPMA(base, leaf_bytes=LB)
    p = oracle.PlainSet(base)
    for r in range(60):
        S = p.S
        k = int(rng.integers(1, 41))
        pick = S[rng.integers(0, S.size, size=k)].astype(np.int64)
        kind = r % 5
        if kind == 0:
            keys = pick + rng.integers(-2, 3, size=k)           # neighbours and equals
        elif kind == 1:
            _, _, heads = g.layout()
            hd = cp.to_u64(heads).astype(np.int64)
            keys = hd[rng.integers(0, hd.size, size=k)] + rng.integers(-3, 2, size=k)
        elif kind == 2:
            keys = np.concatenate([pick[:1] + np.arange(1, k + 1), pick[:1] + 1])  # one gap
        elif kind == 3:
            keys = np.int64(S[-1]) + rng.integers(1, 1 << 20, size=k)  # past the end
        else:
            keys = np.concatenate([pick, pick[:3]])
        keys = np.clip(keys, 0, None).astype(np.uint64)
        if r % 3 == 2:
            got = int(g.delete_batch(T(keys)).item())
            assert got == o.delete_batch(keys) == p.delete_batch(keys)
        else:
            got = int(g.insert_batch(T(keys)).item())
            assert got == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    same_queries(g, p, 85)


@pytest.mark.parametrize("LB", [256, 512, 2048])
def test_graph_updates_match_oracle(LB):
    """Updates whose front segment runs as a replayed CUDA graph (batches
    padded to a size bucket with copies of their last key) give the same
    counts, sets and byte layout as the oracle, through resizes (which force
    a new capture) and with several batch sizes sharing one bucket."""
    base = W.uniform_keys(31, 6000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB)
    g.set_point_max(0)  # small inserts take the batch algorithm (its graphs)
    g.use_graphs(1 << 20)
    g.reserve(4500)
    o = oracle.SeqCPMA(base, leaf_bytes=LB)
    p = oracle.PlainSet(base)
    sizes = [1, 7, 16, 17, 4000, 4100, 4095, 300, 300, 300, 4096, 4097]
    for r, k in enumerate(sizes * 2):
        if r % 3 == 2 and len(p):
            keys = W.sample_present(p.S, 800 + r, min(k, len(p)))
            keys = np.concatenate([keys, W.uniform_keys(850 + r, 5, bits=40)])
            got = int(g.delete_batch(T(keys)).item())
            assert got == o.delete_batch(keys) == p.delete_batch(keys)
        else:
            keys = W.uniform_keys(700 + r, k, bits=40)
            if r % 4 == 1:
                keys = np.sort(keys)
                got = int(g.insert_batch(T(keys), sorted=True).item())
            else:
                got = int(g.insert_batch(T(keys)).item())
            assert got == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    same_queries(g, p, 77, 200)
    st = g.graph_stats()
    assert st["launches"] == 2 * len(sizes)
    assert 0 < st["captures"] < st["launches"]


def test_graphs_replay_within_a_bucket():
    """After a reserve, batches of different sizes in one bucket reuse one
    captured graph until the leaf arrays are replaced."""
    base = W.uniform_keys(41, 200000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    g.set_point_max(0)
    g.use_graphs(1 << 20)
    g.reserve(1100)
    p = oracle.PlainSet(base)
    L0 = g.leaves()
    for r, k in enumerate([1000, 1001, 1024, 1010, 1023, 1017]):  # bucket 1024
        keys = W.uniform_keys(900 + r, k, bits=40)
        assert int(g.insert_batch(T(keys)).item()) == p.insert_batch(keys)
    assert g.leaves() == L0  # no resize at this fill
    assert g.graph_stats() == {"captures": 1, "launches": 6}
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == p.sum() and int(c.item()) == len(p)


def test_max_key_with_trailing_empty_leaf():
    """Low lower bounds leave an empty leaf after the one holding 2^64-1; the
    key must still route to the last non-empty leaf (has, insert, ranges)."""
    keys = np.array([4 * i for i in range(3000)] + [M64], dtype=np.uint64)
    cfg = dict(leaf_bytes=256, tau_leaf=900, tau_root=700, rho_leaf=5, rho_root=20)
    g = cp.CPMA(T(keys), **cfg)
    o = oracle.SeqCPMA(keys, **cfg)
    p = oracle.PlainSet(keys)
    dele = keys[2400:-1]
    assert int(g.delete_batch(T(dele)).item()) == o.delete_batch(dele) == p.delete_batch(dele)
    same_layout(g, o)
    _, used, _ = o.layout()
    assert used[-1] == 0 and used[-2] > 0
    q = np.array([M64, M64 - 1, 0, 4 * 2399], dtype=np.uint64)
    assert g.has_batch(T(q)).cpu().numpy().tolist() == p.has_batch(q).tolist() == [1, 0, 1, 1]
    for k in ([M64], [M64 - 1, M64]):
        k = np.array(k, dtype=np.uint64)
        assert int(g.insert_batch(T(k)).item()) == o.insert_batch(k) == p.insert_batch(k)
        same_layout(g, o)
    same_queries(g, p, 31, 100)


@pytest.mark.parametrize("LB", [256, 512, 2048])
def test_range_map_length_matches_oracle(LB):
    """App. A map_range_length: first `length` keys >= start, sum and count,
    against the plain set; lengths from 0 to 2^64-1, starts below, inside,
    between and above the keys, and after updates that empty leaves."""
    base = W.uniform_keys(51, 60000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB)
    p = oracle.PlainSet(base)
    rng = np.random.default_rng(LB)
    for step in range(3):
        S = p.S
        starts = np.concatenate([W.uniform_keys(60 + step, 2000, bits=40),
                                 S[rng.integers(0, S.size, 500)],
                                 S[rng.integers(0, S.size, 200)] + np.uint64(1),
                                 np.array([0, 1, M64, M64 - 1, S[-1], S[0]], np.uint64)])
        lens = np.concatenate([W.log_uniform_int(70 + step, starts.size - 6, 1, 10 ** 5)
                               .astype(np.uint64),
                               np.array([0, M64, 1, 5, 1, S.size + 3], np.uint64)])
        lens[::97] = 0
        lens[1::89] = M64
        s, c = g.range_map_length(T(starts), T(lens))
        ws, wc = p.range_map_length(starts, lens)
        assert np.array_equal(cp.to_u64(c), wc)
        assert np.array_equal(cp.to_u64(s), ws)
        # then change the set: a big delete (leaves empty and get refilled)
        dele = W.sample_present(S, 80 + step, S.size // 3)
        assert int(g.delete_batch(T(dele)).item()) == p.delete_batch(dele)
    # whole set, successor, empty set
    s, c = g.range_map_length(T(np.array([0], np.uint64)), M64)
    assert int(cp.to_u64(s)[0]) == p.sum() and int(c.item()) == len(p)
    e = cp.CPMA(None, leaf_bytes=LB)
    s, c = e.range_map_length(T(np.array([0, 5, M64], np.uint64)), 10)
    assert cp.to_u64(s).tolist() == [0, 0, 0] and cp.to_u64(c).tolist() == [0, 0, 0]


@pytest.mark.parametrize("op", ["sum", "min", "max", "xor"])
def test_range_reduce_matches_oracle(op):
    base = np.concatenate([W.uniform_keys(52, 80000, bits=40), np.array([0, M64 - 1], np.uint64)])
    g = cp.CPMA(T(base), leaf_bytes=512)
    p = oracle.PlainSet(base)
    lo, hi, _ = W.range_queries_by_rank(p.S, 53, 1500, 1, 20000)
    lo = np.concatenate([lo, np.array([0, 0, 5, M64, M64 - 1], np.uint64)])
    hi = np.concatenate([hi, np.array([M64, 1, 5, M64, M64], np.uint64)])
    for mask, value in [(0, 0), (1, 0), (0xFF, 0x3C), (1 << 39, 1 << 39)]:
        r, c = g.range_reduce(T(lo), T(hi), op, mask, value)
        wr, wc = p.range_reduce(lo, hi, op, mask, value)
        assert np.array_equal(cp.to_u64(c), wc)
        assert np.array_equal(cp.to_u64(r), wr)


@pytest.mark.parametrize("LB", [256, 512, 2048])
def test_rebuild_threshold_matches_oracle(LB):
    """rebuild_pm > 0: batches with 1000 k >= rebuild_pm n are applied by a
    merge of everything and a fresh build (reading R14); the others by the
    batch merge.  Counts, sets and layouts against the oracle, across the
    threshold, for inserts, deletes, sorted batches and an empty start."""
    cfg = dict(leaf_bytes=LB, rebuild_pm=100)
    g = cp.CPMA(None, **cfg)
    o = oracle.SeqCPMA([], **cfg)
    p = oracle.PlainSet([])
    rng = np.random.default_rng(LB + 1)
    for r in range(14):
        n = len(p)
        kind = r % 4
        if kind == 0 or n == 0:   # large insert: rebuild (or first fill)
            keys = W.uniform_keys(400 + r, max(n // 5, 5000), bits=40)
            keys = np.concatenate([keys, keys[:100]])
        elif kind == 1:           # small insert, below the threshold: merge
            keys = W.uniform_keys(400 + r, max(1, n // 50), bits=40)
        elif kind == 2:           # large delete of present and absent keys
            keys = np.concatenate([W.sample_present(p.S, 500 + r, n // 4),
                                   W.uniform_keys(600 + r, 50, bits=40)])
        else:                     # sorted batch exactly at the threshold
            k = -(-100 * n // 1000)
            keys = np.sort(W.uniform_keys(700 + r, k, bits=40))
        srt = kind == 3
        if kind == 2:
            got = int(g.delete_batch(T(keys)).item())
            assert got == o.delete_batch(keys) == p.delete_batch(keys)
        else:
            got = int(g.insert_batch(T(keys), sorted=srt).item())
            assert got == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    same_queries(g, p, 88, 200)
    # an unsorted batch flagged sorted is rejected on the rebuild path too
    bad = np.array([9, 3, 5], np.uint64)
    small = cp.CPMA(T(np.array([1, 2], np.uint64)), **cfg)
    with pytest.raises(cp.CPMAError):
        small.insert_batch(T(bad), sorted=True)
    assert small.size() == 2


@pytest.mark.parametrize("LB", [256, 512, 2048])
def test_range_extract_matches_oracle(LB):
    base = np.concatenate([W.uniform_keys(54, 70000, bits=40), np.array([0, M64], np.uint64)])
    g = cp.CPMA(T(base), leaf_bytes=LB)
    p = oracle.PlainSet(base)
    lo, hi, _ = W.range_queries_by_rank(p.S, 55, 700, 1, 30000)
    lo = np.concatenate([lo, np.array([0, 0, 5, M64, M64 - 1, 9], np.uint64)])
    hi = np.concatenate([hi, np.array([M64, 1, 5, M64, M64, 3], np.uint64)])
    off, keys = g.range_extract(T(lo), T(hi))
    woff, wkeys = p.range_extract(lo, hi)
    assert np.array_equal(cp.to_u64(off), woff)
    assert np.array_equal(cp.to_u64(keys), wkeys)
    # counts agree with range_map
    s, c = g.range_map(T(lo), T(hi))
    assert np.array_equal(np.diff(cp.to_u64(off)), cp.to_u64(c))
    # no queries
    off, keys = g.range_extract(T(np.zeros(0, np.uint64)), T(np.zeros(0, np.uint64)))
    assert cp.to_u64(off).tolist() == [0] and keys.numel() == 0


@pytest.mark.parametrize("LB", [512, 2048])
def test_full_scan_large(LB):
    """Full scan at 1e7 keys (every warp walks many 32-leaf groups with the
    next group's chunks loaded ahead): sum and count against the plain set,
    also after a skewed insert that leaves leaves of very different fill."""
    keys = W.uniform_keys(71, 10 ** 7, bits=40)
    g = cp.CPMA(T(keys), leaf_bytes=LB)
    S = sorted_unique(keys)
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == int(np.sum(S, dtype=np.uint64)) and int(c.item()) == S.size
    ins = W.zipf_keys(72, 10 ** 6, bits=40)
    g.insert_batch(T(ins))
    S = union(S, ins)
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == int(np.sum(S, dtype=np.uint64)) and int(c.item()) == S.size


@pytest.mark.parametrize("LB", [256, 512, 2048])
@pytest.mark.parametrize("n", [0, 1, 5000, 70000])
def test_pma_build_layout(LB, n):
    """Uncompressed PMA (codec 1): build layout and queries against the
    oracle's cells."""
    keys = W.uniform_keys(13 + n, n, bits=40)
    keys = np.concatenate([keys, keys[: n // 4], np.array([M64], np.uint64)]) if n else keys
    g = cp.CPMA(T(keys) if keys.size else None, leaf_bytes=LB, codec=1)
    o = oracle.SeqCPMA(keys, leaf_bytes=LB, codec=1)
    same_layout(g, o)
    same_queries(g, oracle.PlainSet(keys), 17 + n)


@pytest.mark.parametrize("LB", [256, 1024])
def test_pma_update_sequence(LB):
    """Uncompressed PMA through inserts, zipfian hot leaves, sorted batches,
    deletes (shrink) and full-range keys: counts, layout and every query
    kind against the oracle."""
    base = W.uniform_keys(23, 30000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=LB, codec=1)
    o = oracle.SeqCPMA(base, leaf_bytes=LB, codec=1)
    p = oracle.PlainSet(base)
    for r in range(18):
        kind = r % 6
        if kind == 0:
            keys = W.uniform_keys(110 + r, 20000, bits=40)
        elif kind == 1:
            keys = W.zipf_keys(210 + r, 20000, bits=34)
        elif kind == 2:
            keys = np.sort(W.uniform_keys(310 + r, 5000, bits=40))
        elif kind == 3:
            keys = np.concatenate([W.sample_present(p.S, 410 + r, 4000),
                                   W.uniform_keys(510 + r, 1000, bits=40)])
        elif kind == 4:
            keys = W.sample_present(p.S, 610 + r, len(p) // 2)
        else:
            keys = W.full_range_keys(710 + r, 3000)
        if kind in (3, 4):
            assert int(g.delete_batch(T(keys)).item()) == o.delete_batch(keys) == p.delete_batch(keys)
        else:
            got = int(g.insert_batch(T(keys), sorted=kind == 2).item())
            assert got == o.insert_batch(keys) == p.insert_batch(keys)
        same_layout(g, o)
    same_queries(g, p, 919, 200)
    lo, hi, c = W.range_queries_by_rank(p.S, 920, 300, 1, 5000)
    s1, c1 = g.range_map_length(T(lo), T(c.astype(np.uint64)))
    ws, wc = p.range_map_length(lo, c.astype(np.uint64))
    assert np.array_equal(cp.to_u64(s1), ws) and np.array_equal(cp.to_u64(c1), wc)
    off, keys = g.range_extract(T(lo), T(hi))
    woff, wkeys = p.range_extract(lo, hi)
    assert np.array_equal(cp.to_u64(off), woff) and np.array_equal(cp.to_u64(keys), wkeys)
    r_, c_ = g.range_reduce(T(lo), T(hi), "max", 3, 1)
    wr, wc = p.range_reduce(lo, hi, "max", 3, 1)
    assert np.array_equal(cp.to_u64(r_), wr) and np.array_equal(cp.to_u64(c_), wc)


def test_degenerate_batches_and_queries():
    """Batches of one repeated key, of keys all present, deletes from an
    empty set, empty query batches, and a batch length at the 2^31 limit
    (rejected before anything is read)."""
    base = W.uniform_keys(81, 50000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    p = oracle.PlainSet(base)
    same = np.full(5000, 123456789, dtype=np.uint64)
    assert int(g.insert_batch(T(same)).item()) == o.insert_batch(same) == p.insert_batch(same) == 1
    present = p.S[::3].copy()
    assert int(g.insert_batch(T(present)).item()) == o.insert_batch(present) == 0
    same_layout(g, o)
    e = cp.CPMA(None, leaf_bytes=256)
    assert int(e.delete_batch(T(base[:100])).item()) == 0 and e.size() == 0
    z = T(np.zeros(0, np.uint64))
    assert int(g.insert_batch(z).item()) == 0 and int(g.delete_batch(z).item()) == 0
    assert g.has_batch(z).numel() == 0
    s, c = g.range_map(z, z)
    assert s.numel() == 0 and c.numel() == 0
    one = T(np.array([5], np.uint64))
    added = torch.zeros(1, dtype=torch.int64, device="cuda")
    rc = cp.lib().cpma_insert_batch(g.handle, cp._ptr(one), 1 << 31, 0, cp._ptr(added), None)
    assert rc == cp.CPMA_EINVAL
    same_layout(g, o)


def test_profiling_with_graph_replays():
    """Per-phase profiling stays live when the front segment is a replayed
    graph (its phase boundaries are event nodes): phase times and calls
    accumulate per replay, and results still match the oracle."""
    base = W.uniform_keys(91, 100000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    g.set_point_max(0)
    g.use_graphs(1 << 20)
    g.reserve(3000)
    g.profile(True)
    for r in range(5):
        keys = W.uniform_keys(920 + r, 3000, bits=40)
        assert int(g.insert_batch(T(keys)).item()) == o.insert_batch(keys)
    prof = g.profile_read()
    same_layout(g, o)
    st = g.graph_stats()
    assert st["launches"] == 5 and st["captures"] >= 1
    for ph in ("sort", "route", "merge"):
        assert prof[ph]["calls"] == 5 and prof[ph]["ms"] > 0, (ph, prof[ph])
    # batches this small merge with a warp per leaf (the lane-granular phase)
    assert prof["merge"]["bytes"] + prof["merge_lane"]["bytes"] > 0
    g.profile(False)


@pytest.mark.parametrize("bits", [40, 26])
def test_insert_five_to_eight_keys_per_leaf(bits):
    """Batches of about six keys per touched leaf: slices of up to 4 keys take
    the thread-granular insert, larger ones the lane-granular insert running
    on the side stream at the same time (or the element-array splice).
    26-bit keys make one-byte codes and full leaves.  Layout against the
    sequential oracle; per-request counts of a tagged insert against applying
    the requests in order."""
    base = W.uniform_keys(71 + bits, 1 << 18, bits=bits)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    p = oracle.PlainSet(base)
    ins = W.uniform_keys(72 + bits, 6 * g.leaves(), bits=bits)
    assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins) == p.insert_batch(ins)
    same_layout(g, o)
    # tagged: 7 requests of consecutive keys
    more = W.uniform_keys(73 + bits, 6 * g.leaves(), bits=bits)
    tags = (np.arange(more.size) * 7 // more.size).astype(np.int32)
    counts = torch.zeros(7, dtype=torch.int64, device="cuda")
    cp.cpma_insert_batch_tagged(g.handle, T(more), torch.from_numpy(tags).cuda(), 7, counts)
    seen = set(p.S.tolist())
    want = [0] * 7
    for x, t in zip(more.tolist(), tags.tolist()):
        if x not in seen:
            seen.add(x)
            want[t] += 1
    assert counts.cpu().tolist() == want
    o.insert_batch(more)
    same_layout(g, o)


@pytest.mark.parametrize("k", [160_000, 320_000, 640_000])
def test_route_tile_sizes(k):
    # batches dense against the leaves, large enough for routing tiles of
    # 2, 4 and 8 keys per thread (512, 1024, 2048 keys per tile), inserted
    # unsorted, pre-sorted (with repeats) and deleted, layout against the oracle
    base = W.uniform_keys(141, 400_000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=512)
    o = oracle.SeqCPMA(base, leaf_bytes=512)
    ins = W.uniform_keys(142 + k, k, bits=40)
    assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins)
    same_layout(g, o)
    srt = np.sort(np.concatenate([W.uniform_keys(143 + k, k - k // 8, bits=40), ins[: k // 8]]))
    assert int(g.insert_batch(T(srt), sorted=True).item()) == o.insert_batch(srt)
    same_layout(g, o)
    gone = W.sample_present(oracle.PlainSet(np.concatenate([base, ins, srt])).S, 144 + k, k)
    assert int(g.delete_batch(T(gone)).item()) == o.delete_batch(gone)
    same_layout(g, o)


def test_route_sparse_tiles():
    # small batches against many leaves: a 256-key tile reaches more heads
    # than shared memory holds, so every step-th head is staged and the last
    # candidates are searched in the global array (keys 0 and 2^64-1 too)
    base = W.uniform_keys(151, 2_000_000, bits=40)
    g = cp.CPMA(T(base), leaf_bytes=256)
    g.set_point_max(0)  # the batch algorithm's routing
    o = oracle.SeqCPMA(base, leaf_bytes=256)
    assert g.leaves() > 4 * 4096
    for r, k in enumerate([1, 37, 1000, 5000]):
        ins = np.concatenate([W.uniform_keys(152 + r, k, bits=40),
                              np.array([0, M64], np.uint64)])
        assert int(g.insert_batch(T(ins)).item()) == o.insert_batch(ins)
        same_layout(g, o)
        gone = W.sample_present(np.unique(ins), 160 + r, max(1, k // 2))
        assert int(g.delete_batch(T(gone)).item()) == o.delete_batch(gone)
        same_layout(g, o)
