"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: codec vectors from
the LEB128 definition, closed forms, hand-derived layouts of small CPMAs
(derivations in the comments, from the readings of Sec. 3-5 listed in
``oracle/cpma_oracle.c``), Python's own set semantics by brute force, and the
structural invariants of Sec. 3 and Sec. 5.
"""
import os
import random

import numpy as np
import pytest

import oracle
from paper_2305_05055_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
M64 = (1 << 64) - 1
CFG = dict(tau_leaf=900, tau_root=700, rho_leaf=100, rho_root=300)


# --------------------------------------------------------------------------
# codec (Sec. 5 "Data compression techniques")
# --------------------------------------------------------------------------

def _golden_leb():
    out = []
    with open(os.path.join(GOLDEN, "leb128.txt")) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                v, h = line.split()
                out.append((int(v), bytes.fromhex(h)))
    return out


@pytest.mark.parametrize("value,enc", _golden_leb())
def test_leb128_vectors(value, enc):
    assert oracle.leb_put(value) == enc
    assert oracle.leb_get(enc) == (value, len(enc))
    assert oracle.leb_len(value) == len(enc)


def test_leb128_length_closed_form_bruteforce():
    # len(d) = max(1, ceil(bitlen(d) / 7)) for every d < 2^16 and at every
    # group boundary up to 2^64 - 1.
    vals = list(range(1 << 16))
    for i in range(1, 10):
        vals += [(1 << (7 * i)) - 1, 1 << (7 * i), (1 << (7 * i)) + 1]
    vals += [M64, M64 - 1, 1 << 63]
    for d in vals:
        want = max(1, -(-d.bit_length() // 7))
        assert oracle.leb_len(d) == want, d


def test_leb128_roundtrip_and_minimal():
    rng = random.Random(7)
    for _ in range(3000):
        d = rng.getrandbits(rng.randint(1, 64))
        b = oracle.leb_put(d)
        assert oracle.leb_get(b) == (d, len(b))
        # continue bit on every byte but the last; no redundant zero group
        assert all(x & 0x80 for x in b[:-1]) and not (b[-1] & 0x80)
        assert len(b) == 1 or b[-1] != 0


def test_leaf_encode_hand_example():
    # e = [5, 6, 306]: head 5 as 8 little-endian bytes, delta 1 -> 01,
    # delta 300 -> ac 02; 11 bytes used, the rest zero (packed left).
    buf, used = oracle.leaf_encode([5, 6, 306], 64)
    assert used == 11
    assert bytes(buf[:11]) == bytes([5, 0, 0, 0, 0, 0, 0, 0, 0x01, 0xAC, 0x02])
    assert not buf[11:].any()
    assert list(oracle.leaf_decode(buf, used)) == [5, 6, 306]
    # head of 2^64-1 and a single element
    buf, used = oracle.leaf_encode([M64], 64)
    assert used == 8 and bytes(buf[:8]) == b"\xff" * 8
    buf, used = oracle.leaf_encode([], 64)
    assert used == 0 and not buf.any()


def test_leaf_roundtrip_random():
    rng = np.random.default_rng(3)
    for bits in (8, 20, 40, 64):
        for m in (1, 2, 17, 60):
            e = np.unique(rng.integers(0, 2 ** min(bits, 63), size=m, dtype=np.uint64))
            if bits == 64:
                e = np.unique(np.concatenate([e, np.array([M64], np.uint64)]))
            nbytes = oracle.leaf_bytes(e)
            assert nbytes == 8 + sum(oracle.leb_len(int(b) - int(a)) for a, b in zip(e[:-1], e[1:]))
            buf, used = oracle.leaf_encode(e, 1024)
            assert used == nbytes
            assert np.array_equal(oracle.leaf_decode(buf, used), e)


# --------------------------------------------------------------------------
# density bounds (Sec. 3; byte density Sec. 5)
# --------------------------------------------------------------------------

def V(H, h, leaves, b, LB=512):
    return oracle.violates(LB, CFG["tau_leaf"], CFG["tau_root"], CFG["rho_leaf"],
                           CFG["rho_root"], H, h, leaves, b)


def test_bounds_hand_values():
    # H = 3, LB = 512.  Leaf (h=0): upper 0.9*512 = 460.8, lower 0.1*512 = 51.2
    assert not V(3, 0, 1, 460) and V(3, 0, 1, 461)
    assert V(3, 0, 1, 51) and not V(3, 0, 1, 52)
    # h = 1, two leaves (cap 1024): tau = 0.9 - 0.2/3 -> 853.33; rho = 0.1 + 0.2/3 -> 170.67
    assert not V(3, 1, 2, 853) and V(3, 1, 2, 854)
    assert V(3, 1, 2, 170) and not V(3, 1, 2, 171)
    # h = 2 clipped to three leaves (L = 7): cap 1536, tau = 0.9 - 0.4/3 -> 1177.6
    # rho = 0.1 + 0.4/3 -> 358.4
    assert not V(3, 2, 3, 1177) and V(3, 2, 3, 1178)
    assert V(3, 2, 3, 358) and not V(3, 2, 3, 359)
    # root h = H = 3, eight leaves (cap 4096): tau_root 2867.2, rho_root 1228.8
    assert not V(3, 3, 8, 2867) and V(3, 3, 8, 2868)
    assert V(3, 3, 8, 1228) and not V(3, 3, 8, 1229)
    # a single leaf is the root: upper 0.7*512 = 358.4, no lower bound
    assert not V(0, 0, 1, 358) and V(0, 0, 1, 359)
    assert not V(0, 0, 1, 0)
    # overflowed leaves (more than LB bytes) always violate
    assert V(5, 0, 1, 600)


def test_build_and_resize_leaf_counts():
    # build: L = max(1, ceil(1000 S / (500*512 - 8000))) = ceil(S / 248)
    assert oracle.build_leaves(0, 512, 500) == 1
    assert oracle.build_leaves(248, 512, 500) == 1
    assert oracle.build_leaves(249, 512, 500) == 2
    assert oracle.build_leaves(248 * 1000, 512, 500) == 1000
    assert oracle.build_leaves(248 * 1000 + 1, 512, 500) == 1001
    # grow (x6/5 rounded up) until 1000 T <= 700 L' 512
    assert oracle.resize_leaves(3585, 10, 512, 700, 300) == 12
    assert oracle.resize_leaves(5000, 10, 512, 700, 300) == 15   # 10 -> 12 -> 15
    assert oracle.resize_leaves(400, 1, 512, 700, 300) == 2
    # shrink (x5/6 rounded down) while 1000 T < 300 L' 512 and L' > 1
    assert oracle.resize_leaves(1000, 10, 512, 700, 300) == 6    # 10 -> 8 -> 6
    assert oracle.resize_leaves(10, 10, 512, 700, 300) == 1


def test_cut_points_hand_values():
    e = list(range(10))  # costs 8,1,1,...,1 -> C = 0,8,9,...,17; S = 17
    # W = 2: theta_1 = floor(17/2) = 8 -> first C_i >= 8 is i = 1
    assert list(oracle.cut_points(e, 2)) == [0, 1, 10]
    # W = 3: thetas 0, 5, 11 -> starts 0, 1, 4
    assert list(oracle.cut_points(e, 3)) == [0, 1, 4, 10]
    # one element over three leaves: C = 0, 8; thetas 0, 2, 5 -> 0, 1, 1
    assert list(oracle.cut_points([42], 3)) == [0, 1, 1, 1]
    # no elements
    assert list(oracle.cut_points([], 4)) == [0, 0, 0, 0, 0]
    # a 3-byte delta: e = [0, 1, 2^14 + 1, 2^14 + 2]: costs 8, 1, 3, 1 -> C = 0, 8, 9, 12, 13
    # W = 2: theta_1 = 6 -> i = 1.  W = 4: thetas 0, 3, 6, 9 -> 0, 1, 1, 2
    e = [0, 1, (1 << 14) + 1, (1 << 14) + 2]
    assert list(oracle.cut_points(e, 2)) == [0, 1, 4]
    assert list(oracle.cut_points(e, 4)) == [0, 1, 1, 2, 4]


# --------------------------------------------------------------------------
# hand-derived sequential CPMA scenarios (LB = 256)
# --------------------------------------------------------------------------
#
# Keys 4i for i < 600: every delta is 4 (one byte), so the stream costs
# S = 8 + 599 = 607 bytes.  Build: L = ceil(607000 / (500*256 - 8000)) =
# ceil(5.06) = 6 leaves, H = 3.  Cut points: C_i = i + 7 for i >= 1 and
# theta_w = floor(607 w / 6) = 0, 101, 202, 303, 404, 505, so s_w = theta_w - 7
# = 0, 94, 195, 296, 397, 498 (s_6 = 600).  Leaf j holds 4i for i in
# [s_j, s_{j+1}) and uses 8 + (count - 1) bytes.

def _base():
    return oracle.SeqCPMA([4 * i for i in range(600)][::-1] + [8, 8, 12],
                          leaf_bytes=256, **CFG)


def test_scenario_build():
    o = _base()
    data, used, head = o.layout()
    assert o.leaves() == 6 and o.size() == 600
    assert list(used) == [101, 108, 108, 108, 108, 109]
    assert list(head) == [0, 376, 780, 1184, 1588, 1992]
    assert o.bytes() == 6 * (256 + 16)
    assert o.check() == 0


def test_scenario_window_at_level_one():
    # Insert 4i+1 and 4i+2 for i in [195, 270): 150 keys, all routed to leaf 2
    # (heads 780 <= key < 1184).  Each splits a 4-delta into 1+1+2... all
    # one-byte codes, so leaf 2 grows from 108 to 258 bytes (> 0.9*256 = 230.4).
    # Level 1, leaves [2, 4): 258 + 108 = 366 bytes against
    # 512 * (0.9 - 0.2/3) = 426.7 and 512 * (0.1 + 0.2/3) = 85.3: within
    # bounds, so the window is leaves [2, 4).  It holds 251 + 101 = 352
    # elements, all deltas one byte: S = 359, theta_1 = floor(359/2) = 179,
    # s_1 = 179 - 7 = 172.  Leaf 2: 172 elements -> 179 bytes; leaf 3: 180
    # elements -> 187 bytes.  Element 172 is the second of triplet 57 of leaf
    # 2's (4i, 4i+1, 4i+2) run: i = 195 + 57 = 252, key 4*252 + 1 = 1009.
    o = _base()
    ins = [4 * i + 1 for i in range(195, 270)] + [4 * i + 2 for i in range(195, 270)]
    assert o.insert_batch(ins) == 150
    lb = o.last_batch()
    assert lb == dict(resized=0, nwindows=1, touched=1)
    assert o.last_windows().tolist() == [[2, 2]]
    data, used, head = o.layout()
    assert list(used) == [101, 108, 179, 187, 108, 109]
    assert list(head) == [0, 376, 780, 1009, 1588, 1992]
    assert o.check() == 0


def test_scenario_in_place():
    # 100 keys 4i+1 for i in [195, 295) into leaf 2: 108 + 100 = 208 bytes,
    # within 230.4, so only leaf 2 is rewritten in place.
    o = _base()
    assert o.insert_batch([4 * i + 1 for i in range(195, 295)]) == 100
    assert o.last_batch() == dict(resized=0, nwindows=0, touched=1)
    _, used, head = o.layout()
    assert list(used) == [101, 108, 208, 108, 108, 109]
    assert list(head) == [0, 376, 780, 1184, 1588, 1992]


def test_resize_leaf_counts_other_growing_factors():
    # App. C sweeps the growing factor over 1.1 ... 2; R9 with g = num/den:
    # grow L' = ceil(L' num / den) while 1000 T > 700 L' 512 = 358400 L',
    # shrink L' = floor(L' den / num) while L' > 1 and 1000 T < 153600 L'.
    R = oracle.resize_leaves
    # g = 11/10, T = 5000 (5,000,000): 10 -> 11 (3,942,400) -> ceil(12.1) = 13
    # (4,659,200) -> ceil(14.3) = 15 (5,376,000 >= 5,000,000)
    assert R(5000, 10, 512, 700, 300, 11, 10) == 15
    # one leaf: ceil(1.1) = 2 (716,800 >= 400,000)
    assert R(400, 1, 512, 700, 300, 11, 10) == 2
    # shrink, T = 1000 (1,000,000): 10 -> floor(100/11) = 9 (1,382,400) -> 8
    # (1,228,800) -> 7 (1,075,200) -> floor(70/11) = 6 (921,600: stop)
    assert R(1000, 10, 512, 700, 300, 11, 10) == 6
    assert R(1000, 11, 512, 700, 300, 11, 10) == 6   # 11 -> 10 -> 9 -> 8 -> 7 -> 6
    # g = 3/2: T = 9000 (9,000,000): 10 -> 15 (5,376,000) -> ceil(22.5) = 23
    # (8,243,200) -> ceil(34.5) = 35 (12,544,000)
    assert R(9000, 10, 512, 700, 300, 3, 2) == 35
    assert R(5000, 10, 512, 700, 300, 3, 2) == 15
    # shrink T = 1000: 10 -> floor(20/3) = 6 (921,600: stop); T = 300
    # (300,000): 10 -> 6 (921,600) -> 4 (614,400) -> 2 (307,200) -> 1
    assert R(1000, 10, 512, 700, 300, 3, 2) == 6
    assert R(300, 10, 512, 700, 300, 3, 2) == 1
    # g = 2: T = 9000: 10 -> 20 (7,168,000) -> 40 (14,336,000)
    assert R(9000, 10, 512, 700, 300, 2, 1) == 40
    assert R(400, 1, 512, 700, 300, 2, 1) == 2
    # shrink T = 1000: 10 -> 5 (768,000: stop); T = 300: 10 -> 5 -> 2
    # (307,200) -> 1
    assert R(1000, 10, 512, 700, 300, 2, 1) == 5
    assert R(300, 10, 512, 700, 300, 2, 1) == 1
    # at the exact bound nothing moves: 1000 T = 358400 L and 153600 L
    for num, den in ((6, 5), (11, 10), (3, 2), (2, 1)):
        assert R(3584, 10, 512, 700, 300, num, den) == 10
        assert R(1536, 10, 512, 700, 300, num, den) == 10


def test_leaf_size_grows_with_log_n():
    # R13: LB(n) = min(2048, max(LB_min, 16 ceil(g bitlen(n) / 16))); g = 0
    # keeps LB_min
    S = oracle.leaf_size
    assert S(10 ** 8, 512, 0) == 512 and S(0, 256, 0) == 256
    assert S(0, 256, 16) == 256                  # bitlen 0
    assert S(10 ** 6, 256, 16) == 320            # bitlen 20: 320
    assert S(10 ** 8, 256, 16) == 432            # bitlen 27: 432
    assert S(1 << 63, 256, 16) == 1024           # bitlen 64
    assert S(10 ** 8, 256, 40) == 1088           # 27 * 40 = 1080 -> 1088
    assert S(1 << 30, 256, 100) == 2048          # 3100 clipped
    assert S(4095, 256, 24) == 288 and S(4096, 256, 24) == 320   # bitlen 12 / 13
    assert S(600, 256, 24) == 256                # 240 < LB_min


def test_scenario_grow_with_leaf_growth():
    # The grow scenario below with g = 24: the build of 600 keys keeps 256-byte
    # leaves (bitlen 10: 240 < 256); after the insert the array holds 2397
    # keys (bitlen 12: LB' = 288).  The resize starts from the leaf count of
    # equal capacity, ceil(6 * 256 / 288) = 6, and grows while 1000 * 2439 >
    # 700 * L' * 288: 6 -> 8 -> 10 -> 12 (2,419,200) -> 15.  The cut points do
    # not depend on LB, so the used bytes and heads are those of the 6/5 case.
    o = oracle.SeqCPMA([4 * i for i in range(600)][::-1] + [8, 8, 12], leaf_bytes=256,
                       leaf_growth=24, **CFG)
    assert o.leaf_bytes() == 256 and o.leaves() == 6
    ins = [4 * i + r for i in range(599) for r in (1, 2, 3)]
    assert o.insert_batch(ins) == 1797
    assert o.last_batch()["resized"] == 1
    assert o.leaf_bytes() == 288 and o.leaves() == 15
    assert o.bytes() == 15 * (288 + 16)
    s = [0] + [2404 * w // 15 - 7 for w in range(1, 15)] + [2397]
    data, used, head = o.layout()
    assert data.size == 15 * 288
    assert list(used) == [s[w + 1] - s[w] + 7 for w in range(15)]
    elems = sorted([4 * i for i in range(600)] + ins)
    assert list(head) == [elems[s[w]] for w in range(15)]
    assert o.check() == 0


def test_scenario_shrink_with_leaf_growth():
    # g = 24, LB_min = 256.  Build from 4i, i < 5000: bitlen 13 -> LB = 320;
    # stream S = 8 + 4999 = 5007 bytes, L = ceil(5,007,000 / (500*320 -
    # 8000)) = 33.  Deleting 4i for 100 <= i < 4900 leaves 200 keys (bitlen 8:
    # 192 -> LB' = 256): leaves 0 and 32 keep 100 keys each (107 bytes), the
    # others empty; the walks pass the root (214 bytes against 300 permille
    # of 33 * 320), so resize: start at ceil(33 * 320 / 256) = 42, shrink
    # while 214,000 < 300 * L' * 256: 42 -> 35 -> 29 -> 24 -> 20 -> 16 -> 13
    # -> 10 -> 8 -> 6 -> 5 -> 4 -> 3 -> 2 (153,600: stop).  Costs: head 8,
    # then 1 per delta of 4 except 19600 - 396 = 19204 (3 bytes): S = 209;
    # s_1 = min{i : C_i >= 104} = 97 (C_i = i + 7 up to i = 100), so leaf 0
    # holds elements 0..96 (8 + 96 = 104 bytes) and leaf 1 the rest, from key
    # 388 (8 + 2 + 3 + 99 = 112 bytes).
    o = oracle.SeqCPMA([4 * i for i in range(5000)], leaf_bytes=256, leaf_growth=24, **CFG)
    assert o.leaf_bytes() == 320 and o.leaves() == 33
    assert o.delete_batch([4 * i for i in range(100, 4900)]) == 4800
    assert o.last_batch()["resized"] == 1
    assert o.leaf_bytes() == 256 and o.leaves() == 2
    _, used, head = o.layout()
    assert list(used) == [104, 112] and list(head) == [0, 388]
    assert o.bytes() == 2 * (256 + 16)
    assert o.check() == 0


@pytest.mark.parametrize("num,den,Lp", [(6, 5, 15), (11, 10, 15), (3, 2, 14), (2, 1, 24)])
def test_scenario_grow(num, den, Lp):
    # Insert 4i+1, 4i+2, 4i+3 for every i < 599: 1797 keys, every delta
    # becomes 1.  Per leaf after the merge: leaf 0 has 94*4 = 376 elements
    # (383 bytes), leaves 1-4 have 404 (411 bytes), leaf 5 has 102 + 101*3 =
    # 405 (412 bytes): T = 383 + 4*411 + 412 = 2439.  Every walk passes the
    # root, so resize while 1000 T = 2,439,000 > 700 * L' * 256, i.e. until
    # L' >= 13.62: g = 6/5: 6 -> 8 -> 10 -> 12 -> 15; g = 11/10: 6 -> 7 -> 8
    # -> 9 -> 10 -> 11 -> 13 -> 15; g = 3/2: 6 -> 9 -> 14; g = 2: 6 -> 12 ->
    # 24.  2397 elements, S = 8 + 2396 = 2404, all costs after the first are
    # 1, so s_w = floor(2404 w / L') - 7 (every cut is past the head's 8
    # bytes) and leaf w uses s_{w+1} - s_w + 7 bytes.
    o = oracle.SeqCPMA([4 * i for i in range(600)][::-1] + [8, 8, 12], leaf_bytes=256,
                       grow_num=num, grow_den=den, **CFG)
    ins = [4 * i + r for i in range(599) for r in (1, 2, 3)]
    assert o.insert_batch(ins) == 1797
    assert o.last_batch()["resized"] == 1
    assert o.leaves() == Lp
    s = [0] + [2404 * w // Lp - 7 for w in range(1, Lp)] + [2397]
    _, used, head = o.layout()
    assert list(used) == [s[w + 1] - s[w] + 7 for w in range(Lp)]
    elems = sorted([4 * i for i in range(600)] + ins)
    assert list(head) == [elems[s[w]] for w in range(Lp)]
    assert o.check() == 0


@pytest.mark.parametrize("num,den", [(6, 5), (11, 10), (3, 2), (2, 1)])
def test_scenario_shrink(num, den):
    # Delete 4i for i in [50, 550): leaves 1-4 become empty (0 bytes), leaves
    # 0 and 5 keep 50 elements (57 bytes).  Leaf 0 is within [25.6, 230.4]:
    # rewritten in place.  Leaf 1: 0 < 25.6 -> walk: [0,2) 57 < 85.3,
    # [0,4) 57 < 1024 * (0.1 + 0.4/3) = 238.9, root [0,6) 114 < 0.3*1536 =
    # 460.8 -> resize.  T = 114: shrink 6 -> 5 -> 4 -> 3 -> 2 -> 1 (at every
    # step 114000 < 300 * L' * 256; with g = 11/10: 6 -> 5 -> 4 -> 3 -> 2 ->
    # 1, g = 3/2: 6 -> 4 -> 2 -> 1, g = 2: 6 -> 3 -> 1).  One leaf: 100
    # elements, deltas 4 (1 byte) except 4*550 - 4*49 = 2004 (2 bytes): 8 +
    # 98 + 2 = 108 bytes.
    o = oracle.SeqCPMA([4 * i for i in range(600)][::-1] + [8, 8, 12], leaf_bytes=256,
                       grow_num=num, grow_den=den, **CFG)
    assert o.delete_batch([4 * i for i in range(50, 550)] + [3, 5, 7]) == 500
    assert o.last_batch()["resized"] == 1
    assert o.leaves() == 1
    _, used, head = o.layout()
    assert list(used) == [108] and list(head) == [0]
    assert o.check() == 0


def test_scenario_empty_and_extremes():
    o = oracle.SeqCPMA([], leaf_bytes=256, **CFG)
    assert o.leaves() == 1 and o.size() == 0
    _, used, head = o.layout()
    assert list(used) == [0] and list(head) == [M64]   # empty leaf: 2^64-1
    assert o.insert_batch([M64, 0, M64]) == 2
    _, used, head = o.layout()
    # head 0 (8 bytes) + delta 2^64-1 (10 bytes)
    assert list(used) == [18] and list(head) == [0]
    assert list(o.has_batch([0, 1, M64, M64 - 1])) == [1, 0, 1, 0]
    s, c = o.range_map([0, 1, 0], [M64, M64, 1])
    assert list(c) == [1, 0, 1] and list(s) == [0, 0, 0]
    assert o.sum() == M64
    assert o.delete_batch([0, M64, 5]) == 2
    _, used, head = o.layout()
    assert list(used) == [0] and list(head) == [M64]
    assert o.check() == 0


def test_scenario_empty_leaf_in_the_middle():
    # With zero lower bounds (rho = 0) a leaf may stay empty.  Deleting all of
    # leaf 2 (4i for i in [195, 296)) leaves it empty and within bounds, so it
    # is rewritten in place with used 0; its head-index entry becomes the head
    # of the next non-empty leaf (1184).  Key 1000 then routes to leaf 1 (the
    # last entry <= 1000 is 376), whose last element 776 gives a delta of 224
    # (two bytes): leaf 1 grows from 108 to 110 bytes.
    o = oracle.SeqCPMA([4 * i for i in range(600)], leaf_bytes=256,
                       tau_leaf=900, tau_root=700, rho_leaf=0, rho_root=0)
    assert o.delete_batch([4 * i for i in range(195, 296)]) == 101
    assert o.last_batch() == dict(resized=0, nwindows=0, touched=1)
    _, used, head = o.layout()
    assert list(used) == [101, 108, 0, 108, 108, 109]
    assert list(head) == [0, 376, 1184, 1184, 1588, 1992]
    assert o.insert_batch([1000]) == 1
    _, used, head = o.layout()
    assert list(used) == [101, 110, 0, 108, 108, 109]
    assert list(head) == [0, 376, 1184, 1184, 1588, 1992]
    assert o.check() == 0


# --------------------------------------------------------------------------
# set semantics by brute force against Python sets
# --------------------------------------------------------------------------

def _brute_range(S, lo, hi):
    sel = [x for x in S if lo <= x < hi]
    return sum(sel) & M64, len(sel)


@pytest.mark.parametrize("LB", [256, 512, 1024, 2048])
def test_plainset_and_seqcpma_vs_python_sets(LB):
    rng = random.Random(LB)
    pyset = set()
    base = [rng.getrandbits(20) for _ in range(3000)] + [0, M64]
    pyset.update(base)
    plain = oracle.PlainSet(base)
    seq = oracle.SeqCPMA(base, leaf_bytes=LB, **CFG)
    for step in range(40):
        k = rng.choice([1, 5, 100, 1500, 6000])
        if rng.random() < 0.55:
            keys = [rng.getrandbits(rng.choice([20, 22, 64])) for _ in range(k)]
            keys += keys[: k // 4]  # repeats
            want = len(set(keys) - pyset)
            pyset.update(keys)
            assert plain.insert_batch(keys) == want
            assert seq.insert_batch(keys) == want
        else:
            present = sorted(pyset)
            keys = [present[rng.randrange(len(present))] for _ in range(min(k, len(present)))] \
                if present else []
            keys += [rng.getrandbits(20) for _ in range(k // 3)]
            want = len(set(keys) & pyset)
            pyset.difference_update(keys)
            assert plain.delete_batch(keys) == want
            assert seq.delete_batch(keys) == want
        S = sorted(pyset)
        assert plain.S.tolist() == S
        assert seq.elements().tolist() == S
        assert seq.size() == len(S)
        assert seq.check() == 0
        if step % 8 == 0:
            q = [rng.getrandbits(20) for _ in range(50)] + S[:5] + [M64, 0]
            want_has = [int(x in pyset) for x in q]
            assert plain.has_batch(q).tolist() == want_has
            assert seq.has_batch(q).tolist() == want_has
            lo = [rng.getrandbits(20) for _ in range(30)] + [0, 5, M64]
            hi = [x + rng.getrandbits(rng.choice([4, 12, 19])) for x in lo[:30]] + [M64, 5, M64]
            hi = [min(h, M64) for h in hi]
            ws = [_brute_range(S, a, b) for a, b in zip(lo, hi)]
            for impl in (plain, seq):
                s, c = impl.range_map(lo, hi)
                assert [(int(x), int(y)) for x, y in zip(s, c)] == ws
            assert seq.sum() == sum(S) & M64


def test_seqcpma_delete_everything_and_rebuild():
    keys = list(range(0, 40000, 3))
    o = oracle.SeqCPMA(keys, leaf_bytes=256, **CFG)
    assert o.delete_batch(keys) == len(keys)
    assert o.size() == 0 and o.leaves() == 1 and o.check() == 0
    assert o.insert_batch(keys) == len(keys)
    assert o.elements().tolist() == keys and o.check() == 0


def test_seqcpma_windows_are_maximal_dyadic_nodes():
    # Skewed inserts force many windows; every reported window must be a node
    # of the implicit tree (aligned, power-of-two or clipped at L) and no
    # window may contain another.
    rng = np.random.default_rng(11)
    base = W.uniform_keys(5, 200000, bits=40)
    o = oracle.SeqCPMA(base, leaf_bytes=256, **CFG)
    seen = 0
    for r in range(6):
        keys = W.zipf_keys(100 + r, 20000, bits=34)
        L = o.leaves()
        o.insert_batch(keys)
        assert o.check() == 0
        if o.last_batch()["resized"]:
            continue
        wins = o.last_windows()
        seen += len(wins)
        for a, w in wins:
            a, w = int(a), int(w)
            h = max(0, (w - 1).bit_length())
            assert a % (1 << h) == 0
            assert w == (1 << h) or a + w == L
        iv = sorted((int(a), int(a + w)) for a, w in wins)
        for (a0, a1), (b0, b1) in zip(iv, iv[1:]):
            assert a1 <= b0
    assert seen > 0


def test_bytes_per_key_sanity_band():
    # Not a pin: Table size-micro reports 4.77 bytes/element for the CPMA at
    # 1e6 uniform 40-bit keys; a fresh build at density 0.5 with 512-byte
    # leaves lands in the same few-bytes band.
    o = oracle.SeqCPMA(W.uniform_keys(9, 10 ** 6), leaf_bytes=512, **CFG)
    bpk = o.bytes() / o.size()
    assert 3.0 < bpk < 8.0


# --------------------------------------------------------------------------
# map_range_length and filtered range reductions, by brute force
# --------------------------------------------------------------------------

def test_range_length_brute_force():
    """App. A map_range_length(start, length): the function sees at most
    `length` elements, the first ones with key >= start."""
    rng = random.Random(7)
    S = sorted(set(rng.getrandbits(16) for _ in range(2000)) | {0, M64, M64 - 1})
    plain = oracle.PlainSet(S)
    starts = [rng.getrandbits(16) for _ in range(200)] + [0, 1, M64, M64 - 1, S[-3], S[5]]
    lens = [rng.choice([0, 1, 2, 7, 100, 5000, M64]) for _ in range(200)] + [3, M64, 1, 5, 2, 0]
    want = []
    for a, ln in zip(starts, lens):
        sel = [x for x in S if x >= a][: min(ln, len(S))]
        want.append((sum(sel) & M64, len(sel)))
    s, c = plain.range_map_length(starts, lens)
    assert [(int(x), int(y)) for x, y in zip(s, c)] == want
    # length 1 gives the successor (the PMA search of Sec. 3)
    s, c = plain.range_map_length([S[10] + 1], [1])
    assert int(c[0]) == 1 and int(s[0]) == S[11]
    # everything: the sum of the whole set
    s, c = plain.range_map_length([0], [M64])
    assert int(s[0]) == sum(S) & M64 and int(c[0]) == len(S)


@pytest.mark.parametrize("op", ["sum", "min", "max", "xor"])
def test_range_reduce_brute_force(op):
    rng = random.Random(11)
    S = sorted(set(rng.getrandbits(18) for _ in range(3000)) | {0, M64 - 1})
    plain = oracle.PlainSet(S)
    lo = [rng.getrandbits(18) for _ in range(120)] + [0, 0, 9, M64]
    hi = [a + rng.getrandbits(rng.choice([3, 10, 17])) for a in lo[:120]] + [M64, 1, 9, M64]
    for mask, value in [(0, 0), (1, 1), (0xF, 0x5), (1 << 17, 0)]:
        want = []
        for a, b in zip(lo, hi):
            sel = [x for x in S if a <= x < b and (x & mask) == value]
            if op == "sum":
                r = sum(sel) & M64
            elif op == "min":
                r = min(sel) if sel else M64
            elif op == "max":
                r = max(sel) if sel else 0
            else:
                r = 0
                for x in sel:
                    r ^= x
            want.append((r, len(sel)))
        r, c = plain.range_reduce(lo, hi, op, mask, value)
        assert [(int(x), int(y)) for x, y in zip(r, c)] == want
    # the unfiltered sum is range_map
    r, c = plain.range_reduce(lo, hi, "sum")
    s2, c2 = plain.range_map(lo, hi)
    assert np.array_equal(r, s2) and np.array_equal(c, c2)


def test_max_key_routes_to_last_nonempty_leaf():
    """With low lower bounds a sparse window at the end of the array can be
    redistributed so that its last leaf stays empty; every head-index entry is
    <= 2^64-1, so that key must route to the last non-empty leaf, not to the
    empty leaf after it (reading R5).  Found by comparing with the plain set."""
    keys = np.array([4 * i for i in range(3000)] + [M64], dtype=np.uint64)
    o = oracle.SeqCPMA(keys, leaf_bytes=256, tau_leaf=900, tau_root=700, rho_leaf=5,
                       rho_root=20)
    p = oracle.PlainSet(keys)
    dele = keys[2400:-1]
    assert o.delete_batch(dele) == p.delete_batch(dele)
    _, used, _ = o.layout()
    assert used[-1] == 0 and used[-2] > 0  # an empty leaf after the one holding 2^64-1
    q = np.array([M64, M64 - 1, 0, 4 * 2399], dtype=np.uint64)
    assert o.has_batch(q).tolist() == p.has_batch(q).tolist() == [1, 0, 1, 1]
    assert o.insert_batch([M64]) == p.insert_batch([M64]) == 0
    assert o.insert_batch([M64 - 1]) == p.insert_batch([M64 - 1]) == 1
    assert o.elements().tolist() == p.S.tolist()
    s, c = o.range_map([M64 - 1], [M64])
    assert int(s[0]) == M64 - 1 and int(c[0]) == 1
    assert o.check() == 0


def test_rebuild_rule():
    """R14: a batch with 1000 k >= rebuild_pm n is applied by rebuilding: the
    set is the plain union / difference and the layout is exactly the
    constructor's over the new set; a batch just below the threshold takes
    the merge path (same layout as rebuild_pm = 0)."""
    rng = random.Random(3)
    base = [rng.getrandbits(30) for _ in range(20000)]
    n = len(set(base))
    for is_del in (False, True):
        o = oracle.SeqCPMA(base, leaf_bytes=256, rebuild_pm=100)
        m = oracle.SeqCPMA(base, leaf_bytes=256)
        p = oracle.PlainSet(base)
        k_lo = (100 * n - 1) // 1000  # 1000 k < 100 n: merge
        keys = sorted(p.S.tolist())[:k_lo] if is_del else [rng.getrandbits(30) for _ in range(k_lo)]
        f = "delete_batch" if is_del else "insert_batch"
        assert getattr(o, f)(keys) == getattr(m, f)(keys) == getattr(p, f)(keys)
        assert o.last_batch()["resized"] == m.last_batch()["resized"]
        for a, b in zip(o.layout(), m.layout()):
            assert np.array_equal(a, b)
        n2 = len(p)
        k_hi = -(-100 * n2 // 1000)  # ceil: 1000 k >= 100 n: rebuild
        keys = p.S.tolist()[::2][:k_hi] if is_del else [rng.getrandbits(30) for _ in range(k_hi)]
        assert getattr(o, f)(keys) == getattr(p, f)(keys)
        assert o.elements().tolist() == p.S.tolist()
        fresh = oracle.SeqCPMA(p.S, leaf_bytes=256)
        for a, b in zip(o.layout(), fresh.layout()):
            assert np.array_equal(a, b)
        assert o.leaves() == fresh.leaves() and o.bytes() == fresh.bytes()
        assert o.check() == 0
    # an empty set always rebuilds (n = 0), into the constructor's layout
    e = oracle.SeqCPMA([], leaf_bytes=512, rebuild_pm=100)
    assert e.insert_batch(base) == n
    for a, b in zip(e.layout(), oracle.SeqCPMA(base, leaf_bytes=512).layout()):
        assert np.array_equal(a, b)


def test_range_extract_brute_force():
    """range_map emitting the keys (offsets + packed keys) against a Python
    filter; empty and inverted ranges, ranges past the ends."""
    rng = random.Random(21)
    S = sorted(set(rng.getrandbits(14) for _ in range(3000)) | {0, M64})
    plain = oracle.PlainSet(S)
    lo = [rng.getrandbits(14) for _ in range(100)] + [0, 5, M64, 9, M64 - 1]
    hi = [a + rng.getrandbits(rng.choice([2, 8, 13])) for a in lo[:100]] + [M64, 5, M64, 3, M64]
    off, keys = plain.range_extract(lo, hi)
    want = [[x for x in S if a <= x < b] for a, b in zip(lo, hi)]
    assert off.tolist() == [0] + list(np.cumsum([len(w) for w in want]))
    assert keys.tolist() == [x for w in want for x in w]


def test_rmat_generator_shape():
    """R-MAT edges stay inside 2^scale vertices and are skewed: the busiest
    source has far more edges than the average."""
    from paper_2305_05055_gb300 import workloads as W
    src, dst = W.rmat_edges(3, 12, 50000)
    assert src.max() < 4096 and dst.max() < 4096
    assert np.array_equal(W.rmat_edges(3, 12, 50000)[0], src)  # seeded
    deg = np.bincount(src.astype(np.int64), minlength=4096)
    assert deg.max() > 20 * deg.mean()


# --------------------------------------------------------------------------
# uncompressed PMA (reading R16): 8-byte cells, same batch algorithm
# --------------------------------------------------------------------------

def test_raw_cells_are_little_endian_values():
    e = np.array([5, 300, 1 << 40, M64 - 1], dtype=np.uint64)
    buf = np.zeros(64, dtype=np.uint8)
    used = oracle.lib().o_raw_leaf_encode(buf, 64, e, e.size)
    assert used == 32
    want = b"".join(int(x).to_bytes(8, "little") for x in e.tolist())
    assert bytes(buf[:32]) == want and not buf[32:].any()
    out = np.zeros(8, dtype=np.uint64)
    assert oracle.lib().o_raw_leaf_decode(buf, used, out) == 4
    assert out[:4].tolist() == e.tolist()


def test_pma_build_by_hand():
    """40 keys, LB 256, build density 500: S = 40 * 8 = 320 bytes, L =
    ceil(1000 * 320 / (500 * 256 - 8000)) = ceil(2.67) = 3.  Element costs
    are all 8, so leaf w starts at the first i with 8 i >= floor(w * 320 / 3):
    i = 14 (>= 106) and i = 27 (>= 213); leaves hold 14, 13, 13 elements.
    An insert into leaf 1 (well within 0.9 * 256 bytes) rewrites it in
    place with 14 cells."""
    keys = [10 * i + 3 for i in range(40)]
    o = oracle.SeqCPMA(keys, leaf_bytes=256, codec=1)
    data, used, head = o.layout()
    assert list(used) == [112, 104, 104]
    assert list(head) == [keys[0], keys[14], keys[27]]
    raw = b"".join(int(x).to_bytes(8, "little") for x in keys[14:27])
    assert bytes(data[256:256 + 104]) == raw
    assert o.insert_batch([145]) == 1  # between 143 (keys[14]) and 153
    data, used, head = o.layout()
    assert list(used) == [112, 112, 104]
    cells = sorted(keys[14:27] + [145])
    assert bytes(data[256:256 + 112]) == b"".join(int(x).to_bytes(8, "little") for x in cells)
    assert o.check() == 0


@pytest.mark.parametrize("LB", [256, 1024])
def test_pma_vs_plain_set(LB):
    rng = random.Random(LB + 7)
    base = [rng.getrandbits(24) for _ in range(4000)] + [0, M64]
    o = oracle.SeqCPMA(base, leaf_bytes=LB, codec=1)
    p = oracle.PlainSet(base)
    for step in range(30):
        if rng.random() < 0.6:
            keys = [rng.getrandbits(rng.choice([24, 64])) for _ in range(rng.choice([1, 30, 2000]))]
            assert o.insert_batch(keys) == p.insert_batch(keys)
        else:
            S = p.S.tolist()
            keys = [S[rng.randrange(len(S))] for _ in range(rng.choice([1, 50, len(S) // 2]))]
            assert o.delete_batch(keys) == p.delete_batch(keys)
        assert o.elements().tolist() == p.S.tolist()
        assert o.check() == 0
    q = [rng.getrandbits(24) for _ in range(100)] + [0, M64]
    assert o.has_batch(q).tolist() == p.has_batch(q).tolist()
    lo = [rng.getrandbits(24) for _ in range(50)]
    hi = [a + rng.getrandbits(18) for a in lo]
    s1, c1 = o.range_map(lo, hi)
    s2, c2 = p.range_map(lo, hi)
    assert np.array_equal(s1, s2) and np.array_equal(c1, c2)
    # 8 bytes per key over the leaves, so more leaves than the CPMA of the same set
    cp_ = oracle.SeqCPMA(p.S, leaf_bytes=LB)
    assert o.leaves() > cp_.leaves()
