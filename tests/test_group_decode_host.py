"""Host check of the arithmetic the thread-per-leaf decoders use (the leaf sum
of range_map / sum and the membership test of has_batch): the leaf's codes
are taken eight bytes at a time with a 32-bit accumulator that is not
cleared at terminators, so the element closed at the k-th terminator of a
group is val + acc_k.  A group adds T * val + sum_k acc_k to the 64-bit leaf
sum; a membership test compares acc_k with x - val.  Both are exact while
every code has at most 4 bytes (Sec. 5 byte codes: deltas below 2^28), which
needs sum_k acc_k < 2^32; a leaf with a longer code must be flagged (the OR
of the per-byte multipliers reaches 2^28) and decoded exactly instead.

The emulation below follows the kernel's steps with 32-bit wrap-around; the
leaves come from the oracle's encoder and the expected values are the plain
sum and set membership of the encoded keys."""
import random

import numpy as np

import oracle

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1


def group_sum(bs, st):
    val, s, acc, pw, pwor = st
    ss = r = 0
    for c in bs:
        acc = (acc + (c & 0x7F) * pw) & M32
        term = not (c & 0x80)
        pwor |= pw
        if term:
            ss = (ss + acc) & M32
            r = acc
        pw = 1 if term else (pw << 7) & M32
    t = sum(1 for c in bs if not c & 0x80)
    return [(val + r) & M64, (s + t * val + ss) & M64, (acc - r) & M32, pw, pwor]


def leaf_sum(buf, u):
    """Sum of the leaf's elements as the thread leaf sum computes it, and
    whether the leaf was flagged for the exact decoder."""
    b = [int(v) for v in buf[:u]] + [0] * 48
    val = int.from_bytes(bytes(b[:8]), "little")
    st = [val, val, 0, 1, 0]
    for p0 in range(0, u, 16):
        if p0:
            st = group_sum(b[p0:p0 + 8], st)
        st = group_sum(b[p0 + 8:p0 + 16], st)
    val, s, _, _, pwor = st
    s = (s - (((u + 15) & ~15) - u) * val) & M64  # the zero bytes after u
    return s, pwor >= (1 << 28)


def leaf_has(buf, u, x):
    b = [int(v) for v in buf[:u]] + [0] * 32
    val = int.from_bytes(bytes(b[:8]), "little")
    if x <= val:
        return x == val, False
    found, acc, pw, pwor = False, 0, 1, 0
    p0 = 0
    while p0 < u and val < x:
        w = [b[p0 + i] if p0 + i < u else 0 for i in range(16)]
        for g in ((w[8:],) if p0 == 0 else (w[:8], w[8:])):
            dx = (x - val) & M64
            d32 = M32 if dx > M32 else dx
            r = 0
            for c in g:
                acc = (acc + (c & 0x7F) * pw) & M32
                term = not (c & 0x80)
                pwor |= pw
                if term and acc == d32:
                    found = True
                if term:
                    r = acc
                pw = 1 if term else (pw << 7) & M32
            val = (val + r) & M64
            acc = (acc - r) & M32
        p0 += 16
    return found, pwor >= (1 << 28)


def longest_code(keys):
    return max((oracle.leb_len(int(b) - int(a)) for a, b in zip(keys, keys[1:])), default=0)


def random_leaves(seed, count, LB=512):
    rng = random.Random(seed)
    for _ in range(count):
        bits = rng.choice([7, 8, 14, 20, 21, 22, 27, 28, 29, 30, 40, 64])
        keys = sorted({rng.randrange(1 << bits) for _ in range(rng.randint(1, 90))})
        if bits >= 28 and rng.random() < 0.3:
            # a 4-byte code closed early in a group, then one-byte codes: the
            # largest in-group sum of closed codes
            base = rng.randrange(1 << 20)
            top = base + (1 << 28) - 1 - rng.randrange(4)
            keys = [base, top] + [top + 1 + i for i in range(rng.randint(0, 40))]
        if oracle.leaf_bytes(keys) > LB:
            continue
        buf, used = oracle.leaf_encode(keys, LB)
        yield keys, buf, used


def test_in_group_sum_fits_32_bits():
    # every composition of one group: an open code carried in with g bytes,
    # then codes closed in the group, each of at most 4 bytes and at its
    # largest value; the trailing open bytes reach no terminator
    best = 0

    def walk(pos, lens, first, g):
        nonlocal best
        if lens:
            acc = ss = 0
            for n in lens:
                acc += (1 << (7 * n)) - 1
                ss += acc
            best = max(best, ss)
        for n in range(1, 5):
            inside = n - g if first else n
            if inside >= 1 and pos + inside <= 8:
                walk(pos + inside, lens + [n], False, g)

    for g in range(4):
        walk(0, [], True, g)
    assert best < 9 * (1 << 28) + (1 << 22) < (1 << 32)


def test_group_sum_matches_plain_sum():
    flagged = exact = 0
    for keys, buf, used in random_leaves(5, 2500):
        s, flag = leaf_sum(buf, used)
        assert flag == (longest_code(keys) > 4)
        if flag:
            flagged += 1
        else:
            assert s == sum(keys) & M64
            exact += 1
    assert flagged > 100 and exact > 1000


def test_group_membership_matches_set():
    rng = random.Random(9)
    checked = 0
    for keys, buf, used in random_leaves(7, 1500):
        present = set(keys)
        for _ in range(5):
            t = rng.random()
            x = rng.choice(keys)
            if t >= 0.4:
                x += rng.choice([-1, 1, 2, 1 << 32, -(1 << 32)])
            x &= M64
            found, flag = leaf_has(buf, used, x)
            if not flag:
                assert found == (x in present)
                checked += 1
    assert checked > 5000


def test_padding_terminators_are_taken_off():
    # leaves whose used bytes end at every offset inside a 16-byte chunk
    for n in range(1, 40):
        keys = list(np.cumsum([5] + [1000] * (n - 1)).astype(int))
        buf, used = oracle.leaf_encode(keys, 512)
        s, flag = leaf_sum(buf, used)
        assert not flag and s == sum(keys)
