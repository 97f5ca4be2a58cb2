"""Host build of the thread-granular leaf insert and delete (the code the
GPU kernel k_insert_thread runs per leaf, for deletes as k_insert_thread<true>) against the
oracle's leaf encoder: inserting (deleting) a slice of at most four keys
must give exactly the bytes of encoding the union (difference) from scratch
(Sec. 5 leaf format, zero bytes after the used ones), the right count, head
and changed-key mask, and must leave the leaf untouched when the result does
not fit or the leaf holds a code longer than 4 bytes.  Every access outside the leaf's
LB bytes faults (guard pages)."""
import ctypes as C
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
M64 = (1 << 64) - 1
UNCHANGED, WRITTEN, TOO_BIG, LONG_CODE = range(4)


@pytest.fixture(scope="module")
def lt(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("lt") / "liblt.so")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", "-o", out,
                    os.path.join(HERE, "leaf_thread_host.cu")], check=True)
    lib = C.CDLL(out)
    lib.lt_insert.restype = C.c_int
    return lib


def encode(keys, LB):
    buf, used = oracle.leaf_encode(np.array(keys, dtype=np.uint64), LB)
    return bytes(buf[:used])


def run(lib, keys, sl, LB, guard_after, delete=False):
    enc = encode(keys, LB)
    leaf = bytearray(LB)
    leaf[:len(enc)] = enc
    buf = (C.c_uint8 * LB).from_buffer(leaf)
    ks = (C.c_uint64 * 4)(*sl)
    out = (C.c_uint32 * 8)()
    st = lib.lt_insert(buf, LB, len(enc), len(keys), ks, len(sl), out, guard_after, int(delete))
    return st, bytes(leaf), list(out), enc


def check(lib, keys, sl, LB, guard_after):
    st, leaf, out, enc = run(lib, keys, sl, LB, guard_after)
    old = set(keys)
    if any(oracle.leb_len(b - a) > 4 for a, b in zip(keys, keys[1:])):
        # a code of more than 4 bytes: nothing written
        assert st == LONG_CODE and leaf[:len(enc)] == enc
        return st
    new = sorted(old | set(sl))
    added = 0
    for q, x in enumerate(sl):
        if x not in old and (q == 0 or sl[q - 1] != x):
            added |= 1 << q
    if added == 0:
        assert st == UNCHANGED and leaf[:len(enc)] == enc
        return st
    nb = oracle.leaf_bytes(np.array(new, dtype=np.uint64))
    assert out[0] == nb and out[1] == len(new) and out[2] == added
    assert out[5] | (out[6] << 32) == new[0]
    if nb > LB:
        assert st == TOO_BIG and leaf[:len(enc)] == enc
        return st
    assert st == WRITTEN
    assert leaf[:nb] == encode(new, LB) and not any(leaf[nb:])
    return st


def leaf_keys(rng, LB):
    mode = rng.random()
    n = rng.randint(1, 300)
    if mode < 0.1:   # deltas at the code-length boundaries (a split may not grow the leaf)
        base = rng.randrange(0, 1 << 64)
        keys = sorted({(base + i * rng.choice([1, 127, 128, 129, 16383, 16384])) & M64
                       for i in range(n)})
    else:
        bits = rng.choice([7, 8, 14, 15, 21, 22, 28, 29, 40, 64])
        keys = sorted({rng.randrange(0, 1 << bits) for _ in range(n)})
    if rng.random() < 0.05:
        keys = sorted(set(keys) | {M64})
    if rng.random() < 0.05:
        keys = sorted(set(keys) | {0})
    while oracle.leaf_bytes(np.array(keys, dtype=np.uint64)) > LB:
        keys = keys[:len(keys) * 3 // 4]
    return keys


def slice_keys(rng, keys):
    sl = []
    for _ in range(rng.randint(1, 4)):
        r = rng.random()
        if r < 0.15:
            sl.append(rng.choice(keys))                                   # present
        elif r < 0.25:
            sl.append(max(0, keys[0] - rng.randint(1, 1000)))             # new head
        elif r < 0.35:
            sl.append(min(M64, keys[-1] + rng.randint(1, 1 << rng.choice([3, 7, 14, 30]))))
        elif r < 0.5 and len(keys) > 1:                                   # inside a gap
            i = rng.randrange(len(keys) - 1)
            sl.append(rng.randrange(keys[i] + 1, keys[i + 1]) if keys[i + 1] - keys[i] > 1
                      else keys[i])
        else:
            sl.append(rng.randrange(keys[0], keys[-1] + 1))
    if rng.random() < 0.2:
        sl.append(sl[-1])                                                 # repeat
    return sorted(sl)[:4]


def test_leaf_thread_random(lt):
    rng = random.Random(20240531)
    seen = set()
    for it in range(4000):
        LB = rng.choice([256, 512, 1024, 2048])
        keys = leaf_keys(rng, LB)
        if keys:
            seen.add(check(lt, keys, slice_keys(rng, keys), LB, it & 1))
    assert seen == {UNCHANGED, WRITTEN, TOO_BIG, LONG_CODE}


def test_leaf_thread_cases(lt):
    # one element, insert before / after it; the head replaced by a smaller key
    assert check(lt, [1000], [5], 256, 0) == WRITTEN
    assert check(lt, [1000], [1000, 1001], 256, 1) == WRITTEN
    assert check(lt, [M64 - 5, M64 - 1], [M64], 256, 0) == WRITTEN
    assert check(lt, [0, M64 - 1], [M64], 256, 1) == LONG_CODE
    # a split that keeps the size (127 + 1 = 128: 1 + 1 bytes replace 2)
    assert check(lt, [0, 128], [127], 256, 1) == WRITTEN
    # the largest key as the last element: present, and with a key before it
    assert check(lt, [M64 - 300, M64], [M64], 256, 0) == UNCHANGED
    assert check(lt, [M64 - 300, M64], [M64 - 1, M64, M64], 256, 1) == WRITTEN
    # keys in the first chunk (the head's) and in a code straddling two chunks
    assert check(lt, [100, 200, 300], [150, 250], 256, 0) == WRITTEN
    assert check(lt, [0] + [i * 16384 for i in range(1, 12)], [16385, 5 * 16384 + 7], 256, 1) == WRITTEN
    # all present, repeats only
    assert check(lt, [3, 9, 27], [3, 3, 27, 27], 256, 0) == UNCHANGED
    # four keys in one gap, then a full leaf that no longer fits
    assert check(lt, [10, 1 << 20], [11, 12, 13, 14], 256, 1) == WRITTEN
    full = list(range(0, 2 * 247, 2))          # 8 + 246 one-byte codes = 254 bytes
    assert check(lt, full, [1, 3, 5], 256, 0) == TOO_BIG


def check_delete(lib, keys, sl, LB, guard_after):
    st, leaf, out, enc = run(lib, keys, sl, LB, guard_after, delete=True)
    old = set(keys)
    if any(oracle.leb_len(b - a) > 4 for a, b in zip(keys, keys[1:])):
        # a code of more than 4 bytes: nothing written
        assert st == LONG_CODE and leaf[:len(enc)] == enc
        return st
    new = sorted(old - set(sl))
    removed = 0
    for q, x in enumerate(sl):
        if x in old and (q == 0 or sl[q - 1] != x):
            removed |= 1 << q
    if removed == 0:
        assert st == UNCHANGED and leaf[:len(enc)] == enc
        return st
    assert st == WRITTEN
    nb = oracle.leaf_bytes(np.array(new, dtype=np.uint64)) if new else 0
    assert out[0] == nb and out[1] == len(new) and out[2] == removed
    assert out[5] | (out[6] << 32) == (new[0] if new else M64)
    assert leaf[:nb] == (encode(new, LB) if new else b"") and not any(leaf[nb:])
    return st


def test_leaf_thread_delete_random(lt):
    rng = random.Random(20240601)
    seen = set()
    for it in range(4000):
        LB = rng.choice([256, 512, 1024, 2048])
        keys = leaf_keys(rng, LB)
        if not keys:
            continue
        r = rng.random()
        if r < 0.5:     # present keys, often neighbours, with absent ones between
            i = rng.randrange(len(keys))
            sl = [keys[min(len(keys) - 1, i + d)] for d in range(rng.randint(1, 4))]
            for q in range(len(sl) - 1):
                if rng.random() < 0.3 and sl[q + 1] - sl[q] > 1:
                    sl.append(rng.randrange(sl[q] + 1, sl[q + 1]))
        elif r < 0.6:   # the head and the last elements
            sl = keys[:rng.randint(1, 4)] if rng.random() < 0.5 else keys[-rng.randint(1, 4):]
        else:
            sl = slice_keys(rng, keys)
        if rng.random() < 0.2:
            sl = sl + [sl[-1]]
        seen.add(check_delete(lt, keys, sorted(sl)[:4], LB, it & 1))
    assert seen == {UNCHANGED, WRITTEN, LONG_CODE}


def test_leaf_thread_delete_cases(lt):
    assert check_delete(lt, [1000], [1000], 256, 0) == WRITTEN               # the only element
    assert check_delete(lt, [5, 6, 7], [5, 6, 7], 256, 1) == WRITTEN         # all of them
    assert check_delete(lt, [5, 6, 7], [5, 5], 256, 0) == WRITTEN            # the head, repeated
    assert check_delete(lt, [5, 6, 7], [7], 256, 1) == WRITTEN               # the last one
    assert check_delete(lt, [0, 127, 128, 300], [127], 256, 0) == WRITTEN    # merged code keeps size
    assert check_delete(lt, [0, 127, 128, 300], [1, 129], 256, 1) == UNCHANGED
    assert check_delete(lt, list(range(0, 2 * 247, 2)), [2, 4, 6, 8], 256, 0) == WRITTEN
    # absent keys between deleted neighbours: still one run
    assert check_delete(lt, [10, 20, 30, 40], [20, 25, 30], 256, 1) == WRITTEN
    assert check_delete(lt, [10, 20, 30, 40], [10, 15, 20, 25], 256, 0) == WRITTEN
    assert check_delete(lt, [10, 20, 30, 40], [30, 35, 40, 45], 256, 1) == WRITTEN
