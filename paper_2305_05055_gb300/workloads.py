"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 6
"Experimental setup": 40-bit uniform keys; 34-bit zipfian keys with skew 0.99
as in YCSB; 1e5 parallel range queries over 1e8 elements).

This module holds no arithmetic of the method itself: only random-number
generation.  Both the CUDA path's tests/benchmarks and the CPU oracle are fed
from it.

* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014): output i of seed s is mix(s + (i+1) * gamma).
* Zipfian ranks by the method of Gray, Sundaresan, Englert, Baclawski and
  Weinberger, "Quickly generating billion-record synthetic databases"
  (SIGMOD 1994), the generator YCSB uses; the zeta constant of a 2^34-item
  universe is evaluated with the Euler-Maclaurin formula.
"""
from __future__ import annotations

import math

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+count-1 of the SplitMix64 stream of `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def uniform_keys(seed: int, count: int, bits: int = 40, offset: int = 0) -> np.ndarray:
    """`count` keys uniform in [0, 2^bits) (repeats possible), unsorted."""
    return splitmix64(seed, count, offset) >> np.uint64(64 - bits)


def full_range_keys(seed: int, count: int) -> np.ndarray:
    """Keys uniform over all of [0, 2^64)."""
    return splitmix64(seed, count)


def zeta(n: int, theta: float, exact_terms: int = 1 << 20) -> float:
    """sum_{i=1..n} i^-theta: exact for the first terms, Euler-Maclaurin for
    the tail (integral, endpoint and first derivative corrections)."""
    m = min(n, exact_terms)
    head = float(np.sum(np.arange(1, m + 1, dtype=np.float64) ** (-theta)))
    if n <= m:
        return head
    a, b = float(m + 1), float(n)
    f = lambda x: x ** (-theta)
    df = lambda x: -theta * x ** (-theta - 1.0)
    integral = (b ** (1.0 - theta) - a ** (1.0 - theta)) / (1.0 - theta)
    return head + integral + 0.5 * (f(a) + f(b)) + (df(b) - df(a)) / 12.0


class Zipf:
    """Zipfian ranks in [0, n) with skew theta (rank 0 most popular)."""

    def __init__(self, n: int, theta: float = 0.99):
        self.n, self.theta = n, theta
        self.zetan = zeta(n, theta)
        zeta2 = 1.0 + 2.0 ** (-theta)
        self.alpha = 1.0 / (1.0 - theta)
        self.eta = (1.0 - (2.0 / n) ** (1.0 - theta)) / (1.0 - zeta2 / self.zetan)

    def ranks(self, seed: int, count: int, offset: int = 0) -> np.ndarray:
        u = uniform01(seed, count, offset)
        uz = u * self.zetan
        r = np.floor(self.n * np.power(self.eta * u - self.eta + 1.0, self.alpha))
        r = np.clip(r, 0, self.n - 1).astype(np.uint64)
        r = np.where(uz < 1.0 + 0.5 ** self.theta, np.uint64(1), r)
        r = np.where(uz < 1.0, np.uint64(0), r)
        return r


def mix_bits(x: np.ndarray, bits: int, seed: int) -> np.ndarray:
    """A seeded bijection on [0, 2^bits): odd multiply, xorshift, odd
    multiply, xorshift, all mod 2^bits."""
    mask = np.uint64((1 << bits) - 1)
    k1 = np.uint64(int(splitmix64(seed, 1)[0]) | 1)
    k2 = np.uint64(int(splitmix64(seed, 1, 1)[0]) | 1)
    s = np.uint64(bits // 2)
    with np.errstate(over="ignore"):
        x = (x.astype(np.uint64) * k1) & mask
        x = x ^ (x >> s)
        x = (x * k2) & mask
        x = x ^ (x >> s)
    return x


def zipf_keys(seed: int, count: int, bits: int = 34, theta: float = 0.99,
              offset: int = 0, _cache={}) -> np.ndarray:
    """Zipfian keys over [0, 2^bits): rank drawn by Gray et al., then mapped
    to a key by a seeded bijection so that hot keys are scattered."""
    z = _cache.get((bits, theta))
    if z is None:
        z = _cache[(bits, theta)] = Zipf(1 << bits, theta)
    return mix_bits(z.ranks(seed, count, offset), bits, seed ^ 0x5A5A)


def sample_present(sorted_keys: np.ndarray, seed: int, count: int) -> np.ndarray:
    """`count` distinct keys drawn without replacement from a sorted set."""
    n = sorted_keys.size
    count = min(count, n)
    if count == 0:
        return np.zeros(0, dtype=np.uint64)
    # partial Fisher-Yates driven by SplitMix64
    r = splitmix64(seed, count)
    idx = np.arange(n, dtype=np.int64) if n <= 4 * count else None
    if idx is not None:
        for i in range(count):
            j = i + int(r[i] % np.uint64(n - i))
            idx[i], idx[j] = idx[j], idx[i]
        return sorted_keys[idx[:count]].copy()
    chosen = {}
    out = np.empty(count, dtype=np.int64)
    for i in range(count):
        j = i + int(r[i] % np.uint64(n - i))
        vi, vj = chosen.get(i, i), chosen.get(j, j)
        out[i] = vj
        chosen[j] = vi
    return sorted_keys[out].copy()


def permuted_indices(n: int, count: int, seed: int, offset: int = 0) -> np.ndarray:
    """Indices offset..offset+count-1 of a seeded permutation of [0, n):
    i -> (a*i + b) mod n with a odd-ish and coprime to n (distinct indices)."""
    a = int(splitmix64(seed, 1)[0] % np.uint64(max(n, 1))) | 1
    while math.gcd(a, n) != 1:
        a += 2
    b = int(splitmix64(seed, 1, 1)[0] % np.uint64(max(n, 1)))
    if n >= (1 << 32) or offset + count >= (1 << 32):
        return np.array([(a * v + b) % n for v in range(offset, offset + count)], dtype=np.int64)
    i = np.arange(offset, offset + count, dtype=np.uint64)
    return ((i * np.uint64(a) % np.uint64(n) + np.uint64(b)) % np.uint64(n)).astype(np.int64)


def range_queries_fixed_width(seed: int, count: int, width: int, bits: int = 40):
    """[lo, lo + width) with lo uniform in [0, 2^bits)."""
    lo = uniform_keys(seed, count, bits)
    return lo, lo + np.uint64(width)


def range_queries_by_rank(sorted_keys: np.ndarray, seed: int, count: int,
                          min_elems: int = 10, max_elems: int = 10 ** 6):
    """Queries covering an exact number of elements c = floor(10^U(log10 min,
    log10 max)): lo = key[r], hi = key[r + c] (2^64-1 past the end)."""
    n = sorted_keys.size
    r = (splitmix64(seed, count) % np.uint64(max(n, 1))).astype(np.int64)
    u = uniform01(seed ^ 0xABCDEF, count)
    a, b = math.log10(min_elems), math.log10(max_elems)
    c = np.floor(10.0 ** (a + (b - a) * u)).astype(np.int64)
    lo = sorted_keys[np.minimum(r, n - 1)] if n else np.zeros(count, np.uint64)
    j = r + c
    hi = np.where(j < n, sorted_keys[np.minimum(j, n - 1)] if n else 0,
                  np.uint64(0xFFFFFFFFFFFFFFFF)).astype(np.uint64)
    return lo.astype(np.uint64), hi, c


def log_uniform_int(seed: int, count: int, lo: int, hi: int) -> np.ndarray:
    """Integers floor(10^U(log10 lo, log10 hi + 1)) clipped to [lo, hi]."""
    u = uniform01(seed, count)
    a, b = math.log10(lo), math.log10(hi + 1)
    return np.clip(np.floor(10.0 ** (a + (b - a) * u)), lo, hi).astype(np.int64)


def rmat_edges(seed: int, scale: int, count: int, a: float = 0.57, b: float = 0.19,
               c: float = 0.19, offset: int = 0):
    """`count` directed edges of an R-MAT graph on 2^scale vertices
    (Chakrabarti, Zhan, Faloutsos, "R-MAT: A recursive model for graph
    mining", SDM 2004; Graph500 probabilities a = 0.57, b = c = 0.19): each
    of the `scale` bit levels picks a quadrant with probabilities a, b, c,
    1 - a - b - c.  Vertex ids are then scattered by a seeded bijection so
    that high-degree vertices are not the small ids.  Returns (src, dst)
    uint64 arrays; repeats and self loops are kept (an edge set drops
    repeats)."""
    if not 1 <= scale <= 31:
        raise ValueError("scale must be in [1, 31]")
    src = np.zeros(count, dtype=np.uint64)
    dst = np.zeros(count, dtype=np.uint64)
    for level in range(scale):
        u = uniform01(seed * 64 + level, count, offset)
        right = (u >= a) & (u < a + b) | (u >= a + b + c)   # dst bit
        down = u >= a + b                                     # src bit
        src = (src << np.uint64(1)) | down.astype(np.uint64)
        dst = (dst << np.uint64(1)) | right.astype(np.uint64)
    return mix_bits(src, scale, seed ^ 0x1234), mix_bits(dst, scale, seed ^ 0x1234)
