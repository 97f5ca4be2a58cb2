"""Sorted-set helpers for building expected values in tests: sort, then a
mask of first occurrences (numpy's unique is slow on 1e7+ uint64 arrays)."""
import numpy as np


def sorted_unique(a) -> np.ndarray:
    s = np.sort(np.asarray(a, dtype=np.uint64))
    if s.size == 0:
        return s
    m = np.empty(s.size, dtype=bool)
    m[0] = True
    np.not_equal(s[1:], s[:-1], out=m[1:])
    return s[m]


def member(x, S) -> np.ndarray:
    """x in S for a sorted S, by binary search."""
    x = np.asarray(x, dtype=np.uint64)
    if S.size == 0:
        return np.zeros(x.size, dtype=bool)
    i = np.searchsorted(S, x, side="left")
    return (i < S.size) & (S[np.minimum(i, S.size - 1)] == x)


def union(S, U) -> np.ndarray:
    """Sorted S with the keys of U added (U need not be sorted or distinct)."""
    U = sorted_unique(U)
    new = U[~member(U, S)]
    return np.insert(S, np.searchsorted(S, new), new)
