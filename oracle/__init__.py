"""CPU oracle for the CPMA hot path (plain C, called through ctypes).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (``paper_2305_05055_gb300``) never imports it and shares no code
with it.

Two oracles (see ``cpma_oracle.c`` for the readings of the paper they take):

* :class:`PlainSet` — the plain definition of the set (Sec. 3 "Design and
  operations"; App. A API): a sorted array of distinct uint64 keys.
* :class:`SeqCPMA` — a sequential CPMA following Sec. 3-5 one batch at a time,
  used to pin the byte layout.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpma_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99 + __int128); returns the path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC",
                           "-Wall", "-o", tmp, _SRC])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            V, S = C.c_void_p, C.c_size_t
            U64, U32, I = C.c_uint64, C.c_uint32, C.c_int
            sig = {
                "oset_sort_unique": (S, [u64p, S]),
                "oset_union": (S, [u64p, S, u64p, S, u64p]),
                "oset_difference": (S, [u64p, S, u64p, S, u64p]),
                "oset_has": (I, [u64p, S, U64]),
                "oset_range": (None, [u64p, S, U64, U64, C.POINTER(U64), C.POINTER(U64)]),
                "oset_range_length": (None, [u64p, S, U64, U64, C.POINTER(U64), C.POINTER(U64)]),
                "oset_range_reduce": (None, [u64p, S, U64, U64, C.c_int, U64, U64,
                                             C.POINTER(U64), C.POINTER(U64)]),
                "o_leb_len": (C.c_uint, [U64]),
                "o_leb_put": (C.c_uint, [u8p, U64]),
                "o_leb_get": (C.c_uint, [u8p, C.POINTER(U64)]),
                "o_leaf_bytes": (U64, [u64p, S]),
                "o_leaf_encode": (U64, [u8p, U32, u64p, S]),
                "o_leaf_decode": (S, [u8p, U64, u64p]),
                "o_violates": (I, [U32, U32, U32, U32, U32, C.c_uint, C.c_uint, U64, U64]),
                "o_build_leaves": (U64, [U64, U32, U32]),
                "o_resize_leaves": (U64, [U64, U64, U32, U32, U32, U32, U32]),
                "o_cut_points": (None, [u64p, S, U64, u64p]),
                "ocpma_create": (I, [C.POINTER(V), U32, U32, U32, U32, U32, U32, U32, U32, U32,
                                     U32, u64p, U64]),
                "ocpma_leaf_bytes": (U32, [V]),
                "o_leaf_size": (U32, [U64, U32, U32]),
                "o_raw_leaf_encode": (U64, [u8p, U32, u64p, S]),
                "o_raw_leaf_decode": (S, [u8p, U64, u64p]),
                "ocpma_destroy": (None, [V]),
                "ocpma_set_rebuild": (None, [V, U32]),
                "ocpma_insert": (I, [V, u64p, U64, C.POINTER(U64)]),
                "ocpma_delete": (I, [V, u64p, U64, C.POINTER(U64)]),
                "ocpma_has": (I, [V, U64]),
                "ocpma_range": (None, [V, U64, U64, C.POINTER(U64), C.POINTER(U64)]),
                "ocpma_sum": (U64, [V]),
                "ocpma_size": (U64, [V]),
                "ocpma_leaves": (U64, [V]),
                "ocpma_bytes": (U64, [V]),
                "ocpma_elements": (U64, [V, u64p]),
                "ocpma_layout": (None, [V, u8p, u32p, u64p]),
                "ocpma_last_batch": (None, [V, C.POINTER(U64), C.POINTER(U64), C.POINTER(U64)]),
                "ocpma_last_windows": (None, [V, u64p]),
                "ocpma_check": (I, [V]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# --------------------------------------------------------------------------
# codec helpers (R1, R2)
# --------------------------------------------------------------------------

def leb_len(d: int) -> int:
    return int(lib().o_leb_len(int(d)))


def leb_put(d: int) -> bytes:
    buf = np.zeros(16, dtype=np.uint8)
    n = lib().o_leb_put(buf, int(d))
    return bytes(buf[:n])


def leb_get(b: bytes):
    buf = np.zeros(16, dtype=np.uint8)
    buf[:len(b)] = np.frombuffer(bytes(b), dtype=np.uint8)
    v = C.c_uint64()
    n = lib().o_leb_get(buf, C.byref(v))
    return int(v.value), int(n)


def leaf_bytes(e) -> int:
    e = _u64(e)
    return int(lib().o_leaf_bytes(e, e.size))


def leaf_encode(e, LB: int):
    e = _u64(e)
    buf = np.zeros(LB, dtype=np.uint8)
    used = lib().o_leaf_encode(buf, LB, e, e.size)
    return buf, int(used)


def leaf_decode(buf, used: int) -> np.ndarray:
    buf = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
    out = np.zeros(max(1, used + 1), dtype=np.uint64)
    m = lib().o_leaf_decode(buf, used, out)
    return out[:m].copy()


def violates(LB, tau_leaf, tau_root, rho_leaf, rho_root, H, h, leaves, nbytes) -> bool:
    return bool(lib().o_violates(LB, tau_leaf, tau_root, rho_leaf, rho_root,
                                 H, h, leaves, nbytes))


def build_leaves(S: int, LB: int, build_pm: int) -> int:
    return int(lib().o_build_leaves(S, LB, build_pm))


def leaf_size(n, lb_min, leaf_growth) -> int:
    """R13: leaf size for an array that will hold n keys."""
    return int(lib().o_leaf_size(n, lb_min, leaf_growth))


def resize_leaves(T, L, LB, tau_root, rho_root, grow_num=6, grow_den=5) -> int:
    return int(lib().o_resize_leaves(T, L, LB, tau_root, rho_root, grow_num, grow_den))


def cut_points(e, W: int) -> np.ndarray:
    e = _u64(e)
    out = np.zeros(W + 1, dtype=np.uint64)
    lib().o_cut_points(e if e.size else np.zeros(1, np.uint64), e.size, W, out)
    return out


# --------------------------------------------------------------------------
# plain definition
# --------------------------------------------------------------------------

class PlainSet:
    """Sorted array of distinct uint64 keys (the plain definition)."""

    def __init__(self, keys=()):
        a = _u64(keys).copy()
        n = lib().oset_sort_unique(a, a.size) if a.size else 0
        self.S = a[:n].copy()

    def __len__(self):
        return int(self.S.size)

    @staticmethod
    def _unique(keys):
        a = _u64(keys).copy()
        n = lib().oset_sort_unique(a, a.size) if a.size else 0
        return a[:n].copy()

    def insert_batch(self, keys) -> int:
        U = self._unique(keys)
        out = np.zeros(self.S.size + U.size + 1, dtype=np.uint64)
        n = lib().oset_union(self.S if self.S.size else np.zeros(1, np.uint64),
                             self.S.size, U if U.size else np.zeros(1, np.uint64),
                             U.size, out)
        added = n - self.S.size
        self.S = out[:n].copy()
        return int(added)

    def delete_batch(self, keys) -> int:
        U = self._unique(keys)
        out = np.zeros(self.S.size + 1, dtype=np.uint64)
        n = lib().oset_difference(self.S if self.S.size else np.zeros(1, np.uint64),
                                  self.S.size, U if U.size else np.zeros(1, np.uint64),
                                  U.size, out)
        removed = self.S.size - n
        self.S = out[:n].copy()
        return int(removed)

    def has_batch(self, keys) -> np.ndarray:
        q = _u64(keys)
        S = self.S if self.S.size else np.zeros(1, np.uint64)
        f = lib().oset_has
        return np.array([f(S, self.S.size, int(x)) for x in q], dtype=np.uint8)

    def range_map(self, lo, hi):
        lo, hi = _u64(lo), _u64(hi)
        S = self.S if self.S.size else np.zeros(1, np.uint64)
        sums = np.zeros(lo.size, dtype=np.uint64)
        cnts = np.zeros(lo.size, dtype=np.uint64)
        s, c = C.c_uint64(), C.c_uint64()
        f = lib().oset_range
        for i in range(lo.size):
            f(S, self.S.size, int(lo[i]), int(hi[i]), C.byref(s), C.byref(c))
            sums[i], cnts[i] = s.value, c.value
        return sums, cnts

    def range_map_length(self, start, length):
        """App. A map_range_length with the sum: the first length[i] keys
        >= start[i]; returns (sums mod 2^64, counts)."""
        start, length = _u64(start), _u64(length)
        S = self.S if self.S.size else np.zeros(1, np.uint64)
        sums = np.zeros(start.size, dtype=np.uint64)
        cnts = np.zeros(start.size, dtype=np.uint64)
        s, c = C.c_uint64(), C.c_uint64()
        f = lib().oset_range_length
        for i in range(start.size):
            f(S, self.S.size, int(start[i]), int(length[i]), C.byref(s), C.byref(c))
            sums[i], cnts[i] = s.value, c.value
        return sums, cnts

    def range_extract(self, lo, hi):
        """Sec. 3 range_map emitting the keys: (offsets, keys) with the keys
        of [lo[i], hi[i]) at keys[offsets[i]:offsets[i+1]]."""
        lo, hi = _u64(lo), _u64(hi)
        parts, off = [], [0]
        for a, b in zip(lo.tolist(), hi.tolist()):
            i = int(np.searchsorted(self.S, np.uint64(a), side="left"))
            j = int(np.searchsorted(self.S, np.uint64(b), side="left")) if a < b else i
            parts.append(self.S[i:j])
            off.append(off[-1] + (j - i))
        keys = np.concatenate(parts) if parts else np.zeros(0, np.uint64)
        return np.array(off, dtype=np.uint64), keys.astype(np.uint64)

    OPS = {"sum": 0, "min": 1, "max": 2, "xor": 3}

    def range_reduce(self, lo, hi, op="sum", mask=0, value=0):
        """range_map with another function over the keys in [lo, hi) whose
        bits under `mask` equal `value`; returns (results, counts)."""
        lo, hi = _u64(lo), _u64(hi)
        S = self.S if self.S.size else np.zeros(1, np.uint64)
        outs = np.zeros(lo.size, dtype=np.uint64)
        cnts = np.zeros(lo.size, dtype=np.uint64)
        r, c = C.c_uint64(), C.c_uint64()
        f = lib().oset_range_reduce
        for i in range(lo.size):
            f(S, self.S.size, int(lo[i]), int(hi[i]), self.OPS[op], int(mask), int(value),
              C.byref(r), C.byref(c))
            outs[i], cnts[i] = r.value, c.value
        return outs, cnts

    def sum(self) -> int:
        return int(np.sum(self.S, dtype=np.uint64)) if self.S.size else 0


# --------------------------------------------------------------------------
# sequential CPMA
# --------------------------------------------------------------------------

DEFAULTS = dict(leaf_bytes=512, tau_leaf=900, tau_root=700, rho_leaf=100,
                rho_root=300, grow_num=6, grow_den=5, build_pm=500, rebuild_pm=0, codec=0,
                leaf_growth=0)


class OracleError(RuntimeError):
    pass


class SeqCPMA:
    """Sequential CPMA (Sec. 3-5), one batch at a time."""

    def __init__(self, keys=(), **cfg):
        c = dict(DEFAULTS)
        c.update(cfg)
        self.cfg = c
        k = _u64(keys)
        h = C.c_void_p()
        rc = lib().ocpma_create(C.byref(h), c["leaf_bytes"], c["tau_leaf"],
                                c["tau_root"], c["rho_leaf"], c["rho_root"],
                                c["grow_num"], c["grow_den"], c["build_pm"], c["codec"],
                                c["leaf_growth"], k if k.size else np.zeros(1, np.uint64),
                                k.size)
        if rc != 0:
            raise OracleError("ocpma_create failed: %d" % rc)
        self._h = h
        if c.get("rebuild_pm"):
            lib().ocpma_set_rebuild(h, int(c["rebuild_pm"]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ocpma_destroy(h)
            self._h = None

    def _batch(self, fn, keys) -> int:
        k = _u64(keys)
        d = C.c_uint64()
        rc = fn(self._h, k if k.size else np.zeros(1, np.uint64), k.size, C.byref(d))
        if rc != 0:
            raise OracleError("batch failed: %d" % rc)
        return int(d.value)

    def insert_batch(self, keys) -> int:
        return self._batch(lib().ocpma_insert, keys)

    def delete_batch(self, keys) -> int:
        return self._batch(lib().ocpma_delete, keys)

    def has_batch(self, keys) -> np.ndarray:
        f = lib().ocpma_has
        return np.array([f(self._h, int(x)) for x in _u64(keys)], dtype=np.uint8)

    def range_map(self, lo, hi):
        lo, hi = _u64(lo), _u64(hi)
        sums = np.zeros(lo.size, dtype=np.uint64)
        cnts = np.zeros(lo.size, dtype=np.uint64)
        s, c = C.c_uint64(), C.c_uint64()
        f = lib().ocpma_range
        for i in range(lo.size):
            f(self._h, int(lo[i]), int(hi[i]), C.byref(s), C.byref(c))
            sums[i], cnts[i] = s.value, c.value
        return sums, cnts

    def sum(self) -> int:
        return int(lib().ocpma_sum(self._h))

    def size(self) -> int:
        return int(lib().ocpma_size(self._h))

    def leaves(self) -> int:
        return int(lib().ocpma_leaves(self._h))

    def bytes(self) -> int:
        return int(lib().ocpma_bytes(self._h))

    def elements(self) -> np.ndarray:
        out = np.zeros(self.size() + 1, dtype=np.uint64)
        m = lib().ocpma_elements(self._h, out)
        return out[:m].copy()

    def leaf_bytes(self) -> int:
        return int(lib().ocpma_leaf_bytes(self._h))

    def layout(self):
        L, LB = self.leaves(), self.leaf_bytes()
        data = np.zeros(L * LB, dtype=np.uint8)
        used = np.zeros(L, dtype=np.uint32)
        head = np.zeros(L, dtype=np.uint64)
        lib().ocpma_layout(self._h, data, used, head)
        return data, used, head

    def last_batch(self):
        r, w, t = C.c_uint64(), C.c_uint64(), C.c_uint64()
        lib().ocpma_last_batch(self._h, C.byref(r), C.byref(w), C.byref(t))
        return dict(resized=int(r.value), nwindows=int(w.value), touched=int(t.value))

    def last_windows(self) -> np.ndarray:
        nw = self.last_batch()["nwindows"]
        out = np.zeros(2 * nw + 2, dtype=np.uint64)
        lib().ocpma_last_windows(self._h, out)
        return out[:2 * nw].reshape(-1, 2).copy()

    def check(self) -> int:
        return int(lib().ocpma_check(self._h))
