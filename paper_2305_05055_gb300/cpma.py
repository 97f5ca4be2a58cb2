"""Python binding of the CPMA C ABI (``include/cpma.h``).

Argument marshalling only: every step of every call runs in the CUDA library
``_build/libcpma.so``.  PyTorch supplies device memory and streams.  Keys are
64-bit unsigned integers; on the torch side they live in int64 (or uint64)
CUDA tensors holding the same bit patterns.

If the library is missing or fails to load, every call raises
:class:`CPMAError`: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np
import torch

from . import build as _build

_lock = threading.Lock()
_lib = None

CPMA_OK, CPMA_EINVAL, CPMA_ENOMEM, CPMA_ECUDA, CPMA_EINTERNAL, CPMA_ETIMEOUT = 0, -1, -2, -3, -4, -5

# device memory callbacks of cpma_config: alloc(bytes, stream, ctx) -> pointer
# (NULL when it cannot), free(pointer, stream, ctx)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class CPMAError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = lib().cpma_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s: %s (%d)" % (what, msg, code))


class cpma_config(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in (
        "leaf_bytes", "tau_leaf", "tau_root", "rho_leaf", "rho_root", "grow_num",
        "grow_den", "build_pm", "rebuild_pm", "codec", "leaf_growth", "reserved")] + [
        ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p),
        ("mem_budget_bytes", C.c_uint64)]


def lib():
    """Load libcpma.so (building it first when the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or os.environ.get("CPMA_REBUILD"):
                path = _build.build()
            try:
                L = C.CDLL(path)
            except OSError as e:  # pragma: no cover - depends on the box
                raise RuntimeError("cannot load the CPMA CUDA library %s: %s" % (path, e))
            V, U64, I = C.c_void_p, C.c_uint64, C.c_int
            P64 = C.POINTER(U64)
            sig = {
                "cpma_default_config": (None, [C.POINTER(cpma_config)]),
                "cpma_create": (I, [C.POINTER(V), C.POINTER(cpma_config), V, U64, V]),
                "cpma_destroy": (I, [V]),
                "cpma_clone": (I, [V, C.POINTER(V), V]),
                "cpma_insert_batch": (I, [V, V, U64, I, V, V]),
                "cpma_delete_batch": (I, [V, V, U64, I, V, V]),
                "cpma_has_batch": (I, [V, V, U64, V, V]),
                "cpma_range_map": (I, [V, V, V, U64, V, V, V]),
                "cpma_sum": (I, [V, V, V, V]),
                "cpma_size": (I, [V, P64]),
                "cpma_bytes": (I, [V, P64]),
                "cpma_leaves": (I, [V, P64]),
                "cpma_export_layout": (I, [V, V, V, V, V]),
                "cpma_stats": (I, [V, P64]),
                "cpma_reset_stats": (I, [V]),
                "cpma_strerror": (C.c_char_p, [I]),
                "cpma_range_map_noalloc": (I, [V, V, V, U64, V, V, V]),
                "cpma_insert_batch_tagged": (I, [V, V, V, U64, I, U64, V, V]),
                "cpma_delete_batch_tagged": (I, [V, V, V, U64, I, U64, V, V]),
                "cpma_sort_batch": (I, [V, V, V, U64, V, V, V]),
                "cpma_profile": (I, [V, I]),
                "cpma_profile_mask": (I, [V, C.c_uint32]),
                "cpma_profile_read": (I, [V, C.POINTER(C.c_double), P64, P64, I]),
                "cpma_reserve": (I, [V, U64, U64, I, V]),
                "cpma_range_map_length": (I, [V, V, V, U64, V, V, V]),
                "cpma_range_reduce": (I, [V, V, V, U64, I, U64, U64, V, V, V]),
                "cpma_range_extract": (I, [V, V, V, U64, V, V, U64, V]),
                "cpma_use_graphs": (I, [V, U64]),
                "cpma_graph_stats": (I, [V, P64, P64]),
                "cpma_set_point_max": (I, [V, U64]),
                "cpma_point_stats": (I, [V, P64, P64]),
                "cpma_leaf_bytes": (I, [V, P64]),
                "cpma_mem_held": (I, [V, P64]),
                "cpma_mem_peak": (I, [V, P64]),
                "cpma_set_mem_budget": (I, [V, U64]),
                "cpma_test_sort_stall": (I, [V, C.c_uint32, C.c_int64]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype, f.argtypes = res, args
            _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != CPMA_OK:
        raise CPMAError(rc, what)


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _keys(t, name="keys") -> torch.Tensor:
    if isinstance(t, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(t).view(np.int64)).cuda()
    if not (t.is_cuda and t.element_size() == 8):
        raise TypeError("%s: expected a CUDA tensor of 64-bit integers" % name)
    return t.contiguous()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None and t.numel() else None


def to_u64(t: torch.Tensor) -> np.ndarray:
    """Device int64/uint64 tensor -> host numpy uint64 (same bits)."""
    return t.detach().cpu().contiguous().view(torch.int64).numpy().view(np.uint64)


def default_config(**overrides) -> cpma_config:
    """The library's defaults with some fields replaced; alloc / free take
    ALLOC_FN / FREE_FN objects (the caller keeps them alive)."""
    c = cpma_config()
    lib().cpma_default_config(C.byref(c))
    for k, v in overrides.items():
        setattr(c, k, v if k in ("alloc", "free", "alloc_ctx") else int(v))
    return c


# ---------------------------------------------------------------------------
# functions with the names of the C ABI
# ---------------------------------------------------------------------------

def cpma_create(keys, config: cpma_config | None = None, stream=None):
    k = _keys(keys) if keys is not None and len(keys) else None
    h = C.c_void_p()
    _check(lib().cpma_create(C.byref(h), C.byref(config) if config is not None else None,
                             _ptr(k), 0 if k is None else k.numel(), C.c_void_p(_stream(stream))),
           "cpma_create")
    return h


def cpma_destroy(h):
    _check(lib().cpma_destroy(h), "cpma_destroy")


def cpma_clone(h, stream=None):
    out = C.c_void_p()
    _check(lib().cpma_clone(h, C.byref(out), C.c_void_p(_stream(stream))), "cpma_clone")
    return out


def cpma_insert_batch(h, keys, sorted=False, out=None, stream=None):
    k = _keys(keys)
    _check(lib().cpma_insert_batch(h, _ptr(k), k.numel(), int(bool(sorted)), _ptr(out),
                                   C.c_void_p(_stream(stream))), "cpma_insert_batch")
    return out


def cpma_delete_batch(h, keys, sorted=False, out=None, stream=None):
    k = _keys(keys)
    _check(lib().cpma_delete_batch(h, _ptr(k), k.numel(), int(bool(sorted)), _ptr(out),
                                   C.c_void_p(_stream(stream))), "cpma_delete_batch")
    return out


def _tags(t):
    if not (t.is_cuda and t.element_size() == 4):
        raise TypeError("tags: expected a CUDA tensor of 32-bit integers")
    return t.contiguous()


def cpma_insert_batch_tagged(h, keys, tags, ntags, counts=None, sorted=False, stream=None):
    """Insert with per-request attribution: counts[t] = keys request t added."""
    k, tg = _keys(keys), _tags(tags)
    if counts is None:
        counts = torch.empty(ntags, dtype=torch.int64, device=k.device)
    _check(lib().cpma_insert_batch_tagged(h, _ptr(k), _ptr(tg), k.numel(), int(bool(sorted)),
                                          ntags, _ptr(counts), C.c_void_p(_stream(stream))),
           "cpma_insert_batch_tagged")
    return counts


def cpma_delete_batch_tagged(h, keys, tags, ntags, counts=None, sorted=False, stream=None):
    """Delete with per-request attribution: counts[t] = keys request t removed."""
    k, tg = _keys(keys), _tags(tags)
    if counts is None:
        counts = torch.empty(ntags, dtype=torch.int64, device=k.device)
    _check(lib().cpma_delete_batch_tagged(h, _ptr(k), _ptr(tg), k.numel(), int(bool(sorted)),
                                          ntags, _ptr(counts), C.c_void_p(_stream(stream))),
           "cpma_delete_batch_tagged")
    return counts


def cpma_sort_batch(h, keys, tags=None, keys_out=None, tags_out=None, stream=None):
    k = _keys(keys)
    if keys_out is None:
        keys_out = torch.empty_like(k)
    tg = _tags(tags) if tags is not None else None
    if tg is not None and tags_out is None:
        tags_out = torch.empty_like(tg)
    _check(lib().cpma_sort_batch(h, _ptr(k), _ptr(tg), k.numel(), _ptr(keys_out),
                                 _ptr(tags_out) if tg is not None else None,
                                 C.c_void_p(_stream(stream))), "cpma_sort_batch")
    return keys_out, tags_out


def cpma_has_batch(h, keys, out=None, stream=None):
    k = _keys(keys)
    if out is None:
        out = torch.empty(k.numel(), dtype=torch.uint8, device=k.device)
    _check(lib().cpma_has_batch(h, _ptr(k), k.numel(), _ptr(out), C.c_void_p(_stream(stream))),
           "cpma_has_batch")
    return out


def cpma_range_map(h, lo, hi, out_sum=None, out_count=None, stream=None):
    lo, hi = _keys(lo, "lo"), _keys(hi, "hi")
    if lo.numel() != hi.numel():
        raise ValueError("lo and hi differ in length")
    q = lo.numel()
    if out_sum is None:
        out_sum = torch.empty(q, dtype=torch.int64, device=lo.device)
    if out_count is None:
        out_count = torch.empty(q, dtype=torch.int64, device=lo.device)
    _check(lib().cpma_range_map(h, _ptr(lo), _ptr(hi), q, _ptr(out_sum), _ptr(out_count),
                                C.c_void_p(_stream(stream))), "cpma_range_map")
    return out_sum, out_count


RANGE_NOALLOC_MAX_QUERIES = 65536


def cpma_range_map_length(h, start, length, out_sum=None, out_count=None, stream=None):
    """App. A map_range_length with (sum, count): the first length[i] keys >=
    start[i] (length may be a scalar)."""
    start = _keys(start, "start")
    if not torch.is_tensor(length):
        length = torch.full_like(start, int(np.uint64(length).view(np.int64)))
    length = _keys(length, "length")
    if length.numel() != start.numel():
        raise ValueError("start and length differ in size")
    q = start.numel()
    s = out_sum if out_sum is not None else torch.empty(q, dtype=torch.int64, device=start.device)
    c = out_count if out_count is not None else torch.empty(q, dtype=torch.int64,
                                                            device=start.device)
    _check(lib().cpma_range_map_length(h, _ptr(start), _ptr(length), q, _ptr(s), _ptr(c),
                                       C.c_void_p(_stream(stream))), "cpma_range_map_length")
    return s, c


def cpma_range_extract(h, lo, hi, stream=None):
    """The keys of every [lo[i], hi[i]), packed: returns (offsets, keys) with
    query i's keys at keys[offsets[i]:offsets[i+1]] (two library calls: the
    first sizes the output)."""
    lo, hi = _keys(lo, "lo"), _keys(hi, "hi")
    if lo.numel() != hi.numel():
        raise ValueError("lo and hi differ in size")
    q = lo.numel()
    off = torch.empty(q + 1, dtype=torch.int64, device=lo.device)
    st = C.c_void_p(_stream(stream))
    _check(lib().cpma_range_extract(h, _ptr(lo), _ptr(hi), q, _ptr(off), None, 0, st),
           "cpma_range_extract")
    total = int(off[q].item())
    out = torch.empty(max(total, 1), dtype=torch.int64, device=lo.device)
    _check(lib().cpma_range_extract(h, _ptr(lo), _ptr(hi), q, _ptr(off), _ptr(out), total, st),
           "cpma_range_extract")
    return off, out[:total]


OPS = {"sum": 0, "min": 1, "max": 2, "xor": 3}


def cpma_range_reduce(h, lo, hi, op="sum", mask=0, value=0, out=None, out_count=None,
                      stream=None):
    """range_map with min / max / xor / sum over the keys of [lo, hi) whose
    bits under mask equal value; returns (results, counts)."""
    lo, hi = _keys(lo, "lo"), _keys(hi, "hi")
    if lo.numel() != hi.numel():
        raise ValueError("lo and hi differ in size")
    q = lo.numel()
    r = out if out is not None else torch.empty(q, dtype=torch.int64, device=lo.device)
    c = out_count if out_count is not None else torch.empty(q, dtype=torch.int64,
                                                            device=lo.device)
    _check(lib().cpma_range_reduce(h, _ptr(lo), _ptr(hi), q, OPS[op] if isinstance(op, str)
                                   else int(op), C.c_uint64(int(mask)), C.c_uint64(int(value)),
                                   _ptr(r), _ptr(c), C.c_void_p(_stream(stream))),
           "cpma_range_reduce")
    return r, c


def cpma_range_map_noalloc(h, lo, hi, out_sum, out_count, stream=None):
    """cpma_range_map with no device allocation inside the call: the caller
    passes the output buffers, the library uses its fixed scratch array."""
    lo, hi = _keys(lo, "lo"), _keys(hi, "hi")
    if lo.numel() != hi.numel():
        raise ValueError("lo and hi differ in length")
    _check(lib().cpma_range_map_noalloc(h, _ptr(lo), _ptr(hi), lo.numel(), _ptr(out_sum),
                                        _ptr(out_count), C.c_void_p(_stream(stream))),
           "cpma_range_map_noalloc")
    return out_sum, out_count


def cpma_sum(h, stream=None, device="cuda"):
    s = torch.empty(1, dtype=torch.int64, device=device)
    c = torch.empty(1, dtype=torch.int64, device=device)
    _check(lib().cpma_sum(h, _ptr(s), _ptr(c), C.c_void_p(_stream(stream))), "cpma_sum")
    return s, c


def _u64_out(fn, h, what):
    v = C.c_uint64()
    _check(fn(h, C.byref(v)), what)
    return int(v.value)


def cpma_size(h) -> int:
    return _u64_out(lib().cpma_size, h, "cpma_size")


def cpma_bytes(h) -> int:
    return _u64_out(lib().cpma_bytes, h, "cpma_bytes")


def cpma_leaves(h) -> int:
    return _u64_out(lib().cpma_leaves, h, "cpma_leaves")


def cpma_leaf_bytes(h) -> int:
    return _u64_out(lib().cpma_leaf_bytes, h, "cpma_leaf_bytes")


def cpma_mem_held(h) -> int:
    return _u64_out(lib().cpma_mem_held, h, "cpma_mem_held")


def cpma_mem_peak(h) -> int:
    return _u64_out(lib().cpma_mem_peak, h, "cpma_mem_peak")


def cpma_set_mem_budget(h, nbytes: int):
    _check(lib().cpma_set_mem_budget(h, int(nbytes)), "cpma_set_mem_budget")


def cpma_test_sort_stall(h, poll_limit: int, silent_tile: int):
    _check(lib().cpma_test_sort_stall(h, int(poll_limit), int(silent_tile)),
           "cpma_test_sort_stall")


def cpma_stats(h) -> int:
    return _u64_out(lib().cpma_stats, h, "cpma_stats")


def cpma_reset_stats(h):
    _check(lib().cpma_reset_stats(h), "cpma_reset_stats")


def cpma_reserve(h, max_batch: int, max_queries: int = 0, tagged: bool = False, stream=None):
    _check(lib().cpma_reserve(h, int(max_batch), int(max_queries), int(bool(tagged)),
                              C.c_void_p(_stream(stream))), "cpma_reserve")


def cpma_use_graphs(h, max_batch: int = 1 << 16):
    """Front segment of untagged updates of <= max_batch keys as CUDA graphs
    (0: off)."""
    _check(lib().cpma_use_graphs(h, int(max_batch)), "cpma_use_graphs")


def cpma_graph_stats(h) -> dict:
    c, n = C.c_uint64(), C.c_uint64()
    _check(lib().cpma_graph_stats(h, C.byref(c), C.byref(n)), "cpma_graph_stats")
    return {"captures": int(c.value), "launches": int(n.value)}


def cpma_set_point_max(h, max_keys: int):
    """Untagged inserts of <= max_keys keys try the point path first (0: never)."""
    _check(lib().cpma_set_point_max(h, int(max_keys)), "cpma_set_point_max")


def cpma_point_stats(h) -> dict:
    c, b = C.c_uint64(), C.c_uint64()
    _check(lib().cpma_point_stats(h, C.byref(c), C.byref(b)), "cpma_point_stats")
    return {"calls": int(c.value), "batch": int(b.value)}


PHASES = ("sort", "route", "merge", "count", "redistribute", "finish", "has",
          "range_prep", "range", "sum", "merge_other", "merge_lane")


def cpma_profile(h, enable: bool = True):
    _check(lib().cpma_profile(h, int(bool(enable))), "cpma_profile")


def cpma_profile_mask(h, phases=None):
    """Time only the named phases (None: all of them)."""
    mask = 0xFFFFFFFF if phases is None else sum(1 << PHASES.index(p) for p in phases)
    _check(lib().cpma_profile_mask(h, mask), "cpma_profile_mask")


def cpma_profile_read(h) -> dict:
    n = len(PHASES)
    ms = (C.c_double * n)()
    by = (C.c_uint64 * n)()
    ca = (C.c_uint64 * n)()
    _check(lib().cpma_profile_read(h, ms, by, ca, n), "cpma_profile_read")
    return {p: dict(ms=float(ms[i]), bytes=int(by[i]), calls=int(ca[i]))
            for i, p in enumerate(PHASES)}


def cpma_export_layout(h, leaf_bytes: int | None = None, stream=None, device="cuda"):
    L = cpma_leaves(h)
    if leaf_bytes is None:
        leaf_bytes = cpma_leaf_bytes(h)
    data = torch.empty(L * leaf_bytes, dtype=torch.uint8, device=device)
    used = torch.empty(L, dtype=torch.int32, device=device)
    heads = torch.empty(L, dtype=torch.int64, device=device)
    _check(lib().cpma_export_layout(h, _ptr(data), _ptr(used), _ptr(heads),
                                    C.c_void_p(_stream(stream))), "cpma_export_layout")
    return data, used, heads


# ---------------------------------------------------------------------------
# object wrapper
# ---------------------------------------------------------------------------

class CPMA:
    """A CPMA on the current CUDA device.  Updates and queries run on the
    current torch stream unless one is given."""

    def __init__(self, keys=None, stream=None, _handle=None, **config):
        self.config = default_config(**config)
        self._h = _handle if _handle is not None else cpma_create(keys, self.config, stream)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.cpma_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h

    def clone(self, stream=None) -> "CPMA":
        c = CPMA.__new__(CPMA)
        c.config = self.config
        c._h = cpma_clone(self._h, stream)
        return c

    def insert_batch(self, keys, sorted=False, stream=None) -> torch.Tensor:
        k = _keys(keys)
        out = torch.empty(1, dtype=torch.int64, device=k.device)
        return cpma_insert_batch(self._h, k, sorted, out, stream)

    def delete_batch(self, keys, sorted=False, stream=None) -> torch.Tensor:
        k = _keys(keys)
        out = torch.empty(1, dtype=torch.int64, device=k.device)
        return cpma_delete_batch(self._h, k, sorted, out, stream)

    def has_batch(self, keys, stream=None) -> torch.Tensor:
        return cpma_has_batch(self._h, keys, None, stream)

    def range_map(self, lo, hi, stream=None):
        return cpma_range_map(self._h, lo, hi, None, None, stream)

    def range_map_length(self, start, length, stream=None):
        return cpma_range_map_length(self._h, start, length, stream=stream)

    def range_extract(self, lo, hi, stream=None):
        return cpma_range_extract(self._h, lo, hi, stream=stream)

    def range_reduce(self, lo, hi, op="sum", mask=0, value=0, stream=None):
        return cpma_range_reduce(self._h, lo, hi, op, mask, value, stream=stream)

    def sum(self, stream=None):
        return cpma_sum(self._h, stream)

    def size(self) -> int:
        return cpma_size(self._h)

    def bytes(self) -> int:
        return cpma_bytes(self._h)

    def leaves(self) -> int:
        return cpma_leaves(self._h)

    def layout(self, stream=None):
        return cpma_export_layout(self._h, None, stream)

    def leaf_bytes(self) -> int:
        return cpma_leaf_bytes(self._h)

    def mem_held(self) -> int:
        return cpma_mem_held(self._h)

    def mem_peak(self) -> int:
        return cpma_mem_peak(self._h)

    def set_mem_budget(self, nbytes: int):
        cpma_set_mem_budget(self._h, nbytes)

    def launches(self) -> int:
        return cpma_stats(self._h)

    def reserve(self, max_batch: int, max_queries: int = 0, tagged: bool = False, stream=None):
        cpma_reserve(self._h, max_batch, max_queries, tagged, stream)

    def use_graphs(self, max_batch: int = 1 << 16):
        cpma_use_graphs(self._h, max_batch)

    def graph_stats(self) -> dict:
        return cpma_graph_stats(self._h)

    def set_point_max(self, max_keys: int):
        cpma_set_point_max(self._h, max_keys)

    def point_stats(self) -> dict:
        return cpma_point_stats(self._h)

    def profile(self, enable: bool = True, phases=None):
        """Reset and enable (or disable) per-phase profiling; `phases` limits
        the timed phases (names of PHASES), the byte counts cover all."""
        cpma_profile_mask(self._h, phases)
        cpma_profile(self._h, enable)

    def profile_read(self) -> dict:
        return cpma_profile_read(self._h)
