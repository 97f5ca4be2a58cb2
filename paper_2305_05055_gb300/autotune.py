"""Autotuner for the CPMA's tunables.

* Leaf size: times the operations that matter for a workload -- batch
  insert, batch delete and range_map over rank-based ranges -- for every
  candidate leaf size on one seeded sample of that workload, with CUDA
  events, and picks the best weighted throughput.
* Merge-versus-rebuild threshold (Sec. 4: small batches merge leaf by leaf,
  batches of k >= n/10 are best applied by rebuilding everything): times
  both strategies on clones of the same state for growing batch sizes and
  sets ``rebuild_pm`` at the smallest batch-to-set ratio from which the
  rebuild stays faster (0 when it never is).
* Growing factor (App. C): grows a set by a run of inserts under each
  candidate factor and weighs time against the final bytes per key.

Set-level results are identical for every configuration (it only changes
the layout), so the choice is purely about speed and space.  The chosen
configuration can be saved as JSON and passed to :class:`cpma.CPMA` as
keyword arguments.
"""
from __future__ import annotations

import json
import math
import statistics

import numpy as np
import torch

from . import cpma as cp
from . import workloads as W

LEAF_BYTES = (256, 512, 1024, 2048)
GROWTH = ((6, 5),)
GROWTH_SWEEP = ((11, 10), (6, 5), (3, 2), (2, 1))
REBUILD_RATIOS = (0.01, 0.03, 0.1, 0.3)


def _timed(fn, reps=3):
    st = torch.cuda.current_stream()
    out = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        out.append(e0.elapsed_time(e1))
    return statistics.median(out)


def measure(base: torch.Tensor, sorted_keys: torch.Tensor, batch: int, queries: int,
            leaf_bytes: int, grow=(6, 5), seed: int = 77, min_width: int = 10,
            max_width: int = 10 ** 6) -> dict:
    """One configuration on one workload sample (all device-resident)."""
    dev = base.device
    g = cp.CPMA(base, leaf_bytes=leaf_bytes, grow_num=grow[0], grow_den=grow[1])
    n = sorted_keys.numel()
    ins = torch.from_numpy(W.uniform_keys(seed, batch, bits=40).view(np.int64)).to(dev)
    r = torch.from_numpy((W.splitmix64(seed + 1, queries) % np.uint64(n)).astype(np.int64)).to(dev)
    u = W.uniform01(seed + 2, queries)
    a, b = np.log10(min_width), np.log10(max_width)
    c = torch.from_numpy(np.floor(10.0 ** (a + (b - a) * u)).astype(np.int64)).to(dev)
    lo = sorted_keys[r]
    j = r + c
    hi = torch.where(j < n, sorted_keys[torch.clamp(j, max=n - 1)], torch.full_like(lo, -1))
    res = {"leaf_bytes": leaf_bytes, "grow": list(grow), "bytes_per_key": g.bytes() / g.size()}
    # insert and delete of the same fresh batch, on clones of one state whose
    # scratch is reserved and warmed by an insert + delete of another batch
    warm = torch.from_numpy(W.uniform_keys(seed + 3, batch, bits=40).view(np.int64)).to(dev)
    ms_ins, ms_del = [], []
    for _ in range(3):
        h = g.clone()
        h.reserve(batch)
        h.insert_batch(warm)
        h.delete_batch(warm)
        torch.cuda.synchronize()
        ms_ins.append(_timed(lambda: h.insert_batch(ins), reps=1))
        ms_del.append(_timed(lambda: h.delete_batch(ins), reps=1))
        del h
    res["insert_keys_per_s"] = batch / (statistics.median(ms_ins) / 1e3)
    res["delete_keys_per_s"] = batch / (statistics.median(ms_del) / 1e3)
    sums, cnts = g.range_map(lo, hi)
    elems = int(cnts.sum().item())
    ms = _timed(lambda: g.range_map(lo, hi))
    res["range_elems_per_s"] = elems / (ms / 1e3)
    res["range_ms"] = ms
    ms = _timed(lambda: g.sum())
    res["scan_elems_per_s"] = g.size() / (ms / 1e3)
    del g
    torch.cuda.synchronize()
    return res


def tune(base: torch.Tensor, sorted_keys: torch.Tensor, batch: int = 10 ** 6,
         queries: int = 10 ** 5, weights=None, leaf_sizes=LEAF_BYTES, growth=GROWTH) -> dict:
    """Measure every candidate and pick the best by the weighted geometric
    mean of insert, delete and range throughput."""
    weights = weights or {"insert_keys_per_s": 1.0, "delete_keys_per_s": 0.5,
                          "range_elems_per_s": 1.0}
    rows = [measure(base, sorted_keys, batch, queries, lb, gr)
            for lb in leaf_sizes for gr in growth]
    tot = sum(weights.values())

    def score(r):
        return float(np.exp(sum(w * np.log(r[k]) for k, w in weights.items()) / tot))

    for r in rows:
        r["score"] = score(r)
    best = max(rows, key=lambda r: r["score"])
    return {"best": {"leaf_bytes": best["leaf_bytes"], "grow_num": best["grow"][0],
                     "grow_den": best["grow"][1]},
            "best_by": {k: max(rows, key=lambda r: r[k])["leaf_bytes"] for k in weights},
            "candidates": rows, "weights": weights}


def _keys(seed, count, dev):
    return torch.from_numpy(W.uniform_keys(seed, count, bits=40).view(np.int64)).to(dev)


def tune_rebuild(base: torch.Tensor, ratios=REBUILD_RATIOS, leaf_bytes: int = 512,
                 trials: int = 2, seed: int = 91) -> dict:
    """Median insert and delete time of a batch of ratio * n fresh keys by
    the batch merge (rebuild_pm = 0) and by the rebuild (rebuild_pm = 1),
    on clones of one state with reserved, warm scratch.  rebuild_pm becomes
    the smallest ratio (in permille) from which the rebuild is faster for
    every larger ratio measured, else 0."""
    dev = base.device
    rows = []
    for pm in (0, 1):
        g = cp.CPMA(base, leaf_bytes=leaf_bytes, rebuild_pm=pm)
        n = g.size()
        for ratio in ratios:
            k = max(1, int(ratio * n))
            b, w = _keys(seed, k, dev), _keys(seed + 1, k, dev)
            ti, td = [], []
            for _ in range(trials):
                h = g.clone()
                h.reserve(k)
                h.insert_batch(w)
                h.delete_batch(w)
                torch.cuda.synchronize()
                ti.append(_timed(lambda: h.insert_batch(b), reps=1))
                td.append(_timed(lambda: h.delete_batch(b), reps=1))
                del h
            rows.append({"rebuild": bool(pm), "ratio": ratio, "batch": k,
                         "insert_ms": statistics.median(ti), "delete_ms": statistics.median(td)})
            del b, w
        del g
        torch.cuda.synchronize()
    merge = {r["ratio"]: r for r in rows if not r["rebuild"]}
    reb = {r["ratio"]: r for r in rows if r["rebuild"]}
    wins = [reb[x]["insert_ms"] + reb[x]["delete_ms"] < merge[x]["insert_ms"] + merge[x]["delete_ms"]
            for x in ratios]
    pm = 0
    for i, x in enumerate(ratios):
        if all(wins[i:]):
            pm = int(math.ceil(1000 * x))
            break
    return {"rebuild_pm": pm, "rows": rows}


def tune_growth(n0: int = 10 ** 7, batch: int = 10 ** 6, steps: int = 40,
                factors=GROWTH_SWEEP, leaf_bytes: int = 512, dev="cuda", seed: int = 61) -> dict:
    """Grow a set of n0 uniform keys by `steps` inserts of `batch` fresh keys
    under each growing factor: total device time, resizes (leaf-count
    changes) and final bytes per key.  The pick minimises time x bytes/key
    (both cost the same fraction when doubled)."""
    base = _keys(seed, n0, dev)
    batches = [_keys(seed + 1 + i, batch, dev) for i in range(steps)]
    rows = []
    for num, den in factors:
        g = cp.CPMA(base, leaf_bytes=leaf_bytes, grow_num=num, grow_den=den)
        g.reserve(batch)
        torch.cuda.synchronize()
        total, resizes, L = 0.0, 0, g.leaves()
        for b in batches:
            total += _timed(lambda: g.insert_batch(b), reps=1)
            if g.leaves() != L:
                resizes += 1
                L = g.leaves()
        rows.append({"grow": [num, den], "total_ms": total, "resizes": resizes,
                     "bytes_per_key": g.bytes() / g.size(), "size": g.size()})
        del g
        torch.cuda.synchronize()
    best = min(rows, key=lambda r: r["total_ms"] * r["bytes_per_key"])
    return {"best": {"grow_num": best["grow"][0], "grow_den": best["grow"][1]}, "rows": rows,
            "n0": n0, "batch": batch, "steps": steps}


def save(result: dict, path: str):
    with open(path, "w") as f:
        json.dump(result["best"], f, indent=1)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)
