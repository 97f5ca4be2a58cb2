"""Latency of small updates (Sec. 4: point updates for batches much smaller
than the set): inserts of fresh keys and deletes of present ones, one call
at a time on a warm structure, with the point path on (the default) and off
(the batch algorithm, its front segment as a CUDA graph).  Each call is
timed by CUDA events on the update stream around the C-ABI call, the status
read included; medians over the trials.

    python -m paper_2305_05055_gb300.latency --n 1e8 --sizes 1,1000,4096

Deletes of more than 4096 keys take the batch algorithm in both columns
(the library's point path stops there for deletes).  With --profile the
timed calls of the point path run between
cudaProfilerStart and cudaProfilerStop (for `ncu --profile-from-start off`).
"""
import argparse
import ctypes as C
import json
import statistics

import numpy as np
import torch

from . import cpma as cp
from . import workloads as W


POINT_MAX = 16384  # the library's largest point-path batch


def _keys(dev, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(dev)


def measure(g, present, sizes=(1, 10, 100, 1000, 4096), trials=35, warm=5, seed=900,
            profile=False):
    """Per size: insert and delete latency (µs) with the point path on and
    off, on the handle g (uniform 40-bit keys; `present`, a device int64
    tensor, holds keys of g to delete).  Every batch is undone again after
    its call (untimed), so g ends as it began."""
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream()
    res = torch.zeros(1, dtype=torch.int64, device=dev)
    g.reserve(max(sizes))
    g.use_graphs(1 << 21)
    out = {}
    ins, dele = cp.lib().cpma_insert_batch, cp.lib().cpma_delete_batch
    calls0 = g.point_stats()
    for point in (True, False):
        g.set_point_max(POINT_MAX if point else 0)
        for k in sizes:
            ib = [_keys(dev, W.uniform_keys(seed + 1000 * k + t, k, bits=40))
                  for t in range(warm + trials)]
            idx = (W.splitmix64(seed + 7 * k, (warm + trials) * k) %
                   np.uint64(present.numel())).astype(np.int64)
            db = [present[torch.from_numpy(idx[t * k:(t + 1) * k]).to(dev)].contiguous()
                  for t in range(warm + trials)]
            row = {}
            for name, fn, batches, undo in (("insert", ins, ib, dele), ("delete", dele, db, ins)):
                ev = []
                for t, b in enumerate(batches):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    timed = t >= warm
                    if timed and profile and point:
                        torch.cuda.cudart().cudaProfilerStart()
                    e0.record(st)
                    rc = fn(g.handle, C.c_void_p(b.data_ptr()), k, 0, C.c_void_p(res.data_ptr()),
                            C.c_void_p(st.cuda_stream))
                    e1.record(st)
                    st.synchronize()
                    if timed and profile and point:
                        torch.cuda.cudart().cudaProfilerStop()
                    if rc != cp.CPMA_OK:
                        raise cp.CPMAError(rc, name)
                    if timed:
                        ev.append(e0.elapsed_time(e1) * 1e3)
                    # put the set back (untimed)
                    undo(g.handle, C.c_void_p(b.data_ptr()), k, 0, None, C.c_void_p(st.cuda_stream))
                    st.synchronize()
                row[name + "_us"] = statistics.median(ev)
            out.setdefault("point" if point else "batch", {})[str(k)] = row
    g.set_point_max(POINT_MAX)
    calls1 = g.point_stats()
    out["point_calls"] = calls1["calls"] - calls0["calls"]
    out["point_fell_back"] = calls1["batch"] - calls0["batch"]
    out["note"] = ("warm, one call at a time, CUDA events around the C-ABI call (status read "
                   "included); 'batch' = point path off, front segment as a CUDA graph")
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--n", type=float, default=1e8)
    ap.add_argument("--sizes", default="1,10,100,1000,4096,16384")
    ap.add_argument("--trials", type=int, default=35)
    ap.add_argument("--leaf-bytes", type=int, default=512)
    ap.add_argument("--profile", action="store_true")
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    base = W.uniform_keys(2, int(a.n), bits=40)
    g = cp.CPMA(_keys(dev, base), leaf_bytes=a.leaf_bytes)
    sizes = tuple(int(float(s)) for s in a.sizes.split(","))
    r = measure(g, _keys(dev, np.unique(base)), sizes=sizes, trials=a.trials, profile=a.profile)
    r["n"] = int(a.n)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
