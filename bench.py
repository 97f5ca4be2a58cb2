#!/usr/bin/env python
"""Benchmark of the GPU CPMA hot path on GB300.

Headline (the timed K steps): batch insert into a CPMA holding 1e8 uniform
40-bit keys, one step = one cpma_insert_batch of 1e6 fresh uniform 40-bit keys
(unsorted, repeats allowed), so the set grows by about 1e6 per step as in the
paper's protocol (start at 1e8, add batches).  value = inserted keys / device
time of the K steps (CUDA events on the stream, max over ranks).

After the timed region the same run measures, with CUDA events, the other rows
of the hot path on the same structure: batch delete of 1e6 present keys,
has_batch of 1e6 keys, range_map of 1e5 queries whose widths are log-uniform
between 10 and 1e6 elements (one launch), map_range_length and filtered
reductions over the same queries, and a full-set scan sum; each with its
algorithmic bytes and achieved fraction of the measured HBM bandwidth.  Then
the batch-size sweep (1e3..1e7 inserts and deletes at 1e8, launch by launch
and with CUDA graphs), the autotuner (leaf size, merge-versus-rebuild
threshold, growing factor), the skewed-update rounds, the continuous-batching
server against one call per request (offered-rate sweep, p50/p99 at 70% of
saturation) and the R-MAT edge set.  Each has a --no-* switch.

--impl reference times the CPU oracle (oracle/, single thread) on a bounded
sample of the same workload.  Several GPUs: independent replicas, one per
rank, no collective on the data path (the timing uses a barrier and a max).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "batch-insert keys/s, range-sum elems/s at n=1e8 (% HBM peak); serve p99 ms"
PAPER_INSERT_1E6 = 1.1e8  # Table batch-ins-del, uniform, batch 1e6, 64-core Xeon (context)


def aggregate(local_ms: float, units_per_rank: float, dist=None):
    """Max of the ranks' times and the whole-job rate: every rank processed
    units_per_rank units, the job took the slowest rank's time."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        import torch
        dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([local_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        local_ms = float(t.item())
        world = dist.get_world_size()
    else:
        world = 1
    return local_ms, world * units_per_rank / (local_ms / 1e3)


KERNEL_SOURCES = ("update.cu", "dev_common.cuh", "query.cu")


def code_only(text: str) -> str:
    """C/CUDA source without its comments and with blank runs collapsed, so
    that a changed comment does not read as a changed kernel (string and
    character literals are kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        c = text[i]
        if c in "\"'":
            j = i + 1
            while j < n and text[j] != c:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_sources_sha(files=KERNEL_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2305_05055_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(code_only(fh.read()).encode())
    return h.hexdigest()


def measured_traffic(kernel: str, alg_bytes_per_launch: float):
    """DRAM bytes per launch from the committed ncu summary, scaled from the
    captured launch to this one by algorithmic bytes; None when the kernel's
    sources (the entry's list) changed since the capture."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        e = t[kernel]
        if e["sources_sha256"] != kernel_sources_sha(tuple(e.get("sources", KERNEL_SOURCES))):
            return None
        return e["dram_bytes"] * alg_bytes_per_launch / e["alg_bytes"]
    except Exception:
        return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=float, default=1e8)
    ap.add_argument("--batch", type=float, default=1e6)
    ap.add_argument("--leaf-bytes", type=int, default=512)
    ap.add_argument("--queries", type=float, default=1e5)
    ap.add_argument("--no-extra", action="store_true", help="headline only")
    ap.add_argument("--no-sweep", action="store_true", help="skip the insert/delete sweep 1e3..1e7")
    ap.add_argument("--no-graph", action="store_true", help="skip the R-MAT edge-set workload")
    ap.add_argument("--no-pma", action="store_true", help="skip the uncompressed-PMA ablation")
    ap.add_argument("--graph-scale", type=int, default=20)
    ap.add_argument("--sweep-trials", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-skew", action="store_true", help="skip the skewed-update rounds")
    ap.add_argument("--skew-rounds", type=int, default=100)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop comparison")
    ap.add_argument("--no-autotune", action="store_true", help="skip the leaf-size autotuning")
    ap.add_argument("--serve-requests", type=int, default=3000)
    ap.add_argument("--serve-rates", type=lambda x: [float(v) for v in x.split(",")],
                    default=[2500, 5000, 10000, 20000, 40000, 80000],
                    help="offered request rates of the serving sweep (comma separated)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_info():
    model = platform.processor() or platform.machine()
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                model = line.split(":", 1)[1].strip()
    except Exception:
        pass
    return model, os.cpu_count()


def oracle_insert_sample(seconds=12.0, n_sample=10 ** 7, k_sample=10 ** 5, steps=None):
    """The sequential oracle CPMA (oracle/, one thread) on a bounded sample of
    the workload: n = 1e7 uniform 40-bit keys, batches of 1e5 (the same 1%
    batch-to-set ratio as 1e6 into 1e8)."""
    import oracle
    from paper_2305_05055_gb300 import workloads as W
    o = oracle.SeqCPMA(W.uniform_keys(2, n_sample, bits=40), leaf_bytes=512)
    done, t_tot, i = 0, 0.0, 0
    while (steps is None and t_tot < seconds) or (steps is not None and i < steps):
        b = W.uniform_keys(5000 + i, k_sample, bits=40)
        t0 = time.perf_counter()
        o.insert_batch(b)
        t_tot += time.perf_counter() - t0
        done += k_sample
        i += 1
    model, _ = cpu_info()
    return {"value": done / t_tot, "unit": "keys/s", "cores": 1, "kind": "oracle",
            "sample": "sequential oracle CPMA of 1e7 uniform 40-bit keys, %d batch inserts of "
                      "1e5 keys (same 1%% batch/set ratio), LB=512; cpu %s" % (i, model),
            "seconds": t_tot}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_2305_05055_gb300 import workloads as W
    oracle.build()
    n_s, k_s = 10 ** 7, 10 ** 5
    o = oracle.SeqCPMA(W.uniform_keys(2, n_s, bits=40), leaf_bytes=a.leaf_bytes)
    for i in range(a.warmup):
        o.insert_batch(W.uniform_keys(7000 + i, k_s, bits=40))
    times = []
    for i in range(a.steps):
        b = W.uniform_keys(8000 + i, k_s, bits=40)
        t0 = time.perf_counter()
        o.insert_batch(b)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    v = a.steps * k_s / tot
    model, ncpu = cpu_info()
    sample = ("sequential oracle CPMA (one thread) of 1e7 uniform 40-bit keys, one batch insert "
              "of 1e5 fresh keys per step (the 1%% batch/set ratio of 1e6 into 1e8); cpu %s" % model)
    line = {"metric": METRIC, "value": v, "unit": "keys/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1e3 * tot / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": v / PAPER_INSERT_1E6, "dtype": "u64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": "batch insert into a CPMA of uniform 40-bit keys "
                                   "(bounded CPU sample: n=1e7, batch=1e5)",
                       "n": n_s, "batch": k_s, "leaf_bytes": a.leaf_bytes},
            "cpu_baseline": {"value": v, "unit": "keys/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "keys/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.impl == "reference":
        return run_reference(a)

    import torch
    from paper_2305_05055_gb300 import cpma as cp
    from paper_2305_05055_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    hbm_peak, peak_kind = peaks()
    n, k = int(a.n), int(a.batch)
    nsteps, nwarm = a.steps, a.warmup

    def T(x):
        return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- build (inputs resident in HBM before anything is timed) ----
    base = T(W.uniform_keys(2 + 1000 * rank, n, bits=40))
    t0 = time.perf_counter()
    g = cp.CPMA(base, leaf_bytes=a.leaf_bytes)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    nphase = 3  # profiled steps after the timed region, for the per-phase split
    batches = [T(W.uniform_keys(10 ** 6 + 1000 * rank + i, k, bits=40))
               for i in range(nwarm + nsteps + 1 + nphase)]
    # the library's fastest form for this batch size: scratch reserved and
    # the batch front segment replayed as a CUDA graph (captured, with its
    # profiling event nodes, during the warm-up steps).  The timed steps time
    # only the merge phase (the dominant kernel) on the device, so that the
    # profiler adds as little as possible to them; the per-phase split comes
    # from a few fully profiled steps afterwards.
    TIMED_PHASES = ["merge"]
    g.reserve(k)
    g.use_graphs(1 << 21)
    g.profile(True, phases=TIMED_PHASES)
    for i in range(nwarm):
        g.insert_batch(batches[i])
    torch.cuda.synchronize()
    ref = g.clone()          # same state, for the end-to-end pass
    torch.cuda.synchronize()

    # ---- timed region: K insert steps ----
    g.profile(True, phases=TIMED_PHASES)  # reset the per-phase counters
    l0 = g.launches()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        e0.record(st)
        for i in range(nsteps):
            g.insert_batch(batches[nwarm + i])
        e1.record(st)
        barrier()
    ms = e0.elapsed_time(e1)
    launches = g.launches() - l0
    prof = g.profile_read()
    ms, value = aggregate(ms, nsteps * k, dist)

    # per-phase split: every phase timed, a few more steps (the first one
    # captures the graph with all its event nodes)
    g.profile(True)
    g.insert_batch(batches[nwarm + nsteps])
    torch.cuda.synchronize()
    g.profile(True)
    for i in range(nphase):
        g.insert_batch(batches[nwarm + nsteps + 1 + i])
    torch.cuda.synchronize()
    prof_all = g.profile_read()
    g.profile(False)

    # roofline of the dominant kernel of the step (timed in the timed region)
    upd = ["sort", "route", "merge", "merge_lane", "merge_other", "count", "redistribute",
           "finish"]
    dom = max(upd, key=lambda p: prof_all[p]["ms"])
    if dom not in TIMED_PHASES:
        prof = prof_all
    kernel_of = {"merge": "k_insert_thread", "merge_lane": "k_insert_lane",
                 "merge_other": "k_merge_small+k_merge",
                 "sort": "radix sort", "route": "route", "count": "counting",
                 "redistribute": "redistribute", "finish": "k_fix_heads"}
    def roof(p, pk=hbm_peak):
        msp, by, calls = prof[p]["ms"], prof[p]["bytes"], max(1, prof[p]["calls"])
        ach = by / (msp / 1e3) / 1e9 if msp > 0 else 0.0
        return {"bound": "hbm", "achieved": ach, "peak": pk, "unit": "GB/s",
                "frac": ach / pk, "traffic": measured_traffic(kernel_of.get(p, p), by / calls),
                "kernel": kernel_of.get(p, p), "ms_per_launch": msp / calls,
                "bytes_per_launch": by / calls, "peak_kind": peak_kind}
    roofline = roof(dom)
    phases = {p: {"ms_per_step": prof_all[p]["ms"] / nphase,
                  "gbs": (prof_all[p]["bytes"] / (prof_all[p]["ms"] / 1e3) / 1e9)
                  if prof_all[p]["ms"] else None}
              for p in upd}
    phases["note"] = ("device time per step of each phase over %d fully profiled steps after "
                      "the timed ones; the timed steps time only %s" % (nphase, TIMED_PHASES))

    # ---- end to end through the public API with host buffers ----
    host_batches = [batches[nwarm + i].cpu().pin_memory() for i in range(nsteps)]
    added_h = torch.empty(1, dtype=torch.int64).pin_memory()
    # two device buffers: batch i+1 is copied in on a copy stream while batch
    # i is inserted (every copy stays inside the timed loop)
    dbufs = [torch.empty(k, dtype=torch.int64, device=dev) for _ in range(2)]
    added_d = torch.empty(1, dtype=torch.int64, device=dev)
    comp = torch.cuda.current_stream()
    copy_st = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    # the public API's fastest form: scratch reserved, the batch front
    # segment as a CUDA graph, captured by an untimed insert + delete of
    # another batch (which leaves the same set)
    ref.reserve(k)
    ref.use_graphs(1 << 21)
    warm = T(W.uniform_keys(424242, k, bits=40))
    ref.insert_batch(warm)
    ref.delete_batch(warm)
    del warm
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(copy_st):
        dbufs[0].copy_(host_batches[0], non_blocking=True)
    copied[0].record(copy_st)
    for i in range(nsteps):
        b = i & 1
        if i + 1 < nsteps:
            copy_st.wait_event(freed[b ^ 1])  # that buffer's last insert is done
            with torch.cuda.stream(copy_st):
                dbufs[b ^ 1].copy_(host_batches[i + 1], non_blocking=True)
            copied[b ^ 1].record(copy_st)
        comp.wait_event(copied[b])
        cp.cpma_insert_batch(ref.handle, dbufs[b], False, added_d)
        freed[b].record(comp)
        added_h.copy_(added_d, non_blocking=True)
        comp.synchronize()
    e2e_ms, e2e_v = aggregate(1e3 * (time.perf_counter() - t0), nsteps * k, dist)
    e2e = {"value": e2e_v, "unit": "keys/s", "ms_per_step": e2e_ms / nsteps,
           "h2d_bytes_per_step": 8 * k, "d2h_bytes_per_step": 8, "graphs": True,
           "copies": "pinned host -> device on a second stream, one batch ahead "
                     "(double-buffered); result read back every step",
           "graph_stats": ref.graph_stats()}
    del ref

    extra = {}
    if not a.no_extra and rank == 0:
        extra = measure_extra(a, g, batches, dev, st, hbm_peak, peak_kind, T)

    cpu_base = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        try:
            cpu_base = oracle_insert_sample()
        except Exception as ex:  # the oracle is optional for the GPU number
            cpu_base = {"error": str(ex)}

    line = {
        "metric": METRIC, "value": value, "unit": "keys/s", "n_gpus": world, "steps": nsteps,
        "warmup": nwarm, "ms_per_step": ms / nsteps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_INSERT_1E6, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "batch insert of 1e6 uniform 40-bit keys into a CPMA holding "
                               "1e8 keys (grows by 1e6 per step)",
                   "n": n, "batch": k, "leaf_bytes": a.leaf_bytes,
                   "graphs": True, "graph_stats": g.graph_stats(),
                   "l2": "inputs larger than L2 (CPMA %.2f GB, fresh 8 MB batch per step)"
                         % (g.bytes() / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "roofline": roofline, "cpu_baseline": cpu_base, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk.summary(), "phases": phases,
        "build_s": build_s, "bytes_per_key": g.bytes() / g.size(), "size": g.size(),
    }
    line.update(extra)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def measure_extra(a, g, ins_batches, dev, st, hbm_peak, peak_kind, T):
    """Secondary workloads on the CPMA of the headline run; ins_batches are
    every batch inserted into it (warm-up and timed), so the set is known."""
    import torch
    from paper_2305_05055_gb300 import cpma as cp
    from paper_2305_05055_gb300 import workloads as W
    out = {}

    def timed(fn, reps=1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    kname = {"range": "k_range", "sum": "k_sum", "has": "k_has", "merge": "k_insert_thread",
             "merge_lane": "k_insert_lane",
             "merge_other": "k_merge_small+k_merge"}
    def roof(prof, p):
        msp, by, calls = prof[p]["ms"], prof[p]["bytes"], max(1, prof[p]["calls"])
        ach = by / (msp / 1e3) / 1e9 if msp > 0 else 0.0
        kn = kname.get(p, p)
        return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "kernel": kn, "ms_per_launch": msp / calls,
                "bytes_per_launch": by / calls, "peak_kind": peak_kind,
                "traffic": measured_traffic(kn, by / calls)}

    # range_map: 1e5 queries by rank, widths log-uniform 10..1e6 elements
    q = int(a.queries)
    S = torch.empty(0)
    n_now = g.size()
    # sorted set on the device (torch) only to place query endpoints
    lay_d, lay_u, lay_h = None, None, None
    allk = torch.cat([T(W.uniform_keys(2, int(a.n), bits=40))] + list(ins_batches))
    S = torch.unique(allk)
    del allk
    r = torch.from_numpy((W.splitmix64(33, q) % np.uint64(S.numel())).astype(np.int64)).to(dev)
    u = W.uniform01(34, q)
    c = torch.from_numpy(np.floor(10.0 ** (1 + 5 * u)).astype(np.int64)).to(dev)
    lo = S[r]
    j = r + c
    hi = torch.where(j < S.numel(), S[torch.clamp(j, max=S.numel() - 1)],
                     torch.full_like(lo, -1))
    g.profile(True)
    ms, (s, cnt) = timed(lambda: g.range_map(lo, hi), reps=3)
    prof = g.profile_read()
    g.profile(False)
    elems = int(cnt.sum().item())
    out["range_map"] = {"metric": "range-sum elems/s", "value": elems / (ms / 1e3),
                        "unit": "elems/s", "queries": q, "elements": elems,
                        "ms_per_call": ms, "roofline": roof(prof, "range"),
                        "note": "widths log-uniform 10..1e6 elements; overlapping queries may "
                                "hit in L2, so algorithmic GB/s can exceed HBM"}
    # map_range_length over the same queries: the first c keys >= lo are
    # exactly [lo, hi) of the rank-based query, so the sums must agree
    g.profile(True)
    ms_l, (s_l, c_l) = timed(lambda: g.range_map_length(lo, c), reps=3)
    prof = g.profile_read()
    g.profile(False)
    same = bool(torch.equal(s_l, s) and torch.equal(c_l, cnt))
    out["range_map_length"] = {"value": int(c_l.sum().item()) / (ms_l / 1e3), "unit": "elems/s",
                               "queries": q, "ms_per_call": ms_l, "equals_range_map": same,
                               "prep_ms_per_call": prof["range_prep"]["ms"] / 3,
                               "roofline": roof(prof, "range")}
    # filtered reductions (decode every covered leaf): odd keys, minimum
    for op, mask, value in (("sum", 1, 1), ("min", 0, 0)):
        ms_r, (r_r, c_r) = timed(lambda: g.range_reduce(lo, hi, op, mask, value), reps=3)
        out["range_reduce_%s%s" % (op, "_odd" if mask else "")] = {
            "value": elems / (ms_r / 1e3), "unit": "elems/s (covered)", "ms_per_call": ms_r,
            "passed": int(c_r.sum().item())}
    # full-set scan
    g.profile(True)
    ms, (s, cnt) = timed(lambda: g.sum(), reps=5)
    prof = g.profile_read()
    g.profile(False)
    out["full_scan"] = {"value": int(cnt.item()) / (ms / 1e3), "unit": "elems/s",
                        "ms_per_call": ms, "roofline": roof(prof, "sum")}
    # has_batch: half present keys
    hq = torch.cat([S[torch.randint(0, S.numel(), (500000,), device=dev,
                                    generator=torch.Generator(device=dev).manual_seed(5))],
                    T(W.uniform_keys(35, 500000, bits=40))])
    g.profile(True)
    ms, found = timed(lambda: g.has_batch(hq), reps=3)
    prof = g.profile_read()
    g.profile(False)
    out["has"] = {"value": hq.numel() / (ms / 1e3), "unit": "keys/s", "ms_per_call": ms,
                  "found": int(found.sum().item()), "roofline": roof(prof, "has")}
    S_host = None if a.no_serve else cp.to_u64(S)
    if not a.no_autotune:
        from paper_2305_05055_gb300 import autotune
        base = T(W.uniform_keys(2, int(a.n), bits=40))
        at = autotune.tune(base, S, batch=int(a.batch), queries=q)
        rb = autotune.tune_rebuild(base)
        del base
        gr = autotune.tune_growth(dev=dev)
        rnd = lambda rows: [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()}
                            for r in rows]
        out["autotune"] = {"best": dict(at["best"], rebuild_pm=rb["rebuild_pm"],
                                        grow_num=gr["best"]["grow_num"],
                                        grow_den=gr["best"]["grow_den"]),
                           "best_by": at["best_by"], "candidates": rnd(at["candidates"]),
                           "rebuild": rnd(rb["rows"]),
                           "growth": dict(rows=rnd(gr["rows"]), n0=gr["n0"], batch=gr["batch"],
                                          steps=gr["steps"])}
    del S
    # delete of present keys (the batches inserted by the timed steps)
    g.profile(True)
    tot = 0.0
    removed = 0
    for b in ins_batches[: min(5, len(ins_batches))]:
        ms, rm = timed(lambda: g.delete_batch(b))
        tot += ms
        removed += int(rm.item())
    prof = g.profile_read()
    g.profile(False)
    upd = ["sort", "route", "merge", "merge_lane", "merge_other", "count", "redistribute",
           "finish"]
    dom = max(upd, key=lambda p: prof[p]["ms"])
    droof = roof(prof, dom)
    if dom == "merge":  # the delete form of the thread-granular kernel: no capture of its own
        droof.update(kernel="k_insert_thread<true> (delete)", traffic=None)
    out["delete"] = {"value": removed / (tot / 1e3), "unit": "keys/s",
                     "batches": min(5, len(ins_batches)), "batch": int(a.batch),
                     "roofline": droof,
                     "phases_ms": {p: prof[p]["ms"] for p in upd}}
    if not a.no_sweep:
        out["sweep"] = sweep(a, g, dev, T, timed)
        out["pipelined"] = pipelined(a, g, dev, T)
        from paper_2305_05055_gb300 import latency
        c = g.clone()
        # keys the timed steps inserted and the deletes above left in place
        present = torch.cat(list(ins_batches[min(5, len(ins_batches) - 1):]))
        out["small_updates"] = latency.measure(c, present, sizes=(1, 100, 1000, 4096, 16384),
                                               trials=15)
        del c, present
    if not a.no_skew:
        out["skew"] = skew(a, dev, T, timed)
    if not a.no_graph:
        out["graph"] = graph_workload(a, dev, timed)
    if not a.no_pma:
        out["pma_ablation"] = pma_ablation(a, dev, lo, hi, timed)
    if not a.no_serve:
        out["serve"] = serving(a, g, S_host)
    return out


def serving(a, g, S):
    """Continuous batching vs one library call per request on the same seeded
    traces: 64 clients with Poisson arrivals, 45% inserts of log-uniform
    1..1e5 fresh keys, 10% deletes of log-uniform 1..1e4 present keys, 45%
    range sums of log-uniform 10..1e6 elements, 16 GB device budget.  A sweep
    of offered rates finds each form's saturation (the throughput it reaches
    when offered far more than it can serve); the headline p50/p99 are
    measured at 70% of the continuous-batching loop's saturation."""
    import torch
    from paper_2305_05055_gb300 import serve

    def point(rate, seed):
        mk = lambda: serve.make_trace(a.serve_requests, rate, seed, S, S)
        plain_g = g.clone()
        torch.cuda.synchronize()
        served = serve.Server(g, mem_budget_bytes=16 << 30).run(mk())
        plain = serve.run_one_at_a_time(plain_g, mk())
        del plain_g
        keep = ("requests_per_s", "p50_ms", "p99_ms", "mean_ms", "max_ms")
        s_ = {k: served[k] for k in keep}
        s_.update(epochs=served["epochs"], max_epoch_requests=served["max_epoch_requests"])
        return {"offered_requests_per_s": rate, "served": s_,
                "one_at_a_time": {k: plain[k] for k in keep}}

    sweep = [point(r, 95 + i) for i, r in enumerate(a.serve_rates)]
    sat_served = max(p["served"]["requests_per_s"] for p in sweep)
    sat_plain = max(p["one_at_a_time"]["requests_per_s"] for p in sweep)
    rate = 0.7 * sat_served
    head = point(rate, 90)
    # a load both forms sustain: 70% of the one-call-per-request saturation
    rate_plain = 0.7 * sat_plain
    low = point(rate_plain, 91)
    return {"requests_per_point": a.serve_requests, "sweep": sweep,
            "saturation_requests_per_s": {"served": sat_served, "one_at_a_time": sat_plain},
            "offered_requests_per_s": rate, "at_offered": head,
            "p50_ms": head["served"]["p50_ms"], "p99_ms": head["served"]["p99_ms"],
            "one_at_a_time_p50_ms": head["one_at_a_time"]["p50_ms"],
            "one_at_a_time_p99_ms": head["one_at_a_time"]["p99_ms"],
            "p99_speedup": head["one_at_a_time"]["p99_ms"] / head["served"]["p99_ms"],
            "throughput_ratio": head["served"]["requests_per_s"] /
                                head["one_at_a_time"]["requests_per_s"],
            "saturation_ratio": sat_served / sat_plain,
            "at_plain_offered": {"offered_requests_per_s": rate_plain,
                                 "p50_ms": low["served"]["p50_ms"],
                                 "p99_ms": low["served"]["p99_ms"],
                                 "one_at_a_time_p50_ms": low["one_at_a_time"]["p50_ms"],
                                 "one_at_a_time_p99_ms": low["one_at_a_time"]["p99_ms"]}}


def pma_ablation(a, dev, lo, hi, timed):
    """The compression ablation (Sec. 6: the CPMA against the uncompressed
    PMA under the same batch algorithm): the same 1e8 uniform keys as an
    uncompressed PMA (codec 1, 8-byte cells) and as the CPMA; bytes per key,
    a 1e6-key insert and delete on warmed clones, range_map over the headline
    queries and a full scan."""
    import torch
    from paper_2305_05055_gb300 import cpma as cp
    from paper_2305_05055_gb300 import workloads as W
    T = lambda x: torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(dev)
    base = T(W.uniform_keys(2, int(a.n), bits=40))
    b = T(W.uniform_keys(808, 10 ** 6, bits=40))
    w = T(W.uniform_keys(809, 10 ** 6, bits=40))
    out = {}
    for name, codec in (("cpma", 0), ("pma", 1)):
        g = cp.CPMA(base, leaf_bytes=a.leaf_bytes, codec=codec)
        ins, dele = [], []
        for _ in range(3):
            c = g.clone()
            c.reserve(10 ** 6)
            c.insert_batch(w)
            c.delete_batch(w)
            flush = flush_l2(dev)
            ms_i, _ = timed(lambda: c.insert_batch(b))
            flush = flush_l2(dev)
            ms_d, _ = timed(lambda: c.delete_batch(b))
            del flush, c
            ins.append(ms_i)
            dele.append(ms_d)
        ms_r, (s_, cnt) = timed(lambda: g.range_map(lo, hi), reps=3)
        ms_s, (s2, c2) = timed(lambda: g.sum(), reps=5)
        out[name] = {"bytes_per_key": g.bytes() / g.size(), "leaves": g.leaves(),
                     "insert_keys_per_s": 10 ** 6 / (statistics.median(ins) / 1e3),
                     "delete_keys_per_s": 10 ** 6 / (statistics.median(dele) / 1e3),
                     "range_elems_per_s": int(cnt.sum().item()) / (ms_r / 1e3),
                     "range_ms": ms_r,
                     "scan_elems_per_s": int(c2.item()) / (ms_s / 1e3),
                     "scan_ms": ms_s, "range_sum_check": int(s_.sum().item())}
        del g
        torch.cuda.synchronize()
    out["same_range_sums"] = out["cpma"].pop("range_sum_check") == out["pma"].pop("range_sum_check")
    return out


def graph_workload(a, dev, timed):
    """F-Graph-style edge set (keys u << 32 | v) on an R-MAT graph with
    2^scale vertices and 16 edges per vertex: build, batch edge inserts,
    a neighbour scan of every vertex (degrees by one range_map, neighbour
    lists by one range_extract) and a BFS (edges scanned per second)."""
    import torch
    from paper_2305_05055_gb300 import graph
    from paper_2305_05055_gb300 import workloads as W
    scale = int(a.graph_scale)
    nv, ne = 1 << scale, 16 << scale
    # warm-up on a small graph: the first use of the torch operations that
    # prepare keys and frontiers can compile kernels for this GPU
    ws, wd = W.rmat_edges(3, 10, 1 << 14)
    warm = graph.EdgeSet(ws, wd, device=dev)
    warm.bfs(int(ws[0]), 1 << 10)
    warm.neighbors(torch.arange(1 << 10, device=dev))
    del warm
    torch.cuda.synchronize()
    src, dst = W.rmat_edges(7, scale, ne)
    t0 = time.perf_counter()
    es = graph.EdgeSet(src, dst, device=dev)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    del src, dst
    m0 = es.num_edges()
    batches = [W.rmat_edges(100 + i, scale, 10 ** 6) for i in range(5)]
    bk = [es._vkeys(s_, d_) for s_, d_ in batches]
    es.g.reserve(10 ** 6)
    ins = []
    for k_ in bk:
        ms, _ = timed(lambda: es.g.insert_batch(k_))
        ins.append(ms)
    verts = torch.arange(nv, dtype=torch.int64, device=dev)
    ms_deg, deg = timed(lambda: es.degrees(verts), reps=3)
    ms_nb, (off, nb) = timed(lambda: es.neighbors(verts), reps=3)
    m = es.num_edges()
    assert int(off[-1].item()) == m == int(deg.sum().item())
    root = int(torch.argmax(deg).item())
    es.bfs(root, nv)  # untimed warm-up
    ms_bfs, lvl = timed(lambda: es.bfs(root, nv))
    reached = lvl >= 0
    scanned = int(deg[reached].sum().item())
    return {"scale": scale, "vertices": nv, "edges_generated": ne, "edges_after_build": m0,
            "build_s": build_s, "edges": m, "bytes_per_edge": es.g.bytes() / m,
            "insert_edges_per_s": 10 ** 6 * len(ins) / (sum(ins) / 1e3),
            "degrees_all_vertices_ms": ms_deg,
            "neighbors_all_vertices_ms": ms_nb,
            "neighbor_scan_edges_per_s": m / (ms_nb / 1e3),
            "bfs_ms": ms_bfs, "bfs_levels": int(lvl.max().item()),
            "bfs_reached": int(reached.sum().item()),
            "bfs_edges_scanned_per_s": scanned / (ms_bfs / 1e3)}


def skew(a, dev, T, timed):
    """Skewed updates: 5e7 keys uniform in [0, 2^34), then 100 rounds of 1e5
    zipfian (0.99, 2^34 universe, scattered ranks) inserts + 5e4 deletes of
    present keys; device time per round and final bytes/key.  Those rounds
    change the set by under a tenth, within the root bounds, so growth and
    shrink at this scale are exercised after them: net-growing rounds of 1e6
    fresh uniform keys of the same universe until the array has grown twice,
    then net-shrinking rounds of 2e6 deletes of the initial keys until it
    has shrunk twice."""
    import torch
    from paper_2305_05055_gb300 import cpma as cp
    from paper_2305_05055_gb300 import workloads as W
    n0, rounds, ki, kd = int(5e7), int(a.skew_rounds), 10 ** 5, 5 * 10 ** 4
    base = W.uniform_keys(4, n0, bits=34)
    S = np.sort(base)
    S = S[np.concatenate([[True], S[1:] != S[:-1]])]  # distinct keys (np.unique is slow here)
    g = cp.CPMA(T(base), leaf_bytes=a.leaf_bytes)
    del base
    L0, b0 = g.leaves(), g.bytes()
    nprof = 10  # rounds after the timed ones, profiled for the phase split
    ins = T(W.zipf_keys(44, (rounds + nprof) * ki, bits=34))
    dels = T(S[W.permuted_indices(S.size, (rounds + nprof) * kd, 45)])
    del S
    per = []
    for r in range(rounds):  # timed without the profiler's event records
        ms, _ = timed(lambda: (g.insert_batch(ins[r * ki:(r + 1) * ki]),
                               g.delete_batch(dels[r * kd:(r + 1) * kd])))
        per.append(ms)
    g.profile(True)
    for r in range(rounds, rounds + nprof):
        g.insert_batch(ins[r * ki:(r + 1) * ki])
        g.delete_batch(dels[r * kd:(r + 1) * kd])
    prof = g.profile_read()
    g.profile(False)
    L_rounds = g.leaves()
    size_rounds, bpk_rounds = g.size(), g.bytes() / max(1, g.size())
    # growth and shrink at this scale
    resize = {"grow": [], "shrink": []}
    Ls, r = g.leaves(), 0
    while len(resize["grow"]) < 2 and r < 60:
        # fresh keys of the same 2^34 universe (zipfian draws repeat their
        # hot keys and barely grow the set)
        zb = T(W.uniform_keys(4400 + r, 2 * 10 ** 6, bits=34))
        ms, _ = timed(lambda: g.insert_batch(zb))
        r += 1
        if g.leaves() != Ls:
            resize["grow"].append({"round": r, "ms": ms, "leaves": [Ls, g.leaves()],
                                   "size": g.size()})
            Ls = g.leaves()
    grow_rounds = r
    del dels
    # then delete everything, 2e6 keys a round: the initial keys, then the
    # grown ones, until the array has shrunk twice
    S0 = np.sort(W.uniform_keys(4, n0, bits=34))
    ns0 = (S0.size + 2 * 10 ** 6 - 1) // (2 * 10 ** 6)
    chunk = lambda q: (S0[q * 2 * 10 ** 6:(q + 1) * 2 * 10 ** 6] if q < ns0 else
                       W.uniform_keys(4400 + q - ns0, 2 * 10 ** 6, bits=34))
    r = 0
    while len(resize["shrink"]) < 2 and r < ns0 + grow_rounds:
        db = T(chunk(r))
        ms, _ = timed(lambda: g.delete_batch(db))
        r += 1
        if g.leaves() != Ls:
            resize["shrink"].append({"round": r, "ms": ms, "leaves": [Ls, g.leaves()],
                                     "size": g.size()})
            Ls = g.leaves()
    resize.update(grow_rounds=grow_rounds, shrink_rounds=r, leaves_end=g.leaves(),
                  size_end=g.size(), bytes_per_key_end=g.bytes() / max(1, g.size()))
    per_s = sorted(per)
    return {"rounds": rounds, "insert_per_round": ki, "delete_per_round": kd,
            "round_ms_median": statistics.median(per), "round_ms_p99": per_s[int(0.99 * (len(per) - 1))],
            "round_ms_max": per_s[-1], "total_ms": sum(per),
            "keys_per_s": rounds * (ki + kd) / (sum(per) / 1e3),
            "leaves_start": L0, "leaves_after_rounds": L_rounds, "size_end": size_rounds,
            "bytes_per_key_end": bpk_rounds,
            "bytes_per_key_start": b0 / n0,
            "phases_ms_per_round": {p: prof[p]["ms"] / nprof for p in prof if prof[p]["ms"] > 0},
            "phases_note": "from %d profiled rounds after the timed ones (the profiler's event "
                           "records are not in the timed rounds); merge_lane overlaps merge" % nprof,
            "growth_and_shrink": resize}


def pipelined(a, g, dev, T, nsteps=10):
    """A stream of insert batches in the API's pipelined form: each batch is
    sorted by cpma_sort_batch on a second handle (its own sort scratch) and
    stream while the batch before it is merged, then inserted with sorted = 1.
    Both forms run on device-to-device clones of the headline state with the
    same fresh batches, scratch reserved and graphs on; the timed region
    (CUDA events on the update stream, after a synchronise) covers every
    sort and every insert."""
    import torch
    from paper_2305_05055_gb300 import cpma as cp
    from paper_2305_05055_gb300 import workloads as W
    k = int(a.batch)
    batches = [T(W.uniform_keys(6 * 10 ** 7 + i, k, bits=40)) for i in range(nsteps + 1)]
    warm = batches[-1]
    comp = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=dev)
    sorter = cp.CPMA(T(W.uniform_keys(7, 1000, bits=40)))
    sorter.reserve(k)
    sbuf = [torch.empty(k, dtype=torch.int64, device=dev) for _ in range(2)]
    res = {}
    for mode in ("sequential", "pipelined"):
        c = g.clone()
        c.reserve(k)
        c.use_graphs(1 << 21)
        ws, _ = cp.cpma_sort_batch(sorter.handle, warm, keys_out=sbuf[0])
        for srt, b in ((False, warm), (True, ws)):  # capture both graphs, same set after
            c.insert_batch(b, sorted=srt)
            c.delete_batch(b, sorted=srt)
        added = torch.zeros(1, dtype=torch.int64, device=dev)
        sorted_ev = [torch.cuda.Event() for _ in range(2)]
        freed_ev = [torch.cuda.Event() for _ in range(2)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(comp)
        if mode == "sequential":
            for i in range(nsteps):
                cp.cpma_insert_batch(c.handle, batches[i], False, added)
        else:
            side.wait_event(e0)
            cp.cpma_sort_batch(sorter.handle, batches[0], keys_out=sbuf[0], stream=side)
            sorted_ev[0].record(side)
            for i in range(nsteps):
                b = i & 1
                if i + 1 < nsteps:
                    side.wait_event(freed_ev[b ^ 1])  # that buffer's last insert is done
                    cp.cpma_sort_batch(sorter.handle, batches[i + 1], keys_out=sbuf[b ^ 1],
                                       stream=side)
                    sorted_ev[b ^ 1].record(side)
                comp.wait_event(sorted_ev[b])
                cp.cpma_insert_batch(c.handle, sbuf[b], True, added)
                freed_ev[b].record(comp)
        e1.record(comp)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[mode] = {"keys_per_s": nsteps * k / (ms / 1e3), "ms_per_step": ms / nsteps,
                     "size_after": c.size()}
        del c
    res["same_set"] = res["sequential"]["size_after"] == res["pipelined"]["size_after"]
    res["speedup"] = res["pipelined"]["keys_per_s"] / res["sequential"]["keys_per_s"]
    res["note"] = ("the next batch sorted on a second handle and stream while the current one "
                   "is merged; batches of the headline size into a clone of the headline state "
                   "after its timed steps; the merge fills every SM, so the sort overlaps "
                   "only partly")
    return res


def flush_l2(dev):
    import torch
    buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    buf.fill_(1)  # larger than the 129 MB L2
    return buf


def sweep(a, g, dev, T, timed):
    """Batch-insert sweep at n = 1e8: for k = 1e3 .. 1e7 fresh uniform keys,
    one untimed warm-up trial and `--sweep-trials` timed ones, each on a
    device-to-device clone of the 1e8 state (clone not timed) whose scratch
    is reserved for k and whose update graphs (graph mode) are warm: a warm-up
    insert + delete of another batch of the same size first, which leaves the
    same set.  Then the insert of the trial's batch and the delete of the
    same keys, each timed alone after an L2 flush.  Reported: medians, launch
    by launch and with the front segment as a CUDA graph; inserts of up to
    4096 keys take the point path in both, so for those sizes a third form
    times the batch algorithm alone (point path off, graphs on)."""
    import torch
    from paper_2305_05055_gb300 import workloads as W
    rows = []
    for kk in (10 ** 3, 10 ** 4, 10 ** 5, 10 ** 6, 10 ** 7):
        res = {"batch": kk}
        batches = [T(W.uniform_keys(3 * 10 ** 7 + 100 * t + kk % 97, kk, bits=40))
                   for t in range(a.sweep_trials + 2)]
        modes = ("eager", "graph") + (("batch_graph",) if kk <= 4096 else ())
        for mode in modes:
            ins_ms, del_ms, added = [], [], []
            for t in range(a.sweep_trials + 1):
                c = g.clone()
                c.reserve(kk)
                c.use_graphs((1 << 31) - 1 if mode != "eager" else 0)
                if mode == "batch_graph":
                    c.set_point_max(0)
                w = batches[-1]
                c.insert_batch(w)
                c.delete_batch(w)
                b = batches[t]
                flush = flush_l2(dev)
                ms_i, ad = timed(lambda: c.insert_batch(b))
                flush = flush_l2(dev)
                ms_d, rm = timed(lambda: c.delete_batch(b))
                del flush
                if t:
                    ins_ms.append(ms_i)
                    del_ms.append(ms_d)
                    added.append(int(ad.item()))
                del c
            mi, md = statistics.median(ins_ms), statistics.median(del_ms)
            res[mode] = {"insert_ms": mi, "delete_ms": md,
                         "insert_keys_per_s": kk / (mi / 1e3),
                         "delete_keys_per_s": kk / (md / 1e3),
                         "insert_ms_min": min(ins_ms), "delete_ms_min": min(del_ms)}
        res["insert_keys_per_s"] = max(res[m]["insert_keys_per_s"] for m in modes)
        res["delete_keys_per_s"] = max(res[m]["delete_keys_per_s"] for m in modes)
        rows.append(res)
        del batches
    return rows


if __name__ == "__main__":
    sys.exit(main())
