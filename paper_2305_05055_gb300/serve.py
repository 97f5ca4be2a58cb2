"""Continuous-batching request loop over a device-resident CPMA.

Clients send insert, delete and range-sum requests.  The loop runs in epochs:

1. every request that has arrived is admitted, in arrival order, while the
   device memory it needs fits the budget (structure + library scratch +
   admitted payloads); the rest wait for the next epoch.  The budget is also
   the library's own memory cap (cpma_set_mem_budget): an update whose
   reservation would exceed it is refused before it changes anything
   (CPMA_ENOMEM), and the loop then defers that run and every request
   admitted after it to the next epoch, which admits them again at the
   front; a single update that does not fit even alone completes with the
   result "ENOMEM";
2. the admitted updates are cut into runs of consecutive requests of the same
   kind; each run is one tagged batch (the library credits every key it adds
   or removes to the request of its first occurrence), so each request's
   result equals running the requests one after another in arrival order;
3. the batch of the first run is sorted on the update stream while the
   previous epoch's range launch still runs on the read stream (sorting does
   not touch the structure); the update stream then waits for those reads
   before it changes the structure;
4. all range requests of the epoch go out as one range_map launch on the read
   stream after the epoch's updates, and complete when that launch does.

Results are therefore those of a serial order: epochs in order; inside an
epoch the updates in arrival order, then the epoch's reads.  The epoch log
records that order so tests can replay it request by request.

Latency of a request = completion time - arrival time on the loop's clock.
:func:`run_one_at_a_time` serves the same trace with one library call per
request (the plain CPMA), for comparison.
"""
from __future__ import annotations

import math
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import cpma as cp
from . import workloads as W


@dataclass
class Request:
    rid: int
    kind: str                      # "insert" | "delete" | "range"
    arrival: float                 # seconds after the start of the trace
    keys: np.ndarray | None = None  # uint64 (insert / delete)
    lo: int = 0                    # range [lo, hi)
    hi: int = 0
    client: int = 0
    result: object = None          # added / removed count, or (sum, count)
    done: float = math.nan

    def device_bytes(self) -> int:
        """Device memory an admitted request may hold until it completes:
        its payload plus the library's per-key scratch for the update path
        (sort ping-pong, route flags and scans, touched-leaf records)."""
        if self.kind == "range":
            return 96
        return 160 * int(self.keys.size) + 64


@dataclass
class EpochLog:
    runs: list = field(default_factory=list)    # [(kind, [rid, ...]), ...] in order
    reads: list = field(default_factory=list)   # [rid, ...] evaluated after the runs


def make_trace(n_requests: int, rate: float, seed: int, present_keys: np.ndarray,
               sorted_keys: np.ndarray, clients: int = 64, max_insert: int = 10 ** 5,
               max_delete: int = 10 ** 4, min_width: int = 10, max_width: int = 10 ** 6,
               p_insert: float = 0.45, p_delete: float = 0.10) -> list:
    """Poisson arrivals of `rate` requests/s from `clients` clients; kinds drawn
    with probabilities p_insert / p_delete / rest range.  Inserts: log-uniform
    1..max_insert fresh uniform 40-bit keys; deletes: log-uniform
    1..max_delete keys drawn from present_keys; ranges: rank-based with
    log-uniform width min_width..max_width elements over sorted_keys."""
    u = W.uniform01(seed, n_requests)
    gaps = -np.log1p(-u) / rate
    arrivals = np.cumsum(gaps)
    kinds_u = W.uniform01(seed + 1, n_requests)
    client = (W.splitmix64(seed + 2, n_requests) % np.uint64(clients)).astype(np.int64)
    ins_sizes = W.log_uniform_int(seed + 3, n_requests, 1, max_insert)
    del_sizes = W.log_uniform_int(seed + 4, n_requests, 1, max_delete)
    lo, hi, _ = W.range_queries_by_rank(sorted_keys, seed + 5, n_requests, min_width, max_width)
    out, ins_off, del_off = [], 0, 0
    for i in range(n_requests):
        if kinds_u[i] < p_insert:
            k = int(ins_sizes[i])
            keys = W.uniform_keys(seed + 6, k, bits=40, offset=ins_off)
            ins_off += k
            out.append(Request(i, "insert", float(arrivals[i]), keys=keys, client=int(client[i])))
        elif kinds_u[i] < p_insert + p_delete:
            k = int(del_sizes[i])
            idx = W.permuted_indices(present_keys.size, k, seed + 7, del_off)
            del_off += k
            out.append(Request(i, "delete", float(arrivals[i]), keys=present_keys[idx],
                               client=int(client[i])))
        else:
            out.append(Request(i, "range", float(arrivals[i]), lo=int(lo[i]), hi=int(hi[i]),
                               client=int(client[i])))
    return out


class Server:
    """Continuous-batching loop over one CPMA (see the module docstring)."""

    def __init__(self, g: "cp.CPMA", mem_budget_bytes: int = 16 << 30,
                 max_epoch_requests: int = 1024):
        self.g = g
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.budget = int(mem_budget_bytes)
        self.max_epoch = int(max_epoch_requests)
        self.s_upd = torch.cuda.Stream()
        self.s_read = torch.cuda.Stream()
        self.epochs: list[EpochLog] = []
        self.stats = dict(epochs=0, admitted=0, deferred=0, deferred_runs=0, rejected=0,
                          max_epoch_requests=0)
        g.set_mem_budget(self.budget)
        # most requests per run: halved when the library refuses a run for
        # memory, doubled back after an epoch without refusal
        self.run_cap = self.max_epoch
        # pinned staging for a run's keys and tags, reused: every run's copy
        # has completed before the next run is staged (each run ends with a
        # wait on the update stream)
        self._pin_keys = torch.empty(0, dtype=torch.int64).pin_memory()
        self._pin_tags = torch.empty(0, dtype=torch.int32).pin_memory()

    def _staging(self, n: int):
        if self._pin_keys.numel() < n:
            cap = max(n, 2 * self._pin_keys.numel(), 1 << 16)
            self._pin_keys = torch.empty(cap, dtype=torch.int64).pin_memory()
            self._pin_tags = torch.empty(cap, dtype=torch.int32).pin_memory()
        return self._pin_keys[:n], self._pin_tags[:n]

    def _admit(self, waiting: deque, now: float) -> list:
        used = self.g.bytes() * 3  # structure plus the library's scratch and a resize
        batch = []
        while waiting and len(batch) < self.max_epoch:
            r = waiting[0]
            if r.arrival > now:
                break
            need = r.device_bytes()
            if batch and used + need > self.budget:
                self.stats["deferred"] += 1
                break
            used += need
            batch.append(waiting.popleft())
        return batch

    def _runs(self, batch: list) -> list:
        runs = []
        for r in batch:
            if r.kind == "range":
                continue
            if runs and runs[-1][0] == r.kind and len(runs[-1][1]) < self.run_cap:
                runs[-1][1].append(r)
            else:
                runs.append((r.kind, [r]))
        return runs

    def _prepare_run(self, reqs: list):
        sizes = [r.keys.size for r in reqs]
        n = sum(sizes)
        pk, pt = self._staging(n)
        np.concatenate([r.keys.view(np.int64) for r in reqs], out=pk.numpy())
        pt.numpy()[:] = np.repeat(np.arange(len(reqs), dtype=np.int32), sizes)
        with torch.cuda.stream(self.s_upd):
            dk = pk.to(self.dev, non_blocking=True)
            dt = pt.to(self.dev, non_blocking=True)
            sk, st = cp.cpma_sort_batch(self.g.handle, dk, dt, stream=self.s_upd)
        return sk, st

    def run(self, trace: list, clock=time.perf_counter) -> dict:
        waiting = deque(sorted(trace, key=lambda r: r.arrival))
        inflight = []  # (event, [requests], sums, counts, inputs kept alive)
        t0 = clock()
        reads_done = None
        while waiting or inflight:
            now = clock() - t0
            # complete finished reads
            still = []
            for ev, reqs, sums, cnts, keep in inflight:
                if ev.query():
                    s = cp.to_u64(sums)
                    c = cp.to_u64(cnts)
                    t = clock() - t0
                    for i, r in enumerate(reqs):
                        r.result = (int(s[i]), int(c[i]))
                        r.done = t
                else:
                    still.append((ev, reqs, sums, cnts, keep))
            inflight = still
            batch = self._admit(waiting, now)
            if not batch:
                if inflight:
                    inflight[0][0].synchronize()
                elif waiting:
                    wait = waiting[0].arrival - (clock() - t0)
                    if wait > 0:
                        time.sleep(min(wait, 0.002))
                continue
            self.stats["epochs"] += 1
            self.stats["max_epoch_requests"] = max(self.stats["max_epoch_requests"], len(batch))
            log = EpochLog()
            runs = self._runs(batch)
            prepared = None
            if runs:  # sorted while the previous epoch's reads still run
                try:
                    prepared = self._prepare_run(runs[0][1])
                except cp.CPMAError as e:
                    if e.code != cp.CPMA_ENOMEM:
                        raise
            # the structure changes only after the previous epoch's reads
            if reads_done is not None:
                self.s_upd.wait_event(reads_done)
            cut = len(batch)  # requests of the batch served in this epoch
            for ri, (kind, reqs) in enumerate(runs):
                try:
                    sk, st = (prepared if ri == 0 and prepared is not None
                              else self._prepare_run(reqs))
                    fn = (cp.cpma_insert_batch_tagged if kind == "insert"
                          else cp.cpma_delete_batch_tagged)
                    with torch.cuda.stream(self.s_upd):
                        counts = torch.empty(len(reqs), dtype=torch.int64, device=self.dev)
                        fn(self.g.handle, sk, st, len(reqs), counts=counts, sorted=True,
                           stream=self.s_upd)
                        res = counts.cpu()
                except cp.CPMAError as e:
                    if e.code != cp.CPMA_ENOMEM:
                        raise
                    # refused before any change: this run and everything
                    # admitted after it go back to the front of the queue
                    cut = batch.index(reqs[0])
                    if cut == 0 and len(reqs) == 1:
                        reqs[0].result = "ENOMEM"   # too large even alone
                        reqs[0].done = clock() - t0
                        self.stats["rejected"] += 1
                        cut = 1
                    self.stats["deferred_runs"] += 1
                    self.run_cap = max(1, len(reqs) // 2)
                    waiting.extendleft(reversed(batch[cut:]))
                    break
                t = clock() - t0
                for i, r in enumerate(reqs):
                    r.result = int(res[i])
                    r.done = t
                log.runs.append((kind, [r.rid for r in reqs]))
            self.stats["admitted"] += cut
            if cut == len(batch):
                self.run_cap = min(self.max_epoch, 2 * self.run_cap)
            reads = [r for r in batch[:cut] if r.kind == "range"]
            if reads:
                upd_done = torch.cuda.Event()
                upd_done.record(self.s_upd)
                self.s_read.wait_event(upd_done)
                lo = np.array([r.lo for r in reads], dtype=np.uint64)
                hi = np.array([r.hi for r in reads], dtype=np.uint64)
                with torch.cuda.stream(self.s_read):
                    dlo = torch.from_numpy(lo.view(np.int64)).to(self.dev, non_blocking=True)
                    dhi = torch.from_numpy(hi.view(np.int64)).to(self.dev, non_blocking=True)
                    sums, cnts = cp.cpma_range_map(self.g.handle, dlo, dhi, stream=self.s_read)
                    ev = torch.cuda.Event()
                    ev.record(self.s_read)
                reads_done = ev
                inflight.append((ev, reads, sums, cnts, (dlo, dhi)))
                log.reads = [r.rid for r in reads]
            self.epochs.append(log)
        torch.cuda.synchronize()
        return summarize(trace, clock() - t0, self.stats)


def run_one_at_a_time(g: "cp.CPMA", trace: list, clock=time.perf_counter) -> dict:
    """The plain CPMA, one library call per request, in arrival order."""
    dev = torch.device("cuda", torch.cuda.current_device())
    t0 = clock()
    for r in sorted(trace, key=lambda r: r.arrival):
        wait = r.arrival - (clock() - t0)
        if wait > 0:
            time.sleep(wait)
        if r.kind == "range":
            lo = torch.tensor([np.int64(np.uint64(r.lo).view(np.int64))], device=dev)
            hi = torch.tensor([np.int64(np.uint64(r.hi).view(np.int64))], device=dev)
            s, c = g.range_map(lo, hi)
            r.result = (int(cp.to_u64(s)[0]), int(cp.to_u64(c)[0]))
        else:
            k = torch.from_numpy(r.keys.view(np.int64)).to(dev)
            out = g.insert_batch(k) if r.kind == "insert" else g.delete_batch(k)
            r.result = int(out.item())
        r.done = clock() - t0
    torch.cuda.synchronize()
    return summarize(trace, clock() - t0, {})


def summarize(trace: list, wall: float, extra: dict) -> dict:
    lat = np.array([r.done - r.arrival for r in trace]) * 1e3
    keys = sum(int(r.keys.size) for r in trace if r.keys is not None)
    out = dict(requests=len(trace), wall_s=wall, requests_per_s=len(trace) / wall,
               update_keys_per_s=keys / wall,
               p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
               max_ms=float(lat.max()), mean_ms=float(lat.mean()),
               offered_requests_per_s=len(trace) / max(trace[-1].arrival, 1e-9))
    for kind in ("insert", "delete", "range"):
        lk = np.array([r.done - r.arrival for r in trace if r.kind == kind]) * 1e3
        if lk.size:
            out["p99_ms_" + kind] = float(np.percentile(lk, 99))
    out.update(extra)
    return out
