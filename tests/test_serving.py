"""The continuous-batching loop: every served result must equal the result of
the same request run alone, one after another in the order the loop
serialised them (its epoch log), both on the CPU oracle and as one library
call per request on the GPU.  All results are integers: exact equality."""
import numpy as np
import pytest
import torch

import oracle
from paper_2305_05055_gb300 import cpma as cp
from paper_2305_05055_gb300 import serve
from paper_2305_05055_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def T(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.uint64)).view(np.int64)).cuda()


def _trace_with_overlaps(S):
    tr = serve.make_trace(500, rate=40000.0, seed=92, present_keys=S, sorted_keys=S,
                          max_insert=3000, max_delete=800, min_width=1, max_width=30000)
    # make requests collide: re-insert the keys of earlier inserts, delete keys
    # an earlier request of the same epoch-sized window inserted, repeat keys
    ins = [r for r in tr if r.kind == "insert"]
    for a, b in zip(ins[::3], ins[1::3]):
        b.keys = np.concatenate([b.keys, a.keys[: a.keys.size // 2], b.keys[:5]])
    dels = [r for r in tr if r.kind == "delete"]
    for d, a in zip(dels, ins[::2]):
        d.keys = np.concatenate([d.keys, a.keys[: 50]])
    return tr


def test_served_results_equal_one_at_a_time():
    assert torch.cuda.is_available()
    base = W.uniform_keys(91, 200000, bits=40)
    S = np.unique(base)
    trace = _trace_with_overlaps(S)
    g = cp.CPMA(T(base), leaf_bytes=512)
    srv = serve.Server(g)
    stats = srv.run(trace)
    assert stats["epochs"] < len(trace)            # requests were coalesced
    assert max(len(e.runs) for e in srv.epochs) >= 1
    check_serial(g, base, trace, srv)


def test_tight_budget_defers_runs_and_keeps_results():
    # All requests arrive at once, nearly all inserts, so the first epoch
    # coalesces them into one large run.  The budget is the most memory a
    # handle held while applying every insert in runs no larger than the
    # largest single request (measured on a probe), plus 1 MiB: the large run is refused by
    # the library (CPMA_ENOMEM, nothing changed), the loop defers it with a
    # smaller run size, and every result still equals its serial replay.  The
    # probe is built like the served handle, so both hold the same scratch.
    base = W.uniform_keys(93, 100000, bits=40)
    S = np.unique(base)
    trace = serve.make_trace(300, rate=1e7, seed=94, present_keys=S, sorted_keys=S,
                             max_insert=3000, max_delete=500, min_width=1, max_width=30000,
                             p_insert=0.9, p_delete=0.05)
    g = cp.CPMA(T(base), leaf_bytes=512)
    ups = [r.keys for r in trace if r.kind != "range"]
    biggest = max(k.size for k in ups)
    allk = np.concatenate([r.keys for r in trace if r.kind == "insert"])
    probe = cp.CPMA(T(base), leaf_bytes=512)
    for i in range(0, allk.size, biggest):     # the loop's form: sorted, tagged runs
        k = T(allk[i:i + biggest])
        tg = torch.zeros(k.numel(), dtype=torch.int32, device="cuda")
        sk, st = cp.cpma_sort_batch(probe.handle, k, tg)
        cp.cpma_insert_batch_tagged(probe.handle, sk, st, 1, sorted=True)
    probe.range_map(T(S[:400]), T(S[1:401]))
    budget = probe.mem_peak() + (1 << 20)
    del probe
    srv = serve.Server(g, mem_budget_bytes=budget)
    stats = srv.run(trace)
    assert stats["deferred_runs"] > 0 and stats["rejected"] == 0, stats
    assert g.mem_held() <= budget
    check_serial(g, base, trace, srv)


def check_serial(g, base, trace, srv):
    """Every served result equals the request run alone in the loop's order."""
    by_id = {r.rid: r for r in trace}
    served = {r.rid: r.result for r in trace}
    # 1. the oracle, one request at a time in the served order
    p = oracle.PlainSet(base)
    order = []
    for ep in srv.epochs:
        for kind, rids in ep.runs:
            for rid in rids:
                r = by_id[rid]
                want = p.insert_batch(r.keys) if kind == "insert" else p.delete_batch(r.keys)
                assert served[rid] == want, (rid, kind)
                order.append(rid)
        if ep.reads:
            lo = np.array([by_id[i].lo for i in ep.reads], np.uint64)
            hi = np.array([by_id[i].hi for i in ep.reads], np.uint64)
            ws, wc = p.range_map(lo, hi)
            for i, rid in enumerate(ep.reads):
                assert served[rid] == (int(ws[i]), int(wc[i])), rid
                order.append(rid)
    assert sorted(order) == sorted(by_id)
    s, c = g.sum()
    assert int(cp.to_u64(s)[0]) == p.sum() and int(c.item()) == len(p) == g.size()
    # 2. the plain library, one call per request, in the same order
    g2 = cp.CPMA(T(base), leaf_bytes=512)
    for rid in order:
        r = by_id[rid]
        if r.kind == "range":
            ss, cc = g2.range_map(T([r.lo]), T([r.hi]))
            alone = (int(cp.to_u64(ss)[0]), int(cp.to_u64(cc)[0]))
        elif r.kind == "insert":
            alone = int(g2.insert_batch(T(r.keys)).item())
        else:
            alone = int(g2.delete_batch(T(r.keys)).item())
        assert alone == served[rid], rid


def test_tagged_batch_credits_first_occurrence():
    base = np.arange(0, 100000, 7, dtype=np.uint64)
    g = cp.CPMA(T(base), leaf_bytes=512)
    keys = np.array([1, 2, 7, 1, 3, 2, 5], np.uint64)    # 7 present; 1, 2 repeated
    tags = torch.tensor([0, 0, 0, 1, 1, 2, 2], dtype=torch.int32, device="cuda")
    counts = cp.cpma_insert_batch_tagged(g.handle, T(keys), tags, 3)
    assert counts.cpu().tolist() == [2, 1, 1]            # {1,2}, {3}, {5}
    keys = np.array([3, 14, 1, 3, 999999], np.uint64)
    tags = torch.tensor([2, 0, 1, 0, 2], dtype=torch.int32, device="cuda")
    counts = cp.cpma_delete_batch_tagged(g.handle, T(keys), tags, 3)
    # sorted: 1(t1) 3(t2) 3(t0) 14(t0) 999999(t2): 3 goes to its first occurrence, t2
    assert counts.cpu().tolist() == [1, 1, 1]
    bad = torch.tensor([0, 5], dtype=torch.int32, device="cuda")
    with pytest.raises(cp.CPMAError):
        cp.cpma_insert_batch_tagged(g.handle, T([10, 11]), bad, 3)
    assert g.size() == base.size + 4 - 3
