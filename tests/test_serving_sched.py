"""Host logic of the serving loop: FIFO admission by device-memory footprint.

A fake runner stands in for the library, so these run without a GPU."""
import threading
import time

import numpy as np

from paper_2310_12000_gb300 import serving


def _req(rid, footprint):
    r = serving.Request(rid=rid, locs=np.zeros((10, 2)), order=np.arange(10, dtype=np.int32), y=np.zeros(10),
                        F=None, cov=1, sigma2=1.0, rho=0.1, m=5, lik=0, test_locs=None, opts={})
    r.footprint = footprint
    return r


def test_admission_respects_budget_and_fifo():
    lock = threading.Lock()
    live = {"bytes": 0, "peak": 0}
    order = []

    def runner(ctx, req):
        with lock:
            live["bytes"] += req.footprint
            live["peak"] = max(live["peak"], live["bytes"])
            order.append(req.rid)
        time.sleep(0.002 * (1 + req.rid % 3))
        with lock:
            live["bytes"] -= req.footprint
        return {"lml": float(req.rid)}

    srv = serving.Server(slots=4, budget_bytes=100, slot_capacity=100, make_ctx=lambda s: None,
                         runner=runner).start()
    sizes = [60, 30, 30, 50, 10, 90, 20, 20, 40, 70] * 3
    for i, fp in enumerate(sizes):
        srv.submit(_req(i, fp))
    res = srv.drain()
    assert [r.rid for r in res] == list(range(len(sizes)))
    assert all(r.error is None and r.lml == r.rid for r in res)
    assert live["peak"] <= 100 and srv.sched.peak_in_use <= 100
    assert order == sorted(order)            # admitted strictly first-come first-served
    assert srv.sched.peak_running <= 4
    assert all(r.t_done >= r.t_admit >= r.t_arrival for r in res)


def test_oversized_request_rejected_and_failures_recorded():
    def runner(ctx, req):
        if req.rid == 2:
            raise RuntimeError("boom")
        return {"lml": 0.0}

    srv = serving.Server(slots=2, budget_bytes=100, slot_capacity=80, make_ctx=lambda s: None, runner=runner).start()
    assert srv.submit(_req(0, 50))
    assert not srv.submit(_req(1, 90))       # above one slot's capacity
    assert srv.submit(_req(2, 10))
    res = {r.rid: r for r in srv.drain()}
    assert res[1].error.startswith("rejected")
    assert "boom" in res[2].error and res[0].error is None
    s = serving.latency_summary(list(res.values()), 1.0)
    assert s["completed"] == 1 and s["failed"] == 2


def test_footprint_grows_with_size():
    a = serving.footprint_bytes(1000, 20)
    b = serving.footprint_bytes(200_000, 20)
    c = serving.footprint_bytes(200_000, 20, k=500)
    assert a < b < c
    assert 2e9 < b < 6e9


def test_slot_classes_take_requests_that_fit():
    seen = {}
    lock = threading.Lock()

    def runner(ctx, req):
        with lock:
            seen[req.rid] = ctx
        time.sleep(0.001)
        return {"lml": 0.0}

    caps = [100, 30, 30, 30]          # one large slot, three small ones
    srv = serving.Server(slots=caps, budget_bytes=190, slot_capacity=None,
                         make_ctx=lambda s, cap: cap, runner=runner).start()
    sizes = [90, 10, 20, 80, 25, 5, 100, 30, 15]
    for i, fp in enumerate(sizes):
        assert srv.submit(_req(i, fp))
    assert not srv.submit(_req(99, 101))     # above every slot
    res = {r.rid: r for r in srv.drain()}
    assert all(r.error is None for i, r in res.items() if i != 99)
    for i, fp in enumerate(sizes):
        assert fp <= seen[i]                  # ran on a slot large enough for it
    assert srv.sched.peak_in_use <= 190


def test_start_fails_loudly_when_a_slot_cannot_be_made():
    import pytest

    def make(slot):
        if slot == 1:
            raise RuntimeError("no device memory")
        return None

    srv = serving.Server(slots=3, budget_bytes=100, slot_capacity=100, make_ctx=make, runner=lambda c, r: {})
    with pytest.raises(RuntimeError, match="slot 1"):
        srv.start()


def test_continuous_batching_groups_within_slot_and_budget():
    """Grouped admission: a free slot takes the head of the queue and every later queued
    request with the same options while the group's footprint fits the slot and the budget;
    every request is served exactly once and gets its own result."""
    lock = threading.Lock()
    live = {"bytes": 0, "peak": 0}
    groups = []

    def batch_runner(ctx, reqs):
        fp = sum(r.footprint for r in reqs)
        with lock:
            live["bytes"] += fp
            live["peak"] = max(live["peak"], live["bytes"])
            groups.append([r.rid for r in reqs])
        assert fp <= ctx                          # the slot's capacity
        assert len({str(r.opts) for r in reqs}) == 1
        time.sleep(0.01)
        with lock:
            live["bytes"] -= fp
        return [{"lml": float(r.rid)} for r in reqs]

    srv = serving.Server(slots=[100, 60], budget_bytes=140, slot_capacity=None, make_ctx=lambda s, cap: cap,
                         batch_runner=batch_runner, max_group=5).start()
    sizes = [30, 20, 10, 50, 40, 5, 25, 60, 15, 10, 35, 20] * 2
    for i, fp in enumerate(sizes):
        r = _req(i, fp)
        r.opts = {"t": 8} if i % 7 else {"t": 16}   # two option sets never share a group
        assert srv.submit(r)
    assert not srv.submit(_req(99, 101))
    res = {r.rid: r for r in srv.drain()}
    assert sorted(res) == list(range(len(sizes))) + [99]
    assert all(res[i].error is None and res[i].lml == i for i in range(len(sizes)))
    served = sorted(x for g in groups for x in g)
    assert served == list(range(len(sizes)))       # each request exactly once
    assert max(len(g) for g in groups) > 1 and max(len(g) for g in groups) <= 5
    assert live["peak"] <= 140 and srv.sched.peak_in_use <= 140
    assert srv.groups and sum(srv.groups) == len(sizes)
    for g in groups:                               # each group's head is the oldest request it could take
        assert g[0] == min(g)
    assert all(r.t_done >= r.t_admit >= r.t_arrival for r in res.values() if r.slot >= 0)


def test_group_failure_fails_every_member_and_drain_ends():
    def batch_runner(ctx, reqs):
        if any(r.rid == 3 for r in reqs):
            raise RuntimeError("group boom")
        return [{"lml": 1.0} for _ in reqs]

    srv = serving.Server(slots=1, budget_bytes=100, slot_capacity=100, make_ctx=lambda s: None,
                         batch_runner=batch_runner, max_group=2)
    import pytest
    with pytest.raises(ValueError):
        serving.Server(slots=1, budget_bytes=1, slot_capacity=1, make_ctx=lambda s: None)
    srv.start()
    for i in range(6):
        srv.submit(_req(i, 10))
    res = srv.drain()
    bad = [r.rid for r in res if r.error]
    assert 3 in bad and all("group boom" in r.error for r in res if r.error)
    assert len(bad) <= 2 and len(res) == 6


def test_batch_footprint_covers_members_and_merged_system():
    a = _req(0, 0)
    b = _req(1, 0)
    a.opts = b.opts = {"t": 50, "s": 100}
    one = serving.batch_footprint_bytes([a])
    two = serving.batch_footprint_bytes([a, b])
    assert serving.footprint_bytes(10, 5, n_test=0) < one < two
    assert serving.batch_footprint_bytes([]) == 0
