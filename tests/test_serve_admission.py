"""Scheduling rules of the serving loop, on the CPU with a fake executor.

The executor records which requests overlap in time; the tests check FIFO
admission, the device-memory budget (slots keep their largest workspace),
reuse of a slot's resident problem by key, rejection of oversized requests,
error isolation, that a request is admitted while others still run, and that
idle slots' resident workspaces are released when a larger request would
otherwise never fit (no deadlock once every slot has grown).
"""
import threading
import time

import pytest

from paper_1901_05188_gb300.serve import GeneoServer, latency_summary


class FakeExecutor:
    def __init__(self, duration=0.05, fail_rids=()):
        self.duration = duration
        self.fail_rids = set(fail_rids)
        self.lock = threading.Lock()
        self.running = set()
        self.overlaps = []          # (rid, set of rids running when it started)
        self.calls = []             # (slot, rid, reuse)
        self.released = []          # (slot, rids running at the time)

    def __call__(self, slot, req, reuse):
        with self.lock:
            self.overlaps.append((req.rid, set(self.running)))
            self.running.add(req.rid)
            self.calls.append((slot, req.rid, reuse))
        d = req.problem.get("duration", self.duration)
        time.sleep(d)
        with self.lock:
            self.running.discard(req.rid)
        if req.rid in self.fail_rids:
            raise RuntimeError("planted failure")
        req.u = ("solution", req.problem["id"])
        req.stats = {"iterations": 1}


    def release(self, slot):
        with self.lock:
            self.released.append((slot, set(self.running)))


def mem_of(req):
    return req.problem["mem"]


def make_server(slots, budget, **kw):
    ex = FakeExecutor(**kw)
    return GeneoServer(slots=slots, mem_budget=budget, executor=ex, memory_of=mem_of), ex


def test_fifo_and_concurrency():
    srv, ex = make_server(slots=3, budget=100)
    reqs = [srv.submit({"id": i, "mem": 10}) for i in range(9)]
    for r in reqs:
        r.wait(10)
    srv.close()
    assert all(r.error is None for r in reqs)
    starts = [rid for rid, _ in ex.overlaps]
    assert starts == sorted(starts)                      # FIFO
    assert srv.peak_inflight == 3
    assert max(len(o) for _, o in ex.overlaps) == 2      # three running together


def test_memory_budget_limits_concurrency():
    # 4 slots but memory for only two 40-byte requests at a time
    srv, ex = make_server(slots=4, budget=90)
    reqs = [srv.submit({"id": i, "mem": 40}) for i in range(6)]
    for r in reqs:
        r.wait(10)
    srv.close()
    assert all(r.error is None for r in reqs)
    assert srv.peak_inflight == 2
    assert max(len(o) for _, o in ex.overlaps) <= 1
    assert srv.peak_mem <= 90


def test_slots_keep_their_workspace():
    # a 60-byte request grows slot 0; later 30-byte requests cannot take a
    # second slot while 60 + 30 + 30 > 100, but fit once placed on slot 0
    srv, ex = make_server(slots=2, budget=100, duration=0.02)
    big = srv.submit({"id": 0, "mem": 60})
    big.wait(10)
    small = [srv.submit({"id": i, "mem": 30}) for i in range(1, 5)]
    for r in small:
        r.wait(10)
    srv.close()
    assert srv.mem_in_use <= 100
    assert srv.peak_mem <= 100
    # after the big one, slot 0 holds 60; slot 1 may grow to 30 (total 90)
    assert sorted(srv.slot_mem) == [30, 60]


def test_oversized_request_rejected_without_blocking():
    srv, ex = make_server(slots=2, budget=50)
    bad = srv.submit({"id": 0, "mem": 51})
    ok = srv.submit({"id": 1, "mem": 10})
    assert bad.wait(1).error is not None and "budget" in bad.error
    assert ok.wait(10).error is None
    srv.close()
    assert [rid for _, rid, _ in ex.calls] == [ok.rid]


def test_resident_problem_reused_by_key():
    srv, ex = make_server(slots=2, budget=100, duration=0.01)
    a1 = srv.submit({"id": "A", "mem": 20}, key="A")
    a1.wait(10)
    a2 = srv.submit({"id": "A", "mem": 20}, key="A")
    a2.wait(10)
    b = srv.submit({"id": "B", "mem": 20}, key="B", prec=1)
    b.wait(10)
    b_fp64 = srv.submit({"id": "B", "mem": 20}, key="B", prec=0)   # other precision: no reuse
    b_fp64.wait(10)
    srv.close()
    assert (a1.reused, a2.reused, b.reused, b_fp64.reused) == (False, True, False, False)
    assert a2.slot == a1.slot
    assert b.slot != a1.slot                # the slot holding A is not evicted while another is free


def test_failure_is_isolated_and_slot_not_reused():
    srv, ex = make_server(slots=1, budget=100, duration=0.01, fail_rids={0})
    r0 = srv.submit({"id": 0, "mem": 10}, key="K")
    r1 = srv.submit({"id": 1, "mem": 10}, key="K")
    r0.wait(10)
    r1.wait(10)
    srv.close()
    assert r0.error is not None and "planted failure" in r0.error
    assert r1.error is None and not r1.reused      # failed resident state is not reused


def test_continuous_admission_while_running():
    # a long request holds one slot; short ones keep flowing through the other
    srv, ex = make_server(slots=2, budget=100)
    long_r = srv.submit({"id": "long", "mem": 10, "duration": 0.5})
    time.sleep(0.02)
    shorts = [srv.submit({"id": i, "mem": 10, "duration": 0.02}) for i in range(5)]
    for r in shorts:
        r.wait(10)
    assert not long_r._done.is_set()             # all short ones finished first
    long_r.wait(10)
    srv.close()
    assert all(long_r.rid in o for rid, o in ex.overlaps if rid in {r.rid for r in shorts})


def test_cancel_queued_request():
    srv, ex = make_server(slots=1, budget=100)
    first = srv.submit({"id": 0, "mem": 10, "duration": 0.2})
    queued = srv.submit({"id": 1, "mem": 10})
    time.sleep(0.02)
    assert srv.cancel(queued)
    first.wait(10)
    srv.close()
    assert queued.error == "cancelled"
    assert [rid for _, rid, _ in ex.calls] == [first.rid]


def test_latency_summary():
    srv, ex = make_server(slots=2, budget=100, duration=0.01)
    reqs = [srv.submit({"id": i, "mem": 10}) for i in range(10)]
    for r in reqs:
        r.wait(10)
    srv.close()
    s = latency_summary(reqs)
    assert s["n"] == 10 and s["failed"] == 0
    assert 0 < s["p50_ms"] <= s["p99_ms"] <= s["max_ms"]
    assert s["solves_per_s"] > 0


def test_repeated_key_waits_for_its_resident_slot():
    # a burst: A, A, B with two slots.  The second A waits for the slot that
    # holds A (reuse) while B takes the other slot.
    srv, ex = make_server(slots=2, budget=100, duration=0.05)
    a1 = srv.submit({"id": "A", "mem": 20}, key="A")
    a2 = srv.submit({"id": "A", "mem": 20}, key="A")
    b = srv.submit({"id": "B", "mem": 20}, key="B")
    for r in (a1, a2, b):
        r.wait(10)
    srv.close()
    assert a2.reused and a2.slot == a1.slot
    assert b.slot != a1.slot and not b.reused
    assert b.t_start < a2.t_start          # B went ahead of the waiting A


def test_idle_slots_released_for_a_larger_request():
    srv, ex = make_server(slots=2, budget=100)
    first = [srv.submit({"id": i, "mem": 45}) for i in range(2)]
    for r in first:
        r.wait(5)
    big = srv.submit({"id": 2, "mem": 70})      # 45 + 45 resident: fits only after releasing both
    big.wait(5)
    srv.close()
    assert big.error is None
    assert srv.evictions == 2
    assert sorted(sl for sl, _ in ex.released) == [0, 1]
    assert all(not running for _, running in ex.released)   # nothing ran on a released slot


def test_no_deadlock_once_every_slot_has_grown():
    srv, ex = make_server(slots=4, budget=100, duration=0.01)
    sizes = [24, 24, 24, 24, 60, 24, 90, 30, 24, 50]
    reqs = [srv.submit({"id": i, "mem": m}) for i, m in enumerate(sizes)]
    for r in reqs:
        r.wait(5)
    srv.close()
    assert all(r.error is None for r in reqs)
    starts = [rid for rid, _ in ex.overlaps]
    assert starts == sorted(starts)                      # still FIFO
    assert srv.peak_mem <= 100


def test_release_waits_for_busy_slots():
    srv, ex = make_server(slots=2, budget=100, duration=0.2)
    a = srv.submit({"id": 0, "mem": 60})
    time.sleep(0.05)
    b = srv.submit({"id": 1, "mem": 60})            # cannot start while a holds 60
    for r in (a, b):
        r.wait(5)
    srv.close()
    assert a.error is None and b.error is None
    assert 1 not in ex.overlaps[0][1] and 0 not in ex.overlaps[1][1]
