"""Admission and batching policy of the request server (host logic, no GPU)."""

from paper_2609_16478_b300.inputs import RequestSpec
from paper_2609_16478_b300.serving import Scheduler

MB = 1 << 20


def _req(rid, dim, N, t):
    return RequestSpec(rid, dim, N, (0,) * dim, t)


def _sched(budget, batch=4, nbytes=100 * MB, max_slots=4):
    return Scheduler(budget, lambda k: batch, lambda k, B: nbytes * B // batch, max_slots)


def test_fifo_batches_by_shape():
    s = _sched(10_000 * MB)
    for rid, (dim, N) in enumerate([(2, 128), (3, 64), (2, 128), (2, 128), (2, 128), (2, 128), (3, 64)]):
        s.arrive(_req(rid, dim, N, 0.1 * rid))
    w = s.next_work(1.0)  # 5 queued, at most 4 per batch: a plan of 4
    assert w.key == (2, 128) and [r.rid for r in w.reqs] == [0, 2, 3, 4] and w.new_slot and w.slot.batch == 4
    w2 = s.next_work(1.0)  # oldest waiting head is now request 1 (3D): a plan of 2 for two requests
    assert w2.key == (3, 64) and [r.rid for r in w2.reqs] == [1, 6] and w2.slot.batch == 2
    w3 = s.next_work(1.0)  # a second plan of the busy 2D shape, sized to its one request
    assert w3.key == (2, 128) and [r.rid for r in w3.reqs] == [5] and w3.new_slot and w3.slot.batch == 1
    assert s.next_work(1.0) is None and s.pending() == 0
    s.release(w3, 2.0)
    s.release(w, 2.0)
    s.arrive(_req(9, 2, 128, 2.5))
    w4 = s.next_work(3.0)  # the idle plan of 1 fits exactly: reused, the plan of 4 stays idle
    assert w4.slot is w3.slot and not w4.new_slot and [r.rid for r in w4.reqs] == [9]
    for rid in range(10, 13):
        s.arrive(_req(rid, 2, 128, 3.0))
    w5 = s.next_work(3.5)  # three requests: the idle plan of 4
    assert w5.slot is w.slot and [r.rid for r in w5.reqs] == [10, 11, 12]


def test_budget_waits_then_evicts_lru():
    s = _sched(250 * MB, nbytes=400 * MB)  # single-request plans of 100 MB: room for two
    s.arrive(_req(0, 2, 128, 0.0))
    s.arrive(_req(1, 2, 256, 0.1))
    s.arrive(_req(2, 3, 64, 0.2))
    a = s.next_work(0.0)
    b = s.next_work(0.0)
    assert {a.key, b.key} == {(2, 128), (2, 256)}
    assert s.next_work(0.0) is None  # no room, nothing idle: the 3D request waits
    s.release(b, 5.0)
    s.release(a, 6.0)  # (2,256) is now the least recently used idle plan
    c = s.next_work(7.0)
    assert c.key == (3, 64) and c.new_slot
    ev = s.take_evicted()
    assert [e.key for e in ev] == [(2, 256)] and s.used == 200 * MB


def test_plan_larger_than_budget():
    s = _sched(150 * MB, batch=4, nbytes=400 * MB)  # B = 4 needs 400 MB, B = 1 needs 100 MB
    for rid in range(3):
        s.arrive(_req(rid, 3, 256, rid))
    w = s.next_work(0.0)
    assert w.slot.batch == 1 and len(w.reqs) == 1
    s2 = _sched(50 * MB, batch=1, nbytes=100 * MB)  # even one problem is over budget: runs alone
    s2.arrive(_req(0, 3, 256, 0.0))
    s2.arrive(_req(1, 2, 128, 0.0))
    w = s2.next_work(0.0)
    assert w is not None and s2.next_work(0.0) is None


def test_deadline_drops_expired_queued_requests():
    s = _sched(10_000 * MB, batch=2)
    a = _req(0, 2, 128, 0.0)
    b = _req(1, 2, 128, 0.1)
    b.deadline = 0.5
    c = _req(2, 2, 128, 0.2)
    for r in (a, b, c):
        s.arrive(r)
    w = s.next_work(1.0)  # b's deadline has passed: dropped, a and c batched
    assert [r.rid for r in w.reqs] == [0, 2]
    assert [r.rid for r in s.take_expired()] == [1] and s.take_expired() == []
    assert s.pending() == 0


def test_cancel_withdraws_a_queued_request():
    s = _sched(10_000 * MB, batch=4)
    for rid in range(3):
        s.arrive(_req(rid, 3, 64, 0.1 * rid))
    assert s.cancel(1) and not s.cancel(1) and not s.cancel(99)
    w = s.next_work(1.0)
    assert [r.rid for r in w.reqs] == [0, 2] and w.slot.batch == 2
    assert not s.cancel(0)  # already in a batch: runs to its end
    s.release(w, 2.0)
    assert not w.slot.busy


def test_no_over_admission_while_all_plans_busy():
    """A shape whose plan is busy and whose next plan would exceed the
    budget waits: the bytes in use never pass the budget (one resident plan
    may run alone over it only when nothing else is resident)."""
    s = _sched(300 * MB, batch=1, nbytes=200 * MB, max_slots=4)
    for rid in range(4):
        s.arrive(_req(rid, 2, 256, 0.0))
    w = s.next_work(0.0)
    assert w is not None and s.used == 200 * MB
    assert s.next_work(0.0) is None and s.used <= s.budget  # a second 200 MB plan would not fit
    s.release(w, 1.0)
    w2 = s.next_work(1.5)  # the idle plan is reused
    assert w2.slot is w.slot and s.used == 200 * MB
