"""Continuous-batching request server for the augmented HOC solver.

Requests (a grid, a coefficient and a right-hand side; see
``inputs.request_stream``) arrive over time.  The server keeps, per grid
shape (dim, N), a pool of batched plans resident on the device -- the DST
twiddles, the per-mode tridiagonal factors, the preconditioner symbols and
the Krylov bases stay allocated between requests -- and admits work by an
HBM budget:

  * every shape has a FIFO queue; a worker takes up to B queued requests of
    one shape (B: the shape's largest batch, from the tuner or a default),
    runs them on the smallest idle plan of that shape whose batch is the
    power of two at or above their number (creating it if the pool has room),
    loads each request's coefficient into a slot of the plan
    (``ahoc_plan_load``), masks the unused slots (``ahoc_set_active``) and
    solves the batch in one set of launches (a plan much larger than its
    batch would launch mostly masked blocks);
  * a new plan is allocated only if the pool's device bytes stay within the
    budget, after evicting idle plans of other shapes (least recently used
    first); otherwise the request waits for a plan to free up;
  * several workers, each with its own CUDA stream, run batches of different
    (or the same) shapes at once, so requests that arrive while others are
    on the GPU are admitted as slots free up and their work overlaps.

A problem's result does not depend on the batch it was solved in: batched
plans give every problem the bits of its own single-problem solve.

The admission and batching policy (``Scheduler``) is plain host code with no
device work, so it can be exercised without a GPU.
"""

from __future__ import annotations

import threading
import time
from collections import deque
from dataclasses import dataclass, field
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple

Key = Tuple[int, int]  # (dim, N)


# ----------------------------------------------------------------------------
# host-side policy
# ----------------------------------------------------------------------------

@dataclass
class SlotState:
    key: Key
    batch: int
    nbytes: int
    busy: bool = False
    last_used: float = 0.0
    handle: object = None  # the executor's plan object (None until created)


@dataclass
class Work:
    key: Key
    slot: SlotState
    reqs: list
    new_slot: bool  # the executor must create the slot's plan first


class Scheduler:
    """Admission and batching by shape under a device-memory budget.

    batch_for(key) gives a shape's batch size, plan_bytes(key, batch) the
    device bytes of one plan with its buffers.  Not thread-safe: the caller
    holds a lock around every call.
    """

    def __init__(self, budget_bytes: int, batch_for: Callable[[Key], int],
                 plan_bytes: Callable[[Key, int], int], max_slots_per_key: int = 4):
        self.budget = int(budget_bytes)
        self.batch_for = batch_for
        self.plan_bytes = plan_bytes
        self.max_slots = max_slots_per_key
        self.queues: Dict[Key, Deque] = {}
        self.slots: Dict[Key, List[SlotState]] = {}
        self.used = 0
        self.evicted: List[SlotState] = []  # plans the executor must free
        self.expired: List = []  # queued requests whose deadline passed before they were admitted

    @staticmethod
    def key_of(req) -> Key:
        return (req.dim, req.N)

    def arrive(self, req) -> None:
        self.queues.setdefault(self.key_of(req), deque()).append(req)

    def pending(self) -> int:
        return sum(len(q) for q in self.queues.values())

    def cancel(self, rid: int) -> bool:
        """Withdraw a queued request; False if it is not queued (already taken
        into a batch, which then runs to its end, or unknown)."""
        for q in self.queues.values():
            for r in q:
                if r.rid == rid:
                    q.remove(r)
                    return True
        return False

    def _expire(self, now: float) -> None:
        for q in self.queues.values():
            keep = [r for r in q if getattr(r, "deadline", None) is None or r.deadline >= now]
            if len(keep) != len(q):
                self.expired += [r for r in q if not (getattr(r, "deadline", None) is None or r.deadline >= now)]
                q.clear()
                q.extend(keep)

    def take_expired(self) -> List:
        out, self.expired = self.expired, []
        return out

    def _evict_for(self, need: int, keep: Key) -> bool:
        """Evict idle plans of other shapes (LRU) until `need` more bytes fit."""
        if self.used + need <= self.budget:
            return True
        idle = [s for k, ss in self.slots.items() if k != keep for s in ss if not s.busy]
        idle.sort(key=lambda s: s.last_used)
        freed = 0
        victims = []
        for s in idle:
            if self.used - freed + need <= self.budget:
                break
            victims.append(s)
            freed += s.nbytes
        if self.used - freed + need > self.budget:
            return False
        for s in victims:
            self.slots[s.key].remove(s)
            self.used -= s.nbytes
            self.evicted.append(s)
        return True

    def next_work(self, now: float) -> Optional[Work]:
        """The batch to run next: the shape whose oldest request has waited
        longest among shapes with an idle plan or room for a new one.  Queued
        requests whose deadline has passed are dropped first (take_expired)."""
        self._expire(now)
        order = sorted((q[0].arrival, k) for k, q in self.queues.items() if q)
        for _, k in order:
            ss = self.slots.setdefault(k, [])
            q = self.queues[k]
            bmax = max(1, int(self.batch_for(k)))
            n = min(bmax, len(q))
            want = 1
            while want < n:
                want *= 2
            want = min(want, bmax)
            idle = [s for s in ss if not s.busy]
            # the smallest idle plan that holds all n, else a new plan of size `want`
            fit = sorted((s for s in idle if s.batch >= n), key=lambda s: s.batch)
            slot = fit[0] if fit and fit[0].batch <= 2 * want else None
            new = False
            if slot is None and len(ss) < self.max_slots:
                B = want
                nb = int(self.plan_bytes(k, B))
                while nb > self.budget and B > 1:  # a smaller batch when one plan would not fit
                    B //= 2
                    nb = int(self.plan_bytes(k, B))
                fits = self._evict_for(nb, k)
                if fits or self.used == 0:  # nothing else resident: run over budget rather than starve
                    slot = SlotState(k, B, nb)
                    ss.append(slot)
                    self.used += nb
                    new = True
            if slot is None and idle:  # no room for a new plan: the largest idle one
                slot = max(idle, key=lambda s: s.batch)
            if slot is None:
                continue
            reqs = [q.popleft() for _ in range(min(slot.batch, len(q)))]
            slot.busy = True
            slot.last_used = now
            return Work(k, slot, reqs, new)
        return None

    def release(self, work: Work, now: float) -> None:
        work.slot.busy = False
        work.slot.last_used = now

    def take_evicted(self) -> List[SlotState]:
        out, self.evicted = self.evicted, []
        return out


# ----------------------------------------------------------------------------
# device executor
# ----------------------------------------------------------------------------

STATUS_CANCELLED = -2  # withdrawn by Server.cancel while queued
STATUS_EXPIRED = 6     # AHOC_ETIMEOUT: its deadline passed while queued


@dataclass
class Record:
    rid: int
    dim: int
    N: int
    arrival: float
    start: float = 0.0   # taken from the queue by a worker
    loaded: float = 0.0  # its coefficient and right-hand side in the plan (request data ready)
    done: float = 0.0    # its solution in device memory (the solve returned)
    batch: int = 0       # requests solved together with this one (itself included)
    status: int = -1
    iters: int = 0
    refine_steps: int = 0
    err_inf: Optional[float] = None
    new_plan: bool = False  # its batch created the plan it ran on

    @property
    def latency(self) -> float:
        return self.done - self.arrival

    @property
    def dof(self) -> int:
        return (self.N - 1) ** self.dim


def default_batch(key: Key) -> int:
    """Problems per launch: enough grid points to fill the GPU (about 4M
    interior points per batch), at most 16."""
    dim, N = key
    pts = (N - 1) ** dim
    return int(max(1, min(16, (4 << 20) // max(pts, 1))))


class Server:
    """Solve a request stream with batched plans on several CUDA streams.

    prec: "mixed" (FP32 inner solves, FP64 refinement) or "fp64";
    tol: relative Schur residual of every solve; workers: concurrent batches;
    batch_for: per-shape batch size (default ``default_batch``; 1 gives the
    plain one-request-per-solve server).
    """

    def __init__(self, device="cuda", prec="mixed", tol: float = 1e-10, workers: int = 4,
                 budget_bytes: Optional[int] = None, batch_for: Optional[Callable[[Key], int]] = None,
                 restart: int = 60, keep_results: bool = False, check_exact: bool = False,
                 data_at_arrival: bool = True, priority_dof: int = 1 << 21):
        import torch

        from . import ahoc
        self.torch = torch
        self.ahoc = ahoc
        self.device = torch.device(device)
        self.prec = prec
        self.tol = tol
        self.workers = workers
        self.restart = restart
        self.keep = keep_results
        self.check_exact = check_exact
        # a request arrives with its data (as a client's upload would): the
        # feeder synthesises alpha and f on its own stream before the request
        # enters the queue, and the worker copies them into its plan slot
        self.data_at_arrival = data_at_arrival
        self.pending: Dict[int, tuple] = {}
        # plans of shapes with at most this many interior points run on
        # high-priority streams, so that small requests are not held up behind
        # the kernels of large ones (the plan's graph stream inherits it)
        self.priority_dof = priority_dof
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(0.6 * free)
        self.sched = Scheduler(budget_bytes, batch_for or default_batch, self._plan_bytes)
        self.results: Dict[int, object] = {}
        self.records: Dict[int, Record] = {}
        # called with (spec, alpha, f) after a request's data are written into
        # its plan slot, before the load (tests use it to alter a request)
        self.data_hook: Optional[Callable] = None
        self.cv = threading.Condition()
        self.error: Optional[BaseException] = None

    def _plan_bytes(self, key: Key, B: int) -> int:
        dim, N = key
        ws = self.ahoc.workspace_bytes(dim, [N] * dim, self.restart, self.prec, -1, B)
        return ws + 3 * B * (N + 1) ** dim * 8  # + alpha, f, u buffers

    # one plan of a shape, with its buffers and stream
    class _Slot:
        def __init__(self, srv: "Server", key: Key, B: int):
            torch = srv.torch
            dim, N = key
            small = (N - 1) ** dim <= srv.priority_dof
            self.stream = torch.cuda.Stream(device=srv.device, priority=-1 if small else 0)
            nf = (N + 1) ** dim
            self.nf = nf
            with torch.cuda.stream(self.stream):
                self.alpha = torch.ones(B * nf, dtype=torch.float64, device=srv.device)
                self.f = torch.zeros(B * nf, dtype=torch.float64, device=srv.device)
                self.u = torch.zeros(B * nf, dtype=torch.float64, device=srv.device)
                self.plan = srv.ahoc.Plan(dim, [N] * dim, self.alpha, prec=srv.prec, restart=srv.restart,
                                          batch=B, stream=self.stream, max_iters=2000)
            self.stream.synchronize()

        def close(self):
            self.plan.close()

    def _run_work(self, w: Work) -> None:
        from . import inputs
        torch = self.torch
        t0 = time.perf_counter()
        if w.new_slot:
            w.slot.handle = Server._Slot(self, w.key, w.slot.batch)
        sl: Server._Slot = w.slot.handle
        B = w.slot.batch
        nf = sl.nf
        with torch.cuda.stream(sl.stream):
            # the request's data into the plan slot: copied from what arrived
            # with it, or synthesised here from its closed form
            for i, spec in enumerate(w.reqs):
                a_i, f_i = sl.alpha[i * nf:(i + 1) * nf], sl.f[i * nf:(i + 1) * nf]
                with self.cv:
                    arrived = self.pending.pop(spec.rid, None)
                if arrived is not None:
                    a_i.copy_(arrived[0])
                    f_i.copy_(arrived[1])
                else:
                    inputs.sample_request(spec, device=self.device, out_alpha=a_i, out_f=f_i)
                    if self.data_hook is not None:
                        self.data_hook(spec, a_i, f_i)
                sl.plan.load(i, a_i)
                del arrived
            sl.stream.synchronize()
            t_loaded = time.perf_counter()
            sl.plan.set_active([1 if i < len(w.reqs) else 0 for i in range(B)])
            _, infos = sl.plan.solve(sl.f, sl.u, tol=self.tol, check=False)
            if B == 1:
                infos = [infos]
            sl.stream.synchronize()
            t1 = time.perf_counter()
            # after the request is done: its result kept, its error against the exact u
            outs = []
            for i, spec in enumerate(w.reqs):
                ui = sl.u[i * nf:(i + 1) * nf]
                err = None
                if self.check_exact and infos[i]["status"] == 0:
                    err = float((ui - inputs.exact_request(spec, self.device)).abs().max())
                outs.append((ui.clone() if self.keep else None, err))
            sl.stream.synchronize()
        for i, spec in enumerate(w.reqs):
            r = self.records[spec.rid]
            r.start, r.loaded, r.done, r.batch, r.new_plan = t0, t_loaded, t1, len(w.reqs), w.new_slot
            r.status, r.iters, r.refine_steps = infos[i]["status"], infos[i]["iters"], infos[i]["refine_steps"]
            r.err_inf = outs[i][1]
            if self.keep:
                self.results[spec.rid] = outs[i][0]

    def _worker(self, t_start: float) -> None:
        try:
            while True:
                with self.cv:
                    while True:
                        if self.error is not None:
                            return
                        if self._fed and self.sched.pending() == 0:
                            return  # every request is taken; in-flight batches finish on their workers
                        now = time.perf_counter()
                        w = self.sched.next_work(now - t_start)
                        for spec in self.sched.take_expired():
                            self.pending.pop(spec.rid, None)
                            r = self.records[spec.rid]
                            r.status, r.start, r.loaded, r.done = STATUS_EXPIRED, now, now, now
                        if w is not None:
                            evicted = self.sched.take_evicted()
                            break
                        self.cv.wait(timeout=0.05)
                for s in evicted:
                    if s.handle is not None:
                        s.handle.close()
                        s.handle = None
                self._run_work(w)
                with self.cv:
                    self.sched.release(w, time.perf_counter() - t_start)
                    self.cv.notify_all()
        except BaseException as e:  # surface worker failures to run()
            with self.cv:
                self.error = e
                self.cv.notify_all()

    def run(self, specs: Sequence, realtime: bool = True) -> List[Record]:
        """Feed the requests at their arrival times (or all at once) and solve them."""
        from . import inputs
        torch = self.torch
        self.records = {s.rid: Record(s.rid, s.dim, s.N, s.arrival) for s in specs}
        self._fed = False
        feed = torch.cuda.Stream(device=self.device) if self.data_at_arrival else None
        t_start = time.perf_counter()
        threads = [threading.Thread(target=self._worker, args=(t_start,), daemon=True)
                   for _ in range(self.workers)]
        for t in threads:
            t.start()
        for s in sorted(specs, key=lambda r: r.arrival):
            if realtime:
                dt = s.arrival - (time.perf_counter() - t_start)
                if dt > 0:
                    time.sleep(dt)
            if feed is not None:
                with torch.cuda.stream(feed):
                    d = inputs.sample_request(s, device=self.device)
                    if self.data_hook is not None:
                        self.data_hook(s, d["alpha"], d["f"])
                feed.synchronize()
            with self.cv:
                if feed is not None:
                    self.pending[s.rid] = (d["alpha"], d["f"])
                self.sched.arrive(s)
                # the time the request (with its data) entered the queue
                self.records[s.rid].arrival = (time.perf_counter() - t_start) if realtime else 0.0
                self.cv.notify_all()
        with self.cv:
            self._fed = True
            self.cv.notify_all()
        for t in threads:
            t.join()
        if self.error is not None:
            raise self.error
        for r in self.records.values():
            r.start -= t_start
            r.loaded -= t_start
            r.done -= t_start
        self.pending.clear()
        return [self.records[s.rid] for s in specs]

    def cancel(self, rid: int) -> bool:
        """Withdraw a request that is still queued (its record gets
        STATUS_CANCELLED); a request already in a batch runs to its end."""
        with self.cv:
            if not self.sched.cancel(rid):
                return False
            self.pending.pop(rid, None)
            r = self.records[rid]
            now = time.perf_counter()
            r.status, r.start, r.loaded, r.done = STATUS_CANCELLED, now, now, now
            self.cv.notify_all()
            return True

    def close(self) -> None:
        for ss in self.sched.slots.values():
            for s in ss:
                if s.handle is not None:
                    s.handle.close()
                    s.handle = None


def summarize(records: Sequence[Record]) -> Dict[str, float]:
    """p50/p99 latency (ms) from arrival to the solution in device memory,
    its parts (queue wait, request data synthesis and load, solve), the
    aggregate DOF/s over the makespan and the batch sizes, over the requests
    that were solved (cancelled and expired ones are counted apart)."""
    import numpy as np
    served = [r for r in records if r.status not in (STATUS_CANCELLED, STATUS_EXPIRED)]
    dropped = len(records) - len(served)
    records = served
    lat = np.array([r.latency for r in records]) * 1e3
    wait = np.array([r.start - r.arrival for r in records]) * 1e3
    data = np.array([r.loaded - r.start for r in records]) * 1e3
    solve = np.array([r.done - r.loaded for r in records]) * 1e3
    t0 = min(r.arrival for r in records)
    t1 = max(r.done for r in records)
    dof = sum(r.dof for r in records)
    parts = {"queue_wait_ms": wait, "data_ms": data, "solve_ms": solve}
    pct = {k: {"p50": float(np.percentile(v, 50)), "p99": float(np.percentile(v, 99))} for k, v in parts.items()}
    # the slowest 1%: where their time went, and how many ran on a plan created for them
    k = max(1, len(records) // 100)
    slow = np.argsort(lat)[-k:]
    tail = {kk: float(np.mean(v[slow])) for kk, v in parts.items()}
    tail["new_plan_fraction"] = float(np.mean([records[i].new_plan for i in slow]))
    shapes = {}
    for k in sorted({(r.dim, r.N) for r in records}):
        ls = np.array([r.latency for r in records if (r.dim, r.N) == k]) * 1e3
        shapes["%dD N=%d" % k] = {"n": int(ls.size), "p50_ms": float(np.percentile(ls, 50)),
                                  "p99_ms": float(np.percentile(ls, 99))}
    return dict(requests=len(records), p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), makespan_s=t1 - t0, dof_per_s=dof / (t1 - t0),
                mean_batch=float(np.mean([r.batch for r in records])),
                failed=int(sum(1 for r in records if r.status != 0)), dropped=dropped, by_shape=shapes,
                parts=pct, slowest_1pct_mean_ms=tail)
