"""Continuous-batching serving loop for client-side encrypted HDC inference.

Requests (one client's batch of feature rows each) arrive over time.  The loop
- admits an arriving request when its feature rows can be placed in the feature
  arena: one device buffer of `budget_bytes`, allocated once beside the resident
  encrypted model and rotation keys and carved first-fit into 256-byte-aligned
  ranges.  On admission the request's features are copied into its range on an
  upload stream (from host memory or from a device tensor, ordered after the
  caller's current stream), and the range is freed when the request completes or is
  cancelled.  A request larger than the whole arena, or than one step, is rejected;
  the others wait in arrival order until a range frees up.  The score ciphertexts
  live in the slots' output buffers, allocated once per slot (slots x max_groups
  groups), so admission changes no other allocation;
- whenever one of its pipeline slots is idle, packs the admitted requests (up to
  the slot's group capacity) into one step and launches it on the slot's stream;
  each slot has its own context scratch, CUDA stream and CUDA graphs, and all slots
  share the device-resident model and keys, so a step can run on the device while
  the next one is being packed and launched;
- when a step's score ciphertexts have reached host memory (the message to the
  server, Sec. 4.1), completes its requests, frees their memory and records each
  request's latency from arrival to completion.

Each request's result is the range of packed queries it owns in its step's score
ciphertexts; decrypting them gives the same scores as running the request alone.

A request can be cancelled at any time: while it waits it is dropped (and its
memory returned); once launched its step runs to completion, the request's rows are
discarded and its memory is returned with the step, so nothing in flight on the
device is interrupted.  The slots are injectable (`slot_factory`), so the admission,
packing, cancellation and bookkeeping logic runs on the host with fake slots.
"""
import collections
import time

import numpy as np
import torch

from . import batching as BT
from . import ephdc as E


ALIGN = 256


def request_bytes(F, B):
    """Arena bytes of a request of B feature rows of F int8 features."""
    return -(-(B * F) // ALIGN) * ALIGN


class FeatureArena:
    """First-fit allocator of 256-byte-aligned ranges of one preallocated device
    buffer (`device` None: the bookkeeping alone, for host tests)."""

    def __init__(self, capacity, device=None):
        self.capacity = int(capacity) // ALIGN * ALIGN
        self.buf = (torch.empty(self.capacity, dtype=torch.int8, device=device)
                    if device is not None and self.capacity else None)
        self.free = [(0, self.capacity)] if self.capacity else []  # sorted, disjoint
        self.used = 0
        self.peak = 0

    def alloc(self, nbytes):
        """Offset of a free range of nbytes (a multiple of ALIGN), or None."""
        for i, (off, size) in enumerate(self.free):
            if size >= nbytes:
                if size == nbytes:
                    del self.free[i]
                else:
                    self.free[i] = (off + nbytes, size - nbytes)
                self.used += nbytes
                self.peak = max(self.peak, self.used)
                return off
        return None

    def release(self, off, nbytes):
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, nbytes))
        # merge with the following and the preceding free range where they touch
        if i + 1 < len(self.free) and off + nbytes == self.free[i + 1][0]:
            self.free[i] = (off, nbytes + self.free[i + 1][1])
            del self.free[i + 1]
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == off:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            del self.free[i]
        self.used -= nbytes

    def view(self, off, B, F):
        return self.buf[off:off + B * F].view(B, F)


class Request:
    __slots__ = ("rid", "arrival", "X", "B", "admitted", "launched", "done", "step",
                 "rows", "nbytes", "cancelled", "off", "ready")

    def __init__(self, rid, arrival, X):
        self.rid, self.arrival, self.X = rid, arrival, X
        self.B = int(X.shape[0])
        self.admitted = self.launched = self.done = None
        self.step = None
        self.rows = None
        self.nbytes = 0
        self.cancelled = False
        self.off = None     # the request's range in the feature arena once admitted
        self.ready = None   # event recorded after its features reached the arena


class Step:
    """One launched packed step: its requests, host copy of the ciphertexts, event."""

    def __init__(self, sid, reqs, packed, host_out, event, slot):
        self.sid, self.reqs, self.packed = sid, reqs, packed
        self.host_out, self.event, self.slot = host_out, event, slot


class Slot:
    def __init__(self, w, Wt, model, gk, max_groups, use_graphs=True):
        cap = 2 * ((w.n // (2 * w.r)) // w.k_in)
        self.ctx = E.Context.for_workload(w, max_batch=max_groups * cap)
        self.pipe = BT.GraphedPipeline(self.ctx, Wt, model, gk, max_groups=max_groups,
                                       use_graphs=use_graphs)
        self.stream = torch.cuda.Stream(device=self.ctx.device)
        self.busy = None

    def warm(self):
        for G in range(1, self.pipe.max_groups + 1):
            self.pipe.graph(G) if self.pipe.use_graphs else None
        torch.cuda.synchronize()

    def submit(self, Xs, ready=None):
        """Launches one packed step on this slot's stream once the events in `ready`
        (one per request: its features are in place; None entries are skipped) have
        completed; without `ready` the step is ordered after the caller's current
        stream.  Returns (pinned host copy of the score ciphertexts, completion event,
        PackedBatch)."""
        if ready is None:
            self.stream.wait_stream(torch.cuda.current_stream())
        else:
            for ev in ready:
                if ev is not None:
                    self.stream.wait_event(ev)
        with torch.cuda.stream(self.stream):
            out, pb = self.pipe.launch(Xs, self.stream)
            host = torch.empty(out.shape, dtype=out.dtype, pin_memory=True)
            host.copy_(out, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        return host, ev, pb


DEFAULT_ARENA = 1 << 30


class Server:
    """budget_bytes: size of the feature arena (default: 1 GiB, or the free device
    memory less 4 GiB if that is smaller).  With `slot_factory` (host tests) the arena
    keeps its bookkeeping only and requests keep their own X."""

    def __init__(self, w, Wt, model, gk, slots=2, max_groups=8, budget_bytes=None,
                 use_graphs=True, keep_outputs=False, slot_factory=None):
        self.w = w
        self.cap = 2 * ((w.n // (2 * w.r)) // w.k_in)
        self.ct_bytes = 2 * w.L * w.n * 4
        self.Kp = w.k // w.k_in
        make = slot_factory or (lambda i: Slot(w, Wt, model, gk, max_groups, use_graphs))
        self.slots = [make(i) for i in range(slots)]
        self.max_queries = max_groups * self.cap
        device = None
        if slot_factory is None:
            device = self.slots[0].ctx.device
            if budget_bytes is None:
                free, _ = torch.cuda.mem_get_info(device)
                budget_bytes = min(DEFAULT_ARENA, max(0, free - (4 << 30)))
            self.upload = torch.cuda.Stream(device=device)
        elif budget_bytes is None:
            budget_bytes = DEFAULT_ARENA
        self.arena = FeatureArena(budget_bytes, device)
        self.waited = 0
        self.keep_outputs = keep_outputs
        self.pending = collections.deque()   # arrived, not admitted (memory)
        self.queue = collections.deque()     # admitted, not launched
        self.steps = []
        self.completed = []
        self.rejected = []
        self.cancelled = []

    @property
    def budget(self):
        return self.arena.capacity

    @property
    def used(self):
        return self.arena.used

    def request_bytes(self, B):
        return request_bytes(self.w.F, B)

    def warm(self):
        for s in self.slots:
            s.warm()

    # ------------------------------------------------------------------ events
    def arrive(self, req, now, admit=True):
        """A request arrives; with admit=False the caller admits a whole batch of
        arrivals at once afterwards (one upload event for all of them)."""
        req.nbytes = self.request_bytes(req.B)
        if req.nbytes > self.budget or req.B > self.max_queries:
            req.done = now
            self.rejected.append(req)
            return
        self.pending.append(req)
        if admit:
            self._admit(now)
            if self.pending and self.pending[-1] is req:
                self.waited += 1   # no free range on arrival: it waits for memory

    def admit_arrivals(self, reqs, now):
        """Admits what fits of a batch of requests that arrived together (see arrive)."""
        self._admit(now)
        waiting = {id(r) for r in self.pending}
        self.waited += sum(1 for r in reqs if id(r) in waiting)

    def _admit(self, now):
        placed = []
        while self.pending:
            r = self.pending[0]
            off = self.arena.alloc(r.nbytes)
            if off is None:
                break
            self.pending.popleft()
            r.off, r.admitted = off, now
            placed.append(r)
            self.queue.append(r)
        if placed and self.arena.buf is not None:
            self._place(placed)

    def _place(self, reqs):
        """Copies admitted requests' features into their arena ranges on the upload
        stream, after the work already on the caller's current stream (which may be
        producing them); each request then holds its arena view and one event recorded
        after all of the copies."""
        # ordered after the caller's stream once for the whole batch
        self.upload.wait_stream(torch.cuda.current_stream(self.arena.buf.device))
        with torch.cuda.stream(self.upload):
            for r in reqs:
                src = r.X if isinstance(r.X, torch.Tensor) else torch.from_numpy(np.asarray(r.X))
                dst = self.arena.view(r.off, r.B, self.w.F)
                dst.copy_(src, non_blocking=True)
                if src.is_cuda:
                    src.record_stream(self.upload)   # the caller may free X after this
                r.X = dst
            ev = torch.cuda.Event()
            ev.record(self.upload)
        for r in reqs:
            r.ready = ev

    def _free(self, r):
        if r.off is not None:
            self.arena.release(r.off, r.nbytes)
            r.off = None

    def _launch(self, slot, now):
        take, total = [], 0
        while self.queue and total + self.queue[0].B <= self.max_queries:
            r = self.queue.popleft()
            take.append(r)
            total += r.B
        if not take:
            return False
        if self.arena.buf is None:
            host, ev, pb = slot.submit([r.X for r in take])
        else:
            ready = list({id(r.ready): r.ready for r in take}.values())
            host, ev, pb = slot.submit([r.X for r in take], ready)
        st = Step(len(self.steps), take, pb, host, ev, slot)
        for i, r in enumerate(take):
            r.launched, r.step, r.rows = now, st.sid, pb.rows(i)
        self.steps.append(st)
        slot.busy = st
        return True

    def poll(self, now):
        """Completes finished steps, admits, launches on idle slots.  Returns True if
        anything is still queued or in flight."""
        for slot in self.slots:
            st = slot.busy
            if st is not None and st.event.query():
                t = time.perf_counter() if now is None else now
                for r in st.reqs:
                    r.done = t
                    self._free(r)
                    if self.arena.buf is not None:
                        r.X = None
                    (self.cancelled if r.cancelled else self.completed).append(r)
                if not self.keep_outputs:
                    st.host_out = None
                slot.busy = None
        self._admit(now)
        for slot in self.slots:
            if slot.busy is None and self.queue:
                self._launch(slot, now)
        return bool(self.queue or self.pending or any(s.busy for s in self.slots))

    def cancel(self, rid, now):
        """Cancels request rid.  Waiting requests leave at once (admitted ones return
        their memory); a launched request's step finishes, its rows are discarded and
        its memory comes back with the step.  Returns False if rid is unknown or
        already finished."""
        for dq, admitted in ((self.pending, False), (self.queue, True)):
            for r in dq:
                if r.rid == rid:
                    dq.remove(r)
                    r.cancelled, r.done = True, now
                    if admitted:
                        # no slot reads it; a later upload into the range is ordered
                        # after this request's own copy on the upload stream
                        self._free(r)
                    self.cancelled.append(r)
                    self._admit(now)
                    return True
        for slot in self.slots:
            st = slot.busy
            if st is not None:
                for r in st.reqs:
                    if r.rid == rid and not r.cancelled:
                        r.cancelled = True
                        return True
        return False

    # ------------------------------------------------------------------ request loop
    def run(self, arrivals, make_X, time_scale=1.0):
        """Replays an arrival schedule in real time (arrival times in seconds,
        multiplied by time_scale) and serves it to completion."""
        order = np.argsort(arrivals, kind="stable")
        t0 = time.perf_counter()
        nxt = 0
        while True:
            now = time.perf_counter() - t0
            due = []
            while nxt < len(order) and arrivals[order[nxt]] * time_scale <= now:
                rid = int(order[nxt])
                due.append(Request(rid, arrivals[rid] * time_scale, make_X(rid)))
                self.arrive(due[-1], now, admit=False)
                nxt += 1
            if due:
                self.admit_arrivals(due, now)
            busy = self.poll(time.perf_counter() - t0)
            if nxt >= len(order) and not busy:
                break
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    def report(self, wall_s):
        lat = np.array([r.done - r.arrival for r in self.completed]) if self.completed else \
            np.zeros(1)
        q = sum(r.B for r in self.completed)
        return {"requests": len(self.completed) + len(self.rejected) + len(self.cancelled),
                "completed": len(self.completed), "rejected": len(self.rejected),
                "cancelled": len(self.cancelled),
                "queries": q, "queries_per_s": q / wall_s if wall_s > 0 else 0.0,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "steps": len(self.steps),
                "mean_queries_per_step": q / max(1, len(self.steps)), "wall_s": wall_s,
                "arena_bytes": self.arena.capacity, "arena_peak_bytes": self.arena.peak,
                "waited_for_memory": self.waited}
