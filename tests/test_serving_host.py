"""Host logic of the serving loop with fake pipeline slots (no GPU): admission by a
device-memory budget in arrival order, rejection of requests that can never fit,
packing of admitted requests into steps, cancellation while waiting and while in
flight, and that every byte admitted is returned.  Failures are made on the host:
a small fake budget, requests cancelled at each stage."""
import numpy as np

from paper_2511_00737_gb300 import batching as BT
from paper_2511_00737_gb300 import serving as SV
from paper_2511_00737_gb300 import workload as WL


class FakeEvent:
    def __init__(self):
        self.done = False

    def query(self):
        return self.done


class FakeSlot:
    def __init__(self, cap):
        self.cap, self.busy, self.events, self.steps = cap, None, [], []

    def submit(self, Xs):
        ev = FakeEvent()
        self.events.append(ev)
        self.steps.append([x.shape[0] for x in Xs])
        return None, ev, BT.PackedBatch([x.shape[0] for x in Xs], self.cap)


W = WL.Workload(name="t", n=1024, L=3, k=3, k_in=1, r=4, D=120, F=32, bits=8, B=0, seed=9)
CAP = 2 * ((W.n // (2 * W.r)) // W.k_in)  # 256


def server(budget, slots=2, max_groups=2):
    fakes = []

    def make(i):
        fakes.append(FakeSlot(CAP))
        return fakes[-1]

    srv = SV.Server(W, None, None, None, slots=slots, max_groups=max_groups, budget_bytes=budget,
                    slot_factory=make)
    return srv, fakes


def req(rid, B, t=0.0):
    return SV.Request(rid, t, np.zeros((B, W.F), np.int8))


def finish_all(srv, fakes, t):
    for f in fakes:
        for ev in f.events:
            ev.done = True
    return srv.poll(t)


def test_admission_in_arrival_order_within_budget():
    one = SV.request_bytes(W.F, 100)
    srv, fakes = server(budget=2 * one)
    for rid in range(4):
        srv.arrive(req(rid, 100), 0.0)
    assert [r.rid for r in srv.queue] == [0, 1] and [r.rid for r in srv.pending] == [2, 3]
    assert srv.used == 2 * one
    srv.poll(0.1)
    # both admitted requests fit one step of 2 groups on the first idle slot
    assert fakes[0].steps == [[100, 100]] and fakes[1].steps == []
    assert [r.rid for r in srv.pending] == [2, 3]
    busy = finish_all(srv, fakes, 0.2)
    assert busy and [r.rid for r in srv.completed] == [0, 1]
    assert fakes[0].steps[-1] == [100, 100] or fakes[1].steps == [[100, 100]]
    while finish_all(srv, fakes, 0.3):
        pass
    assert sorted(r.rid for r in srv.completed) == [0, 1, 2, 3]
    assert srv.used == 0 and not srv.pending and not srv.queue


def test_requests_that_can_never_fit_are_rejected():
    srv, _ = server(budget=10 ** 9)
    srv.arrive(req(0, 2 * CAP + 1), 0.0)            # more than a step's 2 groups
    assert [r.rid for r in srv.rejected] == [0] and srv.used == 0
    srv, _ = server(budget=SV.request_bytes(W.F, 50) - 1)
    srv.arrive(req(1, 50), 0.0)                     # more than the whole arena
    assert [r.rid for r in srv.rejected] == [1] and srv.used == 0
    assert srv.report(1.0)["rejected"] == 1


def test_cancel_waiting_queued_and_in_flight():
    srv, fakes = server(budget=2 * SV.request_bytes(W.F, 200), slots=1, max_groups=1)
    for rid, B in enumerate([200, 200, 200, 10]):
        srv.arrive(req(rid, B), 0.0)
    srv.poll(0.0)                      # request 0 in flight (a step holds one group)
    assert fakes[0].steps == [[200]]
    assert [r.rid for r in srv.queue] == [1] and [r.rid for r in srv.pending] == [2, 3]
    assert srv.cancel(2, 0.1)          # waiting for memory: dropped
    assert srv.cancel(1, 0.1)          # admitted, not launched: memory returned, 3 admitted
    assert [r.rid for r in srv.queue] == [3]
    assert srv.cancel(0, 0.1)          # in flight: finishes, rows discarded
    assert not srv.cancel(0, 0.1) and not srv.cancel(99, 0.1)
    while finish_all(srv, fakes, 0.2):
        pass
    assert [r.rid for r in srv.completed] == [3]
    assert sorted(r.rid for r in srv.cancelled) == [0, 1, 2]
    assert srv.used == 0
    rep = srv.report(1.0)
    assert rep["completed"] == 1 and rep["cancelled"] == 3 and rep["requests"] == 4


def test_each_completed_request_owns_its_packed_rows():
    srv, fakes = server(budget=10 ** 9, slots=2, max_groups=2)
    sizes = [5, 250, 1, 100, 64, 300, 17]
    for rid, B in enumerate(sizes):
        srv.arrive(req(rid, B), 0.0)
    while srv.poll(0.0) or any(not ev.done for f in fakes for ev in f.events):
        finish_all(srv, fakes, 0.0)
    assert sorted(r.rid for r in srv.completed) == list(range(len(sizes)))
    for st in srv.steps:
        end = 0
        for r in st.reqs:
            assert r.rows.start == end and r.rows.stop - r.rows.start == r.B
            end = r.rows.stop
        assert end <= 2 * CAP


def test_feature_arena_first_fit_and_coalescing():
    a = SV.FeatureArena(10 * SV.ALIGN)
    x = a.alloc(3 * SV.ALIGN)
    y = a.alloc(3 * SV.ALIGN)
    z = a.alloc(3 * SV.ALIGN)
    assert (x, y, z) == (0, 3 * SV.ALIGN, 6 * SV.ALIGN) and a.used == 9 * SV.ALIGN
    assert a.alloc(2 * SV.ALIGN) is None            # one aligned unit left
    a.release(y, 3 * SV.ALIGN)
    assert a.alloc(4 * SV.ALIGN) is None            # 3 + 1 free units, not adjacent
    a.release(z, 3 * SV.ALIGN)                      # merges with y's range and the tail
    assert a.free == [(3 * SV.ALIGN, 7 * SV.ALIGN)]
    assert a.alloc(7 * SV.ALIGN) == 3 * SV.ALIGN
    a.release(x, 3 * SV.ALIGN)
    a.release(3 * SV.ALIGN, 7 * SV.ALIGN)
    assert a.free == [(0, 10 * SV.ALIGN)] and a.used == 0 and a.peak == 10 * SV.ALIGN


def test_admission_waits_for_a_contiguous_range():
    unit = SV.request_bytes(W.F, 8)                  # 256 bytes
    srv, fakes = server(budget=4 * unit, slots=1, max_groups=1)
    for rid, B in enumerate([8, 8, 8, 8]):
        srv.arrive(req(rid, B), 0.0)
    assert srv.used == 4 * unit and srv.waited == 0
    srv.arrive(req(4, 16), 0.0)                       # needs two adjacent units
    assert [r.rid for r in srv.pending] == [4] and srv.waited == 1
    srv.poll(0.0)                                     # one step takes all four
    assert fakes[0].steps == [[8, 8, 8, 8]]
    while finish_all(srv, fakes, 0.1):
        pass
    assert sorted(r.rid for r in srv.completed) == [0, 1, 2, 3, 4] and srv.used == 0
    assert srv.report(1.0)["waited_for_memory"] == 1
