"""Scheduler of the serving loop, on the CPU with a fake executor: HBM-budget admission,
one edit per session per batch in arrival order, a fixed number of batches in flight,
latency from arrival to completion, sessions leaving only when idle, and cancelled
requests (withdrawn before they reach the device), withdrawn waiting sessions, and the
eviction of idle sessions (least recently used first) with readmission on their next edit."""
import pytest

from paper_2407_21552_gb300.serving import Scheduler, SessionSpec


class FakeExec:
    def __init__(self):
        self.t = 0.0
        self.admitted, self.released, self.launched = [], [], []

    def clock(self):
        return self.t

    def admit(self, spec):
        self.admitted.append(spec.sid)

    def release(self, sid):
        self.released.append(sid)

    def launch(self, slot, reqs):
        h = {"slot": slot, "reqs": [(r.session, r.tf) for r in reqs], "done": False}
        self.launched.append(h)
        return h

    def done(self, h):
        return h["done"]


def test_budget_admission_and_release():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=100, slots=2)
    assert s.open_session(SessionSpec(0, 60))
    assert s.open_session(SessionSpec(1, 30))
    assert not s.open_session(SessionSpec(2, 30))      # would exceed the budget: waits
    assert not s.open_session(SessionSpec(3, 5))       # queued behind session 2 (FIFO)
    assert ex.admitted == [0, 1] and s.used == 90
    s.close_session(0)                                 # frees 60: 2 and 3 are admitted
    assert ex.admitted == [0, 1, 2, 3] and s.used == 65 and ex.released == [0]
    with pytest.raises(ValueError):
        s.open_session(SessionSpec(9, 101))
    with pytest.raises(KeyError):
        s.submit(0, "tf")                              # no longer admitted


def test_one_edit_per_session_per_batch_in_order_and_slots():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=2)
    for sid in range(3):
        s.open_session(SessionSpec(sid, 1))
    for k in range(3):
        s.submit(0, f"a{k}")
    s.submit(1, "b0")
    s.poll()
    # the oldest edit of each session; sessions 0 and 1 are then on the device, so the
    # second slot stays free although session 0 has more edits
    assert len(ex.launched) == 1
    assert ex.launched[0]["reqs"] == [(0, "a0"), (1, "b0")]
    s.submit(2, "c0")
    s.poll()                                           # session 2 is idle: second slot
    assert len(ex.launched) == 2 and ex.launched[1]["reqs"] == [(2, "c0")]
    s.poll()                                           # no free slot, busy sessions
    assert len(ex.launched) == 2
    ex.t = 5.0
    ex.launched[0]["done"] = True
    s.poll()                                           # retire batch 0: a1 goes next
    assert len(ex.launched) == 3 and ex.launched[2]["reqs"] == [(0, "a1")]
    assert sorted(s.stats.latencies) == [5.0, 5.0]
    ex.t = 7.0
    while s.has_work():
        for h in ex.launched:
            h["done"] = True
        s.poll()
    assert len(s.completed) == 5 and not s.has_work()
    assert [r.tf for r in s.completed if r.session == 0] == ["a0", "a1", "a2"]


def test_session_with_edits_in_flight_cannot_close():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=1)
    s.open_session(SessionSpec(0, 1))
    s.submit(0, "x")
    s.poll()
    with pytest.raises(RuntimeError):
        s.close_session(0)
    ex.launched[0]["done"] = True
    s.poll()
    s.close_session(0)
    assert ex.released == [0]


def test_max_batch_and_rotation():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=100, slots=1, max_batch=2)
    for sid in range(3):
        s.open_session(SessionSpec(sid, 1))
        s.submit(sid, f"s{sid}")
    s.poll()
    assert ex.launched[0]["reqs"] == [(0, "s0"), (1, "s1")]
    ex.launched[0]["done"] = True
    s.poll()
    assert ex.launched[1]["reqs"] == [(2, "s2")]


def test_cancelled_requests_never_reach_the_device():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=1)
    s.open_session(SessionSpec(0, 1))
    s.open_session(SessionSpec(1, 1))
    a0 = s.submit(0, "a0")
    a1 = s.submit(0, "a1")
    a2 = s.submit(0, "a2")
    b0 = s.submit(1, "b0")
    s.poll()                                           # batch {a0, b0} on the device
    assert ex.launched[0]["reqs"] == [(0, "a0"), (1, "b0")]
    assert not s.cancel(a0)                            # in flight: runs to completion
    assert s.cancel(a1) and a1.cancelled
    assert not s.cancel(a1)                            # already withdrawn
    ex.launched[0]["done"] = True
    s.poll()                                           # next batch skips a1
    assert ex.launched[1]["reqs"] == [(0, "a2")]
    assert s.stats.cancelled == 1
    ex.launched[1]["done"] = True
    s.poll()
    assert not s.has_work()
    assert [r.tf for r in s.completed] == ["a0", "b0", "a2"]


def test_cancel_session_edits_then_close():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=1)
    s.open_session(SessionSpec(0, 4))
    reqs = [s.submit(0, f"e{i}") for i in range(5)]
    s.poll()                                           # e0 on the device
    assert s.cancel_session_edits(0) == 4
    assert all(r.cancelled for r in reqs[1:]) and not reqs[0].cancelled
    with pytest.raises(RuntimeError):
        s.close_session(0)                             # e0 still in flight
    ex.launched[0]["done"] = True
    s.poll()
    s.close_session(0)
    assert ex.released == [0] and s.used == 0 and len(ex.launched) == 1


def test_withdraw_a_waiting_session():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=1)
    assert s.open_session(SessionSpec(0, 8))
    assert not s.open_session(SessionSpec(1, 5))       # waits for budget
    assert not s.open_session(SessionSpec(2, 2))       # queued behind 1
    assert s.withdraw_waiting(1)                       # 2 now fits and is admitted
    assert ex.admitted == [0, 2] and s.used == 10
    assert not s.withdraw_waiting(1)


class EvictExec(FakeExec):
    def __init__(self):
        super().__init__()
        self.events = []

    def evict(self, sid):
        self.events.append(("evict", sid))

    def readmit(self, spec):
        self.events.append(("readmit", spec.sid))


def _finish_all(ex, sch):
    for h in ex.launched:
        h["done"] = True
    sch.poll()


def test_eviction_frees_room_from_the_least_recently_used_idle_session():
    ex = EvictExec()
    sch = Scheduler(ex, budget_bytes=100, slots=1, evict_idle=True)
    for sid in (0, 1):
        assert sch.open_session(SessionSpec(sid, 50))
    sch.submit(0, "a")                        # session 0 used last
    sch.poll()
    _finish_all(ex, sch)
    # a third session needs room: session 1 (never used) goes, session 0 stays
    assert sch.open_session(SessionSpec(2, 50))
    assert ex.events == [("evict", 1)] and sch.used == 100
    assert set(sch.sessions) == {0, 2} and set(sch.evicted) == {1}
    assert sch.stats.evictions == 1


def test_busy_or_pending_sessions_are_never_evicted():
    ex = EvictExec()
    sch = Scheduler(ex, budget_bytes=100, slots=1, evict_idle=True)
    for sid in (0, 1):
        sch.open_session(SessionSpec(sid, 50))
    sch.submit(0, "a")
    sch.poll()                                # session 0 on the device
    sch.submit(1, "b")                        # session 1 pending (slot busy)
    assert not sch.open_session(SessionSpec(2, 50))
    assert ex.events == [] and [sp.sid for sp in sch.waiting] == [2]
    _finish_all(ex, sch)                      # 0 idle now; 1's edit launched
    # session 0 is idle and is evicted for session 2; session 1 is on the device
    assert ex.events == [("evict", 0)] and 2 in sch.sessions
    assert ex.admitted == [0, 1, 2]


def test_an_edit_of_an_evicted_session_readmits_it_in_order():
    ex = EvictExec()
    sch = Scheduler(ex, budget_bytes=100, slots=2, evict_idle=True)
    sch.open_session(SessionSpec(0, 60))
    sch.open_session(SessionSpec(1, 60))      # evicts 0
    assert ex.events == [("evict", 0)]
    r1 = sch.submit(0, "x")                   # 0 is evicted: queued for readmission
    r2 = sch.submit(0, "y")
    assert [sp.sid for sp in sch.waiting] == [0]
    sch.poll()                                # 1 is idle: evicted, 0 readmitted, x launched
    assert ex.events == [("evict", 0), ("evict", 1), ("readmit", 0)]
    assert ex.launched[-1]["reqs"] == [(0, "x")]
    _finish_all(ex, sch)
    assert ex.launched[-1]["reqs"] == [(0, "y")]
    _finish_all(ex, sch)
    assert r1.t_done is not None and r2.t_done is not None and not sch.has_work()
    assert sch.stats.readmissions == 1 and sch.used == 60
    assert ex.admitted == [0, 1]              # readmission is not a new admission


def test_no_eviction_unless_enabled_and_closing_an_evicted_session():
    ex = EvictExec()
    sch = Scheduler(ex, budget_bytes=100, slots=1)
    sch.open_session(SessionSpec(0, 60))
    assert not sch.open_session(SessionSpec(1, 60))
    assert ex.events == []
    ex2 = EvictExec()
    sch2 = Scheduler(ex2, budget_bytes=100, slots=1, evict_idle=True)
    sch2.open_session(SessionSpec(0, 60))
    sch2.open_session(SessionSpec(1, 60))     # evicts 0
    sch2.submit(0, "x")                       # 0 waits for readmission
    sch2.close_session(0)                     # closing drops the waiting readmission too
    assert not sch2.waiting and 0 not in sch2.evicted and ex2.released == [0]
    assert sch2.used == 60
    with pytest.raises(KeyError):
        sch2.submit(0, "z")


def test_cancelling_an_evicted_sessions_edits_drops_its_readmission():
    ex = EvictExec()
    sch = Scheduler(ex, budget_bytes=100, slots=1, evict_idle=True)
    sch.open_session(SessionSpec(0, 60))
    sch.open_session(SessionSpec(1, 60))      # evicts 0
    sch.submit(0, "x")
    assert sch.cancel_session_edits(0) == 1
    assert not sch.waiting
    sch.poll()
    assert ("readmit", 0) not in ex.events and not sch.has_work()


class CheckingExec(EvictExec):
    """Fake executor that checks, at every call, what the device side may assume: a
    session is evicted only when nothing of it is on the device, launched only while
    resident, and readmitted only after an eviction."""

    def __init__(self):
        super().__init__()
        self.resident, self.on_device = set(), set()

    def admit(self, spec):
        assert spec.sid not in self.resident
        self.resident.add(spec.sid)
        super().admit(spec)

    def release(self, sid):
        assert sid not in self.on_device
        self.resident.discard(sid)
        super().release(sid)

    def evict(self, sid):
        assert sid in self.resident and sid not in self.on_device
        self.resident.discard(sid)
        super().evict(sid)

    def readmit(self, spec):
        assert spec.sid not in self.resident
        self.resident.add(spec.sid)
        super().readmit(spec)

    def launch(self, slot, reqs):
        for r in reqs:
            assert r.session in self.resident and r.session not in self.on_device
            self.on_device.add(r.session)
        return super().launch(slot, reqs)

    def finish(self, h):
        h["done"] = True
        for sid, _ in h["reqs"]:
            self.on_device.discard(sid)


@pytest.mark.parametrize("seed", range(6))
def test_random_workload_with_eviction_keeps_invariants(seed):
    import random
    rnd = random.Random(seed)
    ex = CheckingExec()
    sch = Scheduler(ex, budget_bytes=100, slots=rnd.choice([1, 2, 3]),
                    max_batch=rnd.choice([1, 3, 64]), evict_idle=True)
    sizes = {sid: rnd.choice([10, 20, 30, 45]) for sid in range(8)}
    opened, closed, submitted = set(), set(), {}
    for step in range(400):
        op = rnd.random()
        if op < 0.1 and len(opened) < len(sizes):
            sid = len(opened)
            sch.open_session(SessionSpec(sid, sizes[sid]))
            opened.add(sid)
        elif op < 0.7 and opened - closed:
            sid = rnd.choice(sorted(opened - closed))
            if sid in sch.sessions or sid in sch.evicted:
                submitted.setdefault(sid, []).append(sch.submit(sid, (sid, step)))
        elif op < 0.9:
            for h in ex.launched:
                if not h["done"] and rnd.random() < 0.6:
                    ex.finish(h)
            sch.poll()
        elif op < 0.95 and submitted:
            sid = rnd.choice(sorted(submitted))
            q = [r for r in submitted[sid] if not r.cancelled and not r.t_done]
            if q:
                sch.cancel(rnd.choice(q))
        else:
            sch.poll()
        assert sch.used <= sch.budget
        assert sch.used == sum(sp.device_bytes for sp in sch.sessions.values())
        assert not (set(sch.sessions) & set(sch.evicted))
        assert sch._npending == sum(len(q) for q in sch.pending.values())
    # drain: the device finishes everything
    for _ in range(2000):
        if not sch.has_work():
            break
        for h in ex.launched:
            if not h["done"]:
                ex.finish(h)
        sch.poll()
    assert not sch.has_work()
    # every edit ran or was cancelled, and each session's edits ran in submission order
    done = {r.rid for r in sch.completed}
    for sid, reqs in submitted.items():
        ran = [r for r in reqs if not r.cancelled]
        assert all(r.rid in done for r in ran)
        order = [tf for h in ex.launched for s, tf in h["reqs"] if s == sid]
        assert order == [r.tf for r in ran]
    assert sch.stats.evictions > 0 and sch.stats.readmissions > 0


def test_edits_of_a_waiting_session_run_after_admission():
    """Edits may be submitted to a session that waits for admission: they stay queued,
    none reaches the device, and once a session leaves and frees budget the waiting one is
    admitted and its edits run in order; the admission wait is recorded."""
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=2)
    assert s.open_session(SessionSpec(0, 8))
    ex.t = 1.0
    assert not s.open_session(SessionSpec(1, 5))        # waits
    s.submit(1, "w0")
    s.submit(1, "w1")
    s.poll()
    assert ex.launched == [] and s.has_work()
    ex.t = 4.0
    s.close_session(0)                                  # frees the budget: 1 is admitted
    assert ex.admitted == [0, 1] and s.stats.admission_waits == [0.0, 3.0]
    s.poll()
    assert [h["reqs"] for h in ex.launched] == [[(1, "w0")]]
    with pytest.raises(KeyError):
        s.submit(7, "x")                                # never opened


def test_several_edits_per_session_in_one_batch():
    """With edits_per_session = 3 a batch takes up to three of a session's oldest edits,
    in order, and the session stays out of further batches until it completes."""
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=2, max_batch=5, edits_per_session=3)
    for sid in range(2):
        s.open_session(SessionSpec(sid, 1))
    for k in range(5):
        s.submit(0, f"a{k}")
    s.submit(1, "b0")
    s.submit(1, "b1")
    s.poll()
    assert ex.launched[0]["reqs"] == [(0, "a0"), (0, "a1"), (0, "a2"), (1, "b0"), (1, "b1")]
    assert len(ex.launched) == 1                        # both sessions on the device
    ex.launched[0]["done"] = True
    s.poll()
    assert ex.launched[1]["reqs"] == [(0, "a3"), (0, "a4")]
    ex.launched[1]["done"] = True
    s.drain()
    assert [r.tf for r in s.completed] == ["a0", "a1", "a2", "b0", "b1", "a3", "a4"]


def test_closing_a_session_that_never_was_admitted():
    ex = FakeExec()
    s = Scheduler(ex, budget_bytes=10, slots=1)
    s.open_session(SessionSpec(0, 10))
    s.open_session(SessionSpec(1, 4))
    s.submit(1, "x")
    s.close_session(1)                                  # leaves the queue, edits dropped
    assert not s.waiting and not s.has_work() and ex.admitted == [0]
    with pytest.raises(KeyError):
        s.close_session(1)
