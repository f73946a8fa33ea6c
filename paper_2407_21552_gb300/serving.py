"""Serving loop: TF edits from many sessions, continuously batched onto one GPU.

Each session is one volume whose partitioned distance maps (§3.1) stay resident on the
device.  Sessions are admitted while their device bytes fit the HBM budget (§5: the
PDMs take n x volumesize / b^3 bytes); the others wait until a session leaves.  TF edits
arrive at any time.  Whenever a batch slot is free, the scheduler takes, for every session
with pending edits and no edit on the device, its oldest one (so every edit gets the map
of its own TF, and a session's working memory is used by one batch at a time), and hands
the batch to the executor, which runs it on the slot's stream without waiting; batches of
different sessions overlap on the device.  A request completes when its batch's
completion event has fired; its latency is arrival to completion.  An edit can be withdrawn
until it joins a batch; a session still waiting for admission can be withdrawn too.

With eviction enabled, a session that needs room (a new one, or an evicted one that got an
edit) evicts the least recently used admitted sessions that are idle (no edit pending or
on the device): their maps move to host memory and their budget is freed.  An evicted
session stays open; its next edit queues it for readmission, which copies the maps back
without recomputing them (the PDMs depend on the volume only, §3.1).

Edits may be submitted to a session still waiting for admission; they run once it is
admitted, and the time each session waited for admission is recorded.  With
`edits_per_session` > 1 a batch takes up to that many of a session's oldest edits at once
(the executor then combines them reading each map plane once); a session still has at
most one batch on the device.  A session's maps can also be built at admission (the
executor's payload gives a builder): the build is queued on a side stream and the
session's first batch waits for it on the device.

The scheduler (`Scheduler`) holds no GPU state and is tested with a fake executor; the
executor for the GPU (`DeviceExecutor`) does every step through libdm: pinned host TFs
are handed to the kernels as they are (the active-set step reads their alpha channel once
per edit over the CPU-GPU link), other TFs are copied to the session's device TF buffer on
the slot's stream; then one
dm_update_tf_batch, or dm_update_tf_batch_ws when a session has several edits in the batch
(or, for the comparison server, one dm_full_recompute per edit).
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    session: int
    tf: object                 # host TF (pinned float32 [N][4]) or anything the executor takes
    t_arrival: float
    rid: int = 0
    t_submit: float = 0.0
    t_done: float = 0.0
    cancelled: bool = False


@dataclass
class SessionSpec:
    sid: int
    device_bytes: int          # bytes the session keeps resident while admitted
    payload: object = None     # executor-specific (volume, config, ...)


@dataclass
class Batch:
    slot: int
    requests: list
    handle: object = None


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    batches: int = 0
    batch_sizes: list = field(default_factory=list)
    admitted: list = field(default_factory=list)
    rejected_waits: int = 0
    cancelled: int = 0
    evictions: int = 0
    readmissions: int = 0
    admission_waits: list = field(default_factory=list)   # open -> admitted, per session
    max_used: int = 0


class Scheduler:
    """Admission by budget, per-session FIFO, at most one batch of a session on the device
    at a time (holding up to `edits_per_session` of its edits), a fixed number of batches
    in flight.  `executor` provides admit(spec), release(sid),
    launch(slot, requests) -> handle, done(handle) -> bool, and clock() -> seconds; with
    `evict_idle`, also evict(sid) and readmit(spec)."""

    def __init__(self, executor, budget_bytes: int, slots: int = 2, max_batch: int = 64,
                 evict_idle: bool = False, edits_per_session: int = 1):
        self.ex = executor
        self.budget = int(budget_bytes)
        self.slots = int(slots)
        self.max_batch = int(max_batch)
        self.evict_idle = bool(evict_idle)
        self.edits_per_session = max(1, int(edits_per_session))
        self.t_open = {}                       # sid -> clock at open (until admitted)
        self.used = 0
        self.sessions = {}                     # sid -> spec (admitted)
        self.evicted = {}                      # sid -> spec (open, maps on the host)
        self.last_use = {}                     # sid -> launch counter (LRU order)
        self._uses = 0
        self.waiting = collections.deque()     # specs not admitted yet
        self.pending = collections.OrderedDict()   # sid -> deque of requests
        self._npending = 0                     # requests in all queues
        self.inflight = []                     # batches on the device
        self.busy = set()                      # sessions with an edit on the device
        self.free_slots = list(range(self.slots))
        self.stats = Stats()
        self.completed = []
        self._rid = 0

    # ------------------------------------------------------------------ sessions
    def open_session(self, spec: SessionSpec) -> bool:
        """Admit now if the budget allows (evicting idle sessions when enabled), else queue
        it; returns whether admitted."""
        if spec.device_bytes > self.budget:
            raise ValueError(f"session {spec.sid} needs more than the whole budget")
        self.t_open[spec.sid] = self.ex.clock()
        if not self.waiting and self._room_for(spec.device_bytes):
            self._admit(spec)
            return True
        self.waiting.append(spec)
        self.stats.rejected_waits += 1
        return False

    def _admit(self, spec):
        if spec.sid in self.evicted:
            del self.evicted[spec.sid]
            self.ex.readmit(spec)
            self.stats.readmissions += 1
        else:
            self.ex.admit(spec)
            self.stats.admitted.append(spec.sid)
            t0 = self.t_open.pop(spec.sid, None)
            if t0 is not None:
                self.stats.admission_waits.append(self.ex.clock() - t0)
        self.sessions[spec.sid] = spec
        self.used += spec.device_bytes
        self.stats.max_used = max(self.stats.max_used, self.used)
        self.last_use[spec.sid] = self._uses

    def _idle(self, sid) -> bool:
        return sid not in self.busy and not self.pending.get(sid)

    def _room_for(self, nbytes: int) -> bool:
        """Whether nbytes fit the budget, after evicting least recently used idle sessions
        if eviction is enabled (nothing is evicted unless enough can be freed)."""
        if self.used + nbytes <= self.budget:
            return True
        if not self.evict_idle:
            return False
        idle = sorted((sid for sid in self.sessions if self._idle(sid)),
                      key=lambda sid: self.last_use.get(sid, 0))
        need, victims = self.used + nbytes - self.budget, []
        for sid in idle:
            if need <= 0:
                break
            victims.append(sid)
            need -= self.sessions[sid].device_bytes
        if need > 0:
            return False
        for sid in victims:
            spec = self.sessions.pop(sid)
            self.ex.evict(sid)
            self.used -= spec.device_bytes
            self.evicted[sid] = spec
            self.stats.evictions += 1
        return True

    def _admit_waiting(self):
        while self.waiting and self._room_for(self.waiting[0].device_bytes):
            self._admit(self.waiting.popleft())

    def close_session(self, sid: int):
        """Leave once no edit of the session is pending or in flight; frees its budget."""
        if any(r.session == sid for b in self.inflight for r in b.requests):
            raise RuntimeError("session has edits in flight")
        self._npending -= len(self.pending.pop(sid, ()))
        self.last_use.pop(sid, None)
        if sid not in self.sessions and sid not in self.evicted:
            if not self.withdraw_waiting(sid):  # never admitted: just leave the queue
                raise KeyError(f"session {sid} is not open")
            self.t_open.pop(sid, None)
            return
        if sid in self.evicted:                 # maps on the host: nothing on the device
            self.evicted.pop(sid)
            self.waiting = collections.deque(sp for sp in self.waiting if sp.sid != sid)
            self.ex.release(sid)
        else:
            spec = self.sessions.pop(sid)
            self.ex.release(sid)
            self.used -= spec.device_bytes
        self._admit_waiting()

    # ------------------------------------------------------------------ requests
    def submit(self, sid: int, tf, t_arrival: float | None = None) -> Request:
        """Queue an edit of an admitted session, of one still waiting for admission, or of
        an evicted one (which then waits for readmission)."""
        if sid not in self.sessions and sid not in self.evicted and \
                all(sp.sid != sid for sp in self.waiting):
            raise KeyError(f"session {sid} is not open")
        if sid in self.evicted and all(sp.sid != sid for sp in self.waiting):
            self.waiting.append(self.evicted[sid])
        r = Request(session=sid, tf=tf,
                    t_arrival=self.ex.clock() if t_arrival is None else t_arrival,
                    rid=self._rid)
        self._rid += 1
        self.pending.setdefault(sid, collections.deque()).append(r)
        self._npending += 1
        return r

    def cancel(self, req: Request) -> bool:
        """Withdraw an edit that has not reached the device yet.  An edit already in a
        batch runs to completion (its device work is not interrupted); returns whether
        the edit was withdrawn."""
        q = self.pending.get(req.session)
        if req.cancelled or q is None or req not in q:
            return False
        q.remove(req)
        self._npending -= 1
        req.cancelled = True
        self.stats.cancelled += 1
        return True

    def cancel_session_edits(self, sid: int) -> int:
        """Withdraw every edit of a session that has not reached the device; returns how
        many.  The session can close once its in-flight edit (if any) completes."""
        q = self.pending.get(sid)
        if not q:
            return 0
        n = len(q)
        for r in q:
            r.cancelled = True
        q.clear()
        self._npending -= n
        self.stats.cancelled += n
        if sid in self.evicted:                 # nothing left to readmit it for
            self.waiting = collections.deque(sp for sp in self.waiting if sp.sid != sid)
        return n

    def withdraw_waiting(self, sid: int) -> bool:
        """Drop a session that is still waiting for admission (it never held budget)."""
        for spec in list(self.waiting):
            if spec.sid == sid and sid not in self.evicted:
                self.waiting.remove(spec)
                self._admit_waiting()
                return True
        return False

    def has_work(self) -> bool:
        return bool(self.inflight) or self._npending > 0

    # ------------------------------------------------------------------ progress
    def poll(self):
        """Retire finished batches, then launch new ones while slots are free."""
        still = []
        for b in self.inflight:
            if self.ex.done(b.handle):
                t = self.ex.clock()
                for r in b.requests:
                    r.t_done = t
                    self.stats.latencies.append(t - r.t_arrival)
                    self.completed.append(r)
                    self.busy.discard(r.session)
                self.free_slots.append(b.slot)
            else:
                still.append(b)
        self.inflight = still
        self._admit_waiting()                   # room freed by retired batches
        while self.free_slots and self._npending:
            reqs = []
            for sid, q in self.pending.items():
                if q and sid not in self.busy and sid in self.sessions:
                    for _ in range(min(len(q), self.edits_per_session,
                                       self.max_batch - len(reqs))):
                        reqs.append(q.popleft())
                    if len(reqs) == self.max_batch:
                        break
            if not reqs:
                break
            self._npending -= len(reqs)
            slot = self.free_slots.pop(0)
            t = self.ex.clock()
            for r in reqs:
                r.t_submit = t
            self.busy.update(r.session for r in reqs)
            self._uses += 1
            for r in reqs:
                self.last_use[r.session] = self._uses
            b = Batch(slot=slot, requests=reqs)
            b.handle = self.ex.launch(slot, reqs)
            self.inflight.append(b)
            self.stats.batches += 1
            self.stats.batch_sizes.append(len(reqs))
            # rotate so that sessions with many pending edits do not starve the others
            for sid in dict.fromkeys(r.session for r in reqs):
                self.pending.move_to_end(sid)

    def drain(self, timeout_s: float = 60.0):
        t0 = time.perf_counter()
        while self.has_work():
            self.poll()
            if time.perf_counter() - t0 > timeout_s:
                raise TimeoutError("serving loop did not drain")


class DeviceExecutor:
    """Runs batches through libdm on one device.  payload of a SessionSpec: dict with
    'engine' (maps.PartitionedDistanceMaps, built) and optionally 'volume'; or, for maps
    built at admission, 'build': a callable(stream) that creates the engine, queues its
    precompute on `stream` and returns (engine, volume or None)."""

    def __init__(self, slots: int = 2, mode: str = "partitioned", device="cuda",
                 edits_per_session: int = 1, max_batch: int = 64, tf_from_host: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.mode = mode                      # "partitioned" or "full"
        # pinned host TFs are read by the kernels in place (one CTA per edit reads its
        # alpha channel over the CPU-GPU link) instead of being copied first
        self.tf_from_host = bool(tf_from_host)
        self.edits_per_session = max(1, int(edits_per_session))
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(slots)]
        # one completion event per slot: a slot takes a new batch only after its last one
        # completed, so the event is free to record again
        self.events = [torch.cuda.Event() for _ in range(slots)]
        self.sessions = {}
        self.evicted = {}                     # sid -> engine whose maps are on the host
        self.side = torch.cuda.Stream(device=self.device)   # eviction / readmission copies
        self.results = {}                     # rid -> device D' (kept if keep_results)
        self.keep_results = False
        self.ws = None                        # per-slot workspaces of the several-edit batch
        from . import _abi as A
        self._lib = A.load()
        if self.edits_per_session > 1 and mode == "partitioned":
            self.ws_bytes = A.dm_batch_workspace_bytes(max_batch)
            self.ws = [torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
                       for _ in range(slots)]
        # per slot: the C item array of its batches (filled in place) and the raw stream
        self._items = [(A.dm_batch_item * max_batch)() for _ in range(slots)]
        self._sh = [ctypes.c_void_p(st.cuda_stream) for st in self.streams]

    def clock(self):
        return time.perf_counter()

    def admit(self, spec):
        torch = self.torch
        volume = spec.payload.get("volume")
        if "build" in spec.payload:           # maps built now, on the side stream
            eng, volume = spec.payload["build"](self.side)
            ready = torch.cuda.Event()
            ready.record(self.side)
            eng.ready_event = ready
            spec.payload["engine"] = eng
        eng = spec.payload["engine"]
        E = self.edits_per_session
        tf = [[torch.empty((eng.N, 4), dtype=torch.float32, device=self.device)
               for _ in range(E)] for _ in self.streams]
        out = [[torch.empty(eng.G, dtype=torch.uint8, device=self.device) for _ in range(E)]
               for _ in self.streams]
        self.sessions[spec.sid] = dict(
            engine=eng, volume=volume, spec=spec, tf=tf, out=out,
            tf_ptr=[[t.data_ptr() for t in row] for row in tf],
            out_ptr=[[t.data_ptr() for t in row] for row in out])
    def release(self, sid):
        """The session left (nothing of it pending or on the device): maps built at
        admission are dropped, so their device memory goes back to torch's allocator."""
        s = self.sessions.pop(sid, None)
        self.evicted.pop(sid, None)
        if s is not None and "build" in s["spec"].payload:
            s["spec"].payload.pop("engine", None)
            s["engine"].close()

    def evict(self, sid):
        """Maps to pinned host memory, device buffers freed once the copy has run (the
        scheduler evicts only sessions with nothing pending or on the device).  The copy is
        queued on the side stream; the host does not wait for it."""
        s = self.sessions.pop(sid)
        s["engine"].offload(self.side, wait=False)
        self.evicted[sid] = s["engine"]

    def readmit(self, spec):
        """Maps back to the device (no recompute), queued on the side stream; the session's
        next batch waits for that copy on the device, not on the host."""
        self.evicted.pop(spec.sid, None)
        spec.payload["engine"].reload(self.side, wait=False)
        self.admit(spec)

    def launch(self, slot, requests):
        from . import _abi as A
        torch = self.torch
        st = self.streams[slot]
        sh = self._sh[slot]
        arr = self._items[slot]
        copies, used = [], {}
        for i, r in enumerate(requests):
            s = self.sessions[r.session]
            eng = s["engine"]
            if eng.ready_event is not None:       # built or readmitted: maps in transit
                st.wait_event(eng.ready_event)
                if eng.ready_event.query():
                    eng.ready_event = None
            e = used.get(r.session, 0)            # the request's place in its session
            used[r.session] = e + 1
            if self.tf_from_host and not r.tf.is_cuda and r.tf.is_pinned():
                tfp = r.tf.data_ptr()             # read in place; the request keeps it alive
            else:
                copies.append((s["tf"][slot][e], r.tf))
                tfp = s["tf_ptr"][slot][e]
            it = arr[i]
            it.ctx = eng.ctx
            it.d_tf_rgba = tfp
            it.d_out = s["out_ptr"][slot][e]
        if copies:
            with torch.cuda.stream(st):
                for dst, src in copies:
                    dst.copy_(src, non_blocking=True)
        n = len(requests)
        if self.mode == "partitioned":
            if any(v > 1 for v in used.values()):
                st_ = self._lib.dm_update_tf_batch_ws(arr, n, None, self.ws[slot].data_ptr(),
                                                      self.ws_bytes, sh)
                where = "dm_update_tf_batch_ws"
            else:
                st_ = self._lib.dm_update_tf_batch(arr, n, None, sh)
                where = "dm_update_tf_batch"
            if st_ != A.DM_OK:
                raise A.DmError(st_, where, self._lib.dm_last_error_string(arr[0].ctx).decode())
        else:
            for i, r in enumerate(requests):
                v = self.sessions[r.session]["volume"]
                A.dm_full_recompute(arr[i].ctx, v.data_ptr() if v is not None else None,
                                    arr[i].d_tf_rgba, arr[i].d_out, sh)
        if self.keep_results:
            with torch.cuda.stream(st):
                used = {}
                for r in requests:
                    e = used.get(r.session, 0)
                    used[r.session] = e + 1
                    self.results[r.rid] = self.sessions[r.session]["out"][slot][e].clone()
        ev = self.events[slot]
        ev.record(st)
        return ev

    def done(self, handle):
        return handle.query()
