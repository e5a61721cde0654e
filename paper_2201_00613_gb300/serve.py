"""Request loop with continuous batching over the batched tiled step.

Requests (a fractal, a level, a seed and a step count) arrive over time.  The
loop admits an arrived request as soon as a slot is free and the device has
room for its two state buffers (checked against the free HBM the driver
reports, minus a reserve), seeds its state on the device, and from then on
advances it together with every other active request: each round runs one
batched launch per CA step (squeeze_batch_run) for the largest chunk of steps
that no active request overshoots.  Requests that arrive while a round is on
the GPU join at the next round boundary, so their work overlaps with that of
the requests already running.  A finished request's state stays on the
device; its latency is the time from arrival to the end of its last round.
A request that does not fit while nothing else of the loop is active can
never be admitted (no memory of the loop's will be given back): it is
rejected and recorded, and the loop goes on with the next one.
cancel() withdraws a request from any thread: at the next round boundary a
queued request is dropped before admission and an active one gives up its
slot and its buffers; a request that has already finished keeps its result.
All computation runs in the CUDA library; this module only schedules.  The
device side sits behind a small backend object (DeviceBackend), so the
scheduling can be exercised without a GPU.
"""
from __future__ import annotations

import dataclasses
import statistics
import threading
import time
from collections import deque


@dataclasses.dataclass
class Slot:
    request: object
    handle: object
    cur: object           # buffer that holds the current state
    other: object
    remaining: int
    admitted_s: float
    done_s: float = -1.0


class DeviceBackend:
    """The device operations the loop needs, through the C ABI and torch."""

    def __init__(self, device="cuda"):
        import torch

        from . import _lib as sq
        from . import inputs as I
        self.torch, self.sq, self.I = torch, sq, I
        self.device = torch.device(device)
        self._rec_bytes = {}   # handle pointer -> bytes of one border-record buffer

    def free_bytes(self) -> int:
        # Blocks that torch's caching allocator holds but no tensor uses are
        # free for the next request's buffers as well.
        free = self.torch.cuda.mem_get_info(self.device)[0]
        cached = (self.torch.cuda.memory_reserved(self.device)
                  - self.torch.cuda.memory_allocated(self.device))
        return free + max(0, cached)

    def handle(self, inst, level):
        h = self.sq.Handle(inst.fractal, inst.r)
        if level:
            try:
                self.sq.squeeze_set_tiled_level(h.h, min(level, inst.r))
            except self.sq.SqueezeError:
                pass   # keep the default level
        return h

    def cells(self, handle) -> int:
        return handle.cells

    def start(self, handle, inst):
        a = self.torch.empty(handle.cells, dtype=self.torch.uint8, device=self.device)
        b = self.torch.empty_like(a)
        self.sq.squeeze_init_bernoulli(handle.h, a, inst.seed, self.I.p_q24(inst.p))
        # Each state buffer carries the border records of its contents, written
        # once here for the start and kept current by every batched run, so a
        # rebuilt batch needs no records-only launch.
        n = self._rec_bytes.get(handle.h)
        if n is None:
            n = self._rec_bytes[handle.h] = self.sq.squeeze_record_bytes(handle.h)
        a._sq_rec = b._sq_rec = None
        if n:
            a._sq_rec = self.torch.empty(n // 4, dtype=self.torch.int32, device=self.device)
            b._sq_rec = self.torch.empty_like(a._sq_rec)
            self.sq.squeeze_write_records(handle.h, a, a._sq_rec)
        return a, b

    def batch(self, slots):
        batch = self.sq.squeeze_batch_create_with_records(
            [(s.handle.h, s.cur, s.other) for s in slots],
            [(s.cur._sq_rec, s.other._sq_rec) for s in slots])
        self.sq.squeeze_batch_configure(batch, 0, 0, False)  # round lengths vary: no graphs
        return batch

    def run(self, batch, k: int):
        self.sq.squeeze_batch_run(batch, k)
        self.torch.cuda.current_stream(self.device).synchronize()

    def destroy(self, batch):
        self.sq.squeeze_batch_destroy(batch)

    def close_handle(self, handle):
        self._rec_bytes.pop(handle.h, None)
        handle.close()


class RequestLoop:
    """Continuous-batching loop on one device."""

    def __init__(self, device="cuda", max_slots=64, chunk=25, reserve_bytes=4 << 30,
                 keep_results=False, levels=None, backend=None):
        self.backend = backend if backend is not None else DeviceBackend(device)
        self.max_slots = max_slots
        self.chunk = chunk
        self.reserve = reserve_bytes
        self.keep = keep_results
        self.levels = levels or {}
        self.finished = []
        self.handles = {}   # (fractal name, r) -> handle, shared by the requests of that shape
        self.rounds = 0
        self.batches_built = 0
        self.refused_for_memory = 0  # requests that had to wait for memory (each counted once)
        self.rejected = []           # requests that could not fit even with nothing else active
        self.max_active = 0
        self._waited = set()
        self.cancelled = []          # (request id, True if it was active when withdrawn)
        self._cancel = set()
        self._cancel_lock = threading.Lock()

    def cancel(self, rid) -> None:
        """Withdraw request `rid` at the next round boundary (thread-safe)."""
        with self._cancel_lock:
            self._cancel.add(rid)

    def _take_cancellations(self):
        with self._cancel_lock:
            ids, self._cancel = self._cancel, set()
        return ids

    def _fits(self, inst) -> bool:
        # two states, the batch's two border-record buffers (at most a quarter
        # of a state each: the carpet's eight halo rings) and tables
        cells = inst.fractal.cells(inst.r)
        need = 2 * cells + cells // 2 + (1 << 20)
        return self.backend.free_bytes() - need >= self.reserve

    def _handle(self, inst):
        key = (inst.fractal.name, inst.r)
        h = self.handles.get(key)
        if h is None:
            h = self.backend.handle(inst, self.levels.get(inst.fractal.name))
            self.handles[key] = h
        return h

    def close(self):
        for h in self.handles.values():
            self.backend.close_handle(h)
        self.handles = {}

    def _admit(self, req, now):
        inst = req.instance
        h = self._handle(inst)
        a, b = self.backend.start(h, inst)
        return Slot(req, h, a, b, req.n_steps, now)

    def run(self, requests, max_seconds=None):
        """Serve `requests` (sorted by arrival); returns a summary dict."""
        be = self.backend
        pending = deque(sorted(requests, key=lambda r: r.arrival_s))
        active = []
        batch, members = None, ()
        cell_updates = 0
        t0 = time.perf_counter()
        while pending or active:
            now = time.perf_counter() - t0
            if max_seconds and now > max_seconds:
                break
            withdrawn = self._take_cancellations()
            if withdrawn:
                kept = deque()
                for req in pending:
                    if req.rid in withdrawn:
                        self.cancelled.append((req.rid, False))
                    else:
                        kept.append(req)
                pending = kept
                dropped = [s for s in active if s.request.rid in withdrawn]
                if dropped:
                    if batch:           # the batch refers to the dropped buffers: end it first
                        be.destroy(batch)
                    batch, members = None, ()
                    for s in dropped:
                        self.cancelled.append((s.request.rid, True))
                        s.cur = s.other = None
                    active = [s for s in active if s.request.rid not in withdrawn]
                if not pending and not active:
                    break
            while pending and pending[0].arrival_s <= now and len(active) < self.max_slots:
                head = pending[0]
                if self._fits(head.instance):
                    active.append(self._admit(pending.popleft(), now))
                    continue
                if not active:
                    # Nothing of this loop is running, so no memory will be
                    # given back: the request can never be admitted.
                    self.rejected.append(pending.popleft().rid)
                    continue
                if head.rid not in self._waited:
                    self._waited.add(head.rid)
                    self.refused_for_memory += 1
                break
            self.max_active = max(self.max_active, len(active))
            if not active:
                if pending:
                    time.sleep(max(0.0, min(0.01, pending[0].arrival_s - now)))
                continue
            ids = tuple(id(s) for s in active)
            if ids != members:
                if batch:
                    be.destroy(batch)
                batch = be.batch(active)
                members = ids
                self.batches_built += 1
            k = min(self.chunk, min(s.remaining for s in active))
            be.run(batch, k)
            self.rounds += 1
            end = time.perf_counter() - t0
            still = []
            for s in active:
                s.remaining -= k
                cell_updates += k * be.cells(s.handle)
                if k % 2:
                    s.cur, s.other = s.other, s.cur
                if s.remaining == 0:
                    s.done_s = end
                    self.finished.append(s)
                else:
                    still.append(s)
            if len(still) != len(active):
                # the batch's parity restarts with the next membership; buffers
                # are passed as (current, other) again then.
                be.destroy(batch)
                batch, members = None, ()
                for s in active:
                    if s.remaining == 0 and not self.keep:
                        s.other = None
                        s.cur = None
            active = still
        if batch:
            be.destroy(batch)
        makespan = time.perf_counter() - t0
        lat = [s.done_s - s.request.arrival_s for s in self.finished]
        lat.sort()
        pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))] if lat else None
        return {
            "requests": len(self.finished),
            "makespan_s": makespan,
            "cell_updates": cell_updates,
            "cell_updates_per_s": cell_updates / makespan if makespan > 0 else 0.0,
            "latency_p50_s": pct(0.50),
            "latency_p99_s": pct(0.99),
            "latency_mean_s": statistics.mean(lat) if lat else None,
            "rounds": self.rounds,
            "batches_built": self.batches_built,
            "refused_for_memory": self.refused_for_memory,
            "rejected_for_memory": len(self.rejected),
            "max_active": self.max_active,
            "cancelled": len(self.cancelled),
        }
