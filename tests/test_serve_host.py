"""The request loop's scheduling, on the CPU, with a stand-in device backend.

The backend counts the CA steps applied to each request's state and the
memory its buffers hold, so the loop's decisions can be checked exactly:
every request gets exactly its number of steps, no round overshoots a
request or exceeds the chunk, the slot limit and the memory reserve hold,
and requests that arrive later still finish.
"""
import weakref

from paper_2201_00613_gb300 import inputs as I
from paper_2201_00613_gb300.serve import RequestLoop


class _State:
    """A request's state: the steps applied so far (both buffers share it)."""

    def __init__(self, backend, nbytes):
        self.steps = 0
        backend.live += nbytes
        weakref.finalize(self, backend.release, nbytes)


class FakeBackend:
    def __init__(self, total_bytes=1 << 50):
        self.total = total_bytes
        self.live = 0
        self.max_live = 0
        self.batch_sizes = []
        self.round_lengths = []
        self.handles_closed = 0

    def release(self, nbytes):
        self.live -= nbytes

    def free_bytes(self):
        return self.total - self.live

    def handle(self, inst, level):
        return (inst.fractal.name, inst.r, inst.fractal.cells(inst.r))

    def cells(self, handle):
        return handle[2]

    def start(self, handle, inst):
        st = _State(self, 2 * handle[2])
        self.max_live = max(self.max_live, self.live)
        return st, st

    def batch(self, slots):
        self.batch_sizes.append(len(slots))
        return [s.cur for s in slots]

    def run(self, batch, k):
        self.round_lengths.append(k)
        for st in batch:
            st.steps += k

    def destroy(self, batch):
        batch.clear()

    def close_handle(self, handle):
        self.handles_closed += 1


LEVELS = {"sierpinski_triangle": (4, 9), "sierpinski_carpet": (2, 4), "vicsek": (3, 6)}


def test_every_request_gets_exactly_its_steps():
    reqs = I.request_stream(seed=3, count=60, rate_per_s=1e5, levels=LEVELS, steps=(1, 40))
    be = FakeBackend()
    loop = RequestLoop(max_slots=8, chunk=7, keep_results=True, backend=be)
    out = loop.run(reqs)
    assert out["requests"] == len(reqs)
    assert sorted(s.request.rid for s in loop.finished) == list(range(len(reqs)))
    for s in loop.finished:
        assert s.cur.steps == s.request.n_steps, s.request.rid
        assert s.remaining == 0 and s.done_s >= s.admitted_s
    assert max(be.batch_sizes) <= 8
    assert max(be.round_lengths) <= 7 and min(be.round_lengths) >= 1
    assert out["rounds"] == len(be.round_lengths)
    assert out["cell_updates"] == sum(r.instance.fractal.cells(r.instance.r) * r.n_steps
                                      for r in reqs)
    assert out["latency_p50_s"] <= out["latency_p99_s"]
    loop.close()
    assert be.handles_closed == len({(r.instance.fractal.name, r.instance.r) for r in reqs})


def test_admission_holds_the_memory_reserve():
    f, r = I.TRIANGLE, 6
    reqs = [I.Request(i, 0.0, I.Instance(f, r, i), 5 + i % 3) for i in range(12)]
    # the loop asks for the two buffers, half a state for border records and
    # 1 MiB of headroom: room for three at a time
    be = FakeBackend(total_bytes=(1 << 20) + 3 * 2 * f.cells(r) + f.cells(r) // 2 + 100)
    loop = RequestLoop(max_slots=16, chunk=4, reserve_bytes=0, backend=be)
    out = loop.run(reqs, max_seconds=30)
    assert out["requests"] == len(reqs)
    assert be.max_live <= 3 * 2 * f.cells(r)
    assert max(be.batch_sizes) <= 3
    # each waiting request is counted once, however many rounds it waited
    assert 0 < out["refused_for_memory"] <= len(reqs) - 3
    assert out["rejected_for_memory"] == 0 and out["max_active"] == 3


def test_a_request_that_can_never_fit_is_rejected_and_the_loop_ends():
    f = I.TRIANGLE
    small, big = I.Instance(f, 5, 1), I.Instance(f, 9, 2)
    reqs = [I.Request(0, 0.0, small, 3), I.Request(1, 0.0, big, 3), I.Request(2, 0.0, small, 2)]
    # room for a small request's buffers, never for the big one's (no max_seconds: the
    # loop must end by itself)
    be = FakeBackend(total_bytes=(1 << 20) + 2 * f.cells(5) + f.cells(5) // 2 + 10)
    loop = RequestLoop(max_slots=4, chunk=4, reserve_bytes=0, backend=be)
    out = loop.run(reqs)
    assert loop.rejected == [1]
    assert out["rejected_for_memory"] == 1 and out["requests"] == 2
    assert sorted(s.request.rid for s in loop.finished) == [0, 2]
    assert be.round_lengths == [3, 2] and be.live == 0


def test_late_arrivals_join_and_finish():
    f = I.VICSEK
    reqs = [I.Request(0, 0.0, I.Instance(f, 5, 1), 30),
            I.Request(1, 0.02, I.Instance(f, 4, 2), 3),
            I.Request(2, 0.04, I.Instance(f, 3, 3), 1)]
    be = FakeBackend()
    loop = RequestLoop(max_slots=4, chunk=2, keep_results=True, backend=be)
    out = loop.run(reqs, max_seconds=30)
    assert out["requests"] == 3
    assert {s.request.rid: s.cur.steps for s in loop.finished} == {0: 30, 1: 3, 2: 1}


class _CancellingBackend(FakeBackend):
    """Withdraws the given requests when the loop starts a given round."""

    def __init__(self, loop_ref, at_round, rids):
        super().__init__()
        self.loop_ref, self.at_round, self.rids = loop_ref, at_round, rids
        self.runs = 0

    def run(self, batch, k):
        self.runs += 1
        if self.runs == self.at_round:
            for rid in self.rids:
                self.loop_ref[0].cancel(rid)
        super().run(batch, k)


def test_cancelled_requests_leave_and_the_rest_finish():
    reqs = I.request_stream(seed=9, count=40, rate_per_s=1e5, levels=LEVELS, steps=(20, 60))
    holder = []
    # cancel 3 requests after the second round: some are active by then, others still queued
    targets = [0, 1, 39]
    be = _CancellingBackend(holder, 2, targets)
    loop = RequestLoop(max_slots=4, chunk=5, keep_results=True, backend=be)
    holder.append(loop)
    out = loop.run(reqs)
    assert out["cancelled"] == 3 and out["requests"] == len(reqs) - 3
    gone = dict(loop.cancelled)
    assert sorted(gone) == sorted(targets)
    assert gone[0] and gone[1] and not gone[39]     # 0 and 1 were running, 39 still queued
    finished = {s.request.rid for s in loop.finished}
    assert finished == set(range(len(reqs))) - set(targets)
    for s in loop.finished:
        assert s.cur.steps == s.request.n_steps
    # results are kept (keep_results): exactly the finished requests still hold buffers
    import gc
    gc.collect()
    assert be.live == sum(2 * s.request.instance.fractal.cells(s.request.instance.r)
                          for s in loop.finished)


def test_cancelling_everything_ends_the_loop_and_frees_the_buffers():
    reqs = I.request_stream(seed=10, count=12, rate_per_s=1e5, levels=LEVELS, steps=(30, 50))
    holder = []
    be = _CancellingBackend(holder, 1, list(range(12)))
    loop = RequestLoop(max_slots=3, chunk=4, backend=be)
    holder.append(loop)
    out = loop.run(reqs)
    assert out["requests"] == 0 and out["cancelled"] == 12
    assert [active for _, active in loop.cancelled].count(True) == 3
    assert be.live == 0                     # no request holds a buffer any more


def test_cancelling_a_finished_or_unknown_request_changes_nothing():
    reqs = I.request_stream(seed=11, count=10, rate_per_s=1e5, levels=LEVELS, steps=(1, 3))
    be = FakeBackend()
    loop = RequestLoop(max_slots=10, chunk=8, keep_results=True, backend=be)
    out = loop.run(reqs)
    loop.cancel(0)
    loop.cancel(12345)
    out2 = loop.run([])
    assert out["requests"] == 10 and out2["cancelled"] == 0
    assert all(s.cur.steps == s.request.n_steps for s in loop.finished)
