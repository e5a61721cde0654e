"""Request loop with continuous batching: results are the same alone and in the mix.

Requests arrive while others are on the GPU and join the running batch at the
next round; every served state must equal the request run alone through
squeeze_step (bit for bit), whatever the other requests were.
"""
import pytest

from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402
from paper_2201_00613_gb300.serve import RequestLoop  # noqa: E402

LEVELS = {"sierpinski_triangle": (6, 12), "sierpinski_carpet": (3, 5), "vicsek": (4, 7)}


def alone(inst, steps):
    with sq.Handle(inst.fractal, inst.r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, inst.seed, I.p_q24(inst.p))
        sq.squeeze_step(h.h, a, b, steps, sq.SQUEEZE_STEP_TILED)
        torch.cuda.synchronize()
        return (b if steps % 2 else a).clone()


def test_served_results_equal_solo_runs():
    reqs = I.request_stream(seed=6, count=40, rate_per_s=400.0, levels=LEVELS, steps=(5, 40))
    loop = RequestLoop(max_slots=16, chunk=7, keep_results=True)
    out = loop.run(reqs)
    assert out["requests"] == len(reqs)
    assert out["batches_built"] > 1 and out["rounds"] >= out["batches_built"]
    assert out["latency_p50_s"] > 0 and out["latency_p99_s"] >= out["latency_p50_s"]
    for s in loop.finished:
        assert torch.equal(s.cur, alone(s.request.instance, s.request.n_steps)), s.request.rid
    loop.close()


def test_admission_respects_free_memory():
    # Six requests of one shape arrive together; the reserve leaves room for
    # one request's buffers (plus slack for the library's own tables) but not
    # for two, so the others must wait for memory, one after the other.
    # Results are not kept, so each finished request gives its memory back.
    f, r = I.TRIANGLE, 15
    reqs = [I.Request(i, 0.0, I.Instance(f, r, 40 + i), 3 + i % 2) for i in range(6)]
    need = 2 * f.cells(r) + (1 << 20)
    loop = RequestLoop(max_slots=8, chunk=2, reserve_bytes=0)
    loop.reserve = loop.backend.free_bytes() - need - (24 << 20)
    out = loop.run(reqs, max_seconds=120)
    loop.close()
    assert out["requests"] == len(reqs) and out["rejected_for_memory"] == 0
    assert out["max_active"] == 1
    assert out["refused_for_memory"] == len(reqs) - 1
