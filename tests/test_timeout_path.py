"""The device-side timeout path of the tiled step, on the GPU.

Every wait of the tiled kernel on its bulk copies gives up after a limit and
latches DEVICE_TIMEOUT in the handle's status word.  The test makes the wait
run out without faulting anything: under the load-withholding hook the
kernel issues no bulk copy at all (so nothing is in flight), its first wait
on a buffer that nothing fills gives up after a 1 ms limit, and the launch
ends.  The status must say DEVICE_TIMEOUT within a bounded wall time, and
the next ordinary step on the same handle and context must be bit-exact
against the oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 12), (I.CARPET, 5), (I.VICSEK, 7)],
                         ids=["triangle12", "carpet5", "vicsek7"])
def test_withheld_loads_time_out_and_the_context_stays_usable(f, r):
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, 5, I.p_q24(0.5))
        start = a.clone()
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)   # program built, kernel loaded
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
        sq.squeeze_set_wait_limit(h.h, 1_000_000)               # 1 ms
        sq.squeeze_set_fault_injection(h.h, sq.SQUEEZE_FAULT_WITHHOLD_LOADS)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)
        status = sq.squeeze_device_status(h.h)                  # synchronises
        took = time.perf_counter() - t0
        assert status == sq.SQUEEZE_ERR_DEVICE_TIMEOUT
        assert took < 1.0, took
        assert torch.equal(a, start)                            # the input is untouched
        # back to normal on the same handle and context
        sq.squeeze_set_fault_injection(h.h, 0)
        sq.squeeze_set_wait_limit(h.h, 0)
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
        want = oracle.run_compact(f, r, start.cpu().numpy(), 1)
        assert np.array_equal(b.cpu().numpy(), want)


def test_wait_limit_and_fault_flags_are_validated():
    with sq.Handle(I.TRIANGLE, 4) as h:
        for bad in (1, 999, 10_000_000_001):
            with pytest.raises(sq.SqueezeError) as e:
                sq.squeeze_set_wait_limit(h.h, bad)
            assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_set_fault_injection(h.h, 2)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_set_wait_limit(h.h, 1000)
        sq.squeeze_set_wait_limit(h.h, 0)
