"""The allocation-free step entry point, checked against squeeze_step.

squeeze_step_noalloc serves callers that may not allocate device memory (an
application that owns the whole memory budget, or latency-critical code that
cannot take cudaMalloc's device-wide synchronisation).  Its scratch lives in a
fixed device array shared by all calls, so the test makes two calls in a row,
each feeding the next, and compares every result bit for bit with the regular
tiled step.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402

B3, S23 = 1 << 3, (1 << 2) | (1 << 3)


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 12), (I.TRIANGLE, 16), (I.VICSEK, 7), (I.CARPET, 5),
                                 (I.TRIANGLE, 3)],
                         ids=["triangle12", "triangle16", "vicsek7", "carpet5", "triangle3"])
def test_noalloc_matches_tiled_step_on_two_calls_in_a_row(f, r):
    dev = torch.device("cuda:0")
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, 11, I.p_q24(0.5))
        start = a.clone()
        want1, want2 = torch.empty_like(a), torch.empty_like(a)
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)
        want1.copy_(b)
        sq.squeeze_step(h.h, b, a, 1, sq.SQUEEZE_STEP_TILED)
        want2.copy_(a)
        out1, out2 = torch.empty_like(a), torch.empty_like(a)
        st1 = sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, start, out1)
        st2 = sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, out1, out2)
        torch.cuda.synchronize()
        assert st1 == sq.SQUEEZE_OK and st2 == sq.SQUEEZE_OK
        assert torch.equal(out1, want1)
        assert torch.equal(out2, want2)


def test_noalloc_other_rule_matches():
    f, r = I.TRIANGLE, 10
    rule = ((1 << 3) | (1 << 6), (1 << 2) | (1 << 3))
    with sq.Handle(f, r) as h:
        sq.squeeze_set_rule(h.h, *rule)
        x = torch.from_numpy(I.bernoulli_bytes(4, h.cells, 0.5)).cuda()
        y = torch.empty_like(x)
        sq.squeeze_step(h.h, x, y, 1, sq.SQUEEZE_STEP_TILED)
        z = torch.empty_like(x)
        assert sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, *rule, x, z) == sq.SQUEEZE_OK
        assert torch.equal(y, z)


def test_noalloc_calls_after_the_first_take_no_device_memory():
    # The first call on a device loads the library's code and the static
    # array there (lazy module loading); later calls must not change the
    # device's free memory.
    f, r = I.VICSEK, 6
    n = f.k ** r
    x = torch.from_numpy(I.bernoulli_bytes(7, n, 0.5)).cuda()
    y, z = torch.empty_like(x), torch.empty_like(x)
    assert sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, x, y) == sq.SQUEEZE_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, y, z) == sq.SQUEEZE_OK
    assert sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, z, y) == sq.SQUEEZE_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_levels_beyond_its_scratch():
    f, r = I.TRIANGLE, 17
    n = f.k ** r
    x = torch.zeros(n, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(sq.SqueezeError) as e:
        sq.squeeze_step_noalloc(f.s, f.k, f.offsets, r, B3, S23, x, y)
    assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
    assert "static maximum" in str(e.value)
