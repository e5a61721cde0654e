"""Block-level layout (Sec. 3.5): rho x rho expanded micro-boxes per block.

The state at block level b (rho = s^b) must hold exactly the compact state's
cells: the seeded start, and every step, gathered back to compact order,
equal the oracle (small levels) and the compact tiled step (r = 16).  Its
size is the closed form k^(r-b) * rho^2 of the paper's memory table.
"""
import numpy as np
import pytest

import oracle
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402

DEV = torch.device("cuda:0")


def max_level(f):
    b, rho = 0, 1
    while rho * f.s <= 32:
        b, rho = b + 1, rho * f.s
    return b


def gather(h, b, blocks):
    st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
    sq.squeeze_block_to_compact(h.h, b, blocks, st)
    return st


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 10), (I.TRIANGLE_PAPER, 7), (I.CARPET, 5),
                                 (I.VICSEK, 5), (I.FULL2, 6)],
                         ids=["triangle10", "paper7", "carpet5", "vicsek5", "full2_6"])
def test_block_layout_start_and_steps_match_oracle(f, r):
    seed, pq = 13, I.p_q24(0.45)
    c0 = oracle.compact_init(f, r, seed, pq)
    want = {t: oracle.run_compact(f, r, c0, t) for t in (1, 2, 5)}
    with sq.Handle(f, r) as h:
        for b in range(0, min(max_level(f), r) + 1):
            rho = f.s ** b
            nbytes = sq.squeeze_block_bytes(h.h, b)
            assert nbytes == f.k ** (r - b) * rho * rho
            assert nbytes == oracle.state_bytes(f, r, rho=rho, cell_bytes=1)
            x = torch.full((nbytes,), 7, dtype=torch.uint8, device=DEV)
            y = torch.empty_like(x)
            sq.squeeze_block_init(h.h, b, x, seed, pq)
            assert np.array_equal(gather(h, b, x).cpu().numpy(), c0), b
            done = 0
            for t in (1, 2, 5):
                sq.squeeze_block_step(h.h, b, x, y, t - done)
                if (t - done) % 2:
                    x, y = y, x
                done = t
                assert np.array_equal(gather(h, b, x).cpu().numpy(), want[t]), (b, t)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


def test_block_layout_r16_equals_tiled():
    w = I.TRIANGLE_R16
    pq = I.p_q24(w.p)
    with sq.Handle(w.fractal, w.r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        bb = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
        sq.squeeze_step(h.h, a, bb, 10, sq.SQUEEZE_STEP_TILED)
        for b in (1, 3, 5):
            nbytes = sq.squeeze_block_bytes(h.h, b)
            x = torch.empty(nbytes, dtype=torch.uint8, device=DEV)
            y = torch.empty_like(x)
            sq.squeeze_block_init(h.h, b, x, w.seed, pq)
            sq.squeeze_block_step(h.h, b, x, y, 10)
            assert torch.equal(gather(h, b, x), a), b
            del x, y


def test_block_layout_argument_checks():
    with sq.Handle(I.TRIANGLE, 6) as h:
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_block_bytes(h.h, 7)           # above r
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
    with sq.Handle(I.TRIANGLE, 8) as h:
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_block_bytes(h.h, 6)           # rho = 64 > 32
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        x = torch.zeros(sq.squeeze_block_bytes(h.h, 2), dtype=torch.uint8, device=DEV)
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_block_step(h.h, 2, x, x, 1)   # the same buffer twice
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
