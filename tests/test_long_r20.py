"""Sierpinski triangle r = 20, 100 steps: the full workload, three kernels, the oracle.

The tiled step, the per-cell integer-ALU step and the per-cell tensor-core
(tcgen05) step each run 100 B3/S23 steps over all 3,486,784,401 cells from the
seeded Bernoulli(0.5) start; their final states must be identical, and a
seeded sample of 2^16 compact indices must match the CPU oracle's light cone
(the state of a cell after T steps depends only on the start within
Chebyshev distance T).  About eight minutes (most of it the two per-cell
kernels and the oracle's 2^16 light cones), so it runs only when
SQUEEZE_LONG=1 is set.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("SQUEEZE_LONG") != "1",
                                 reason="long run: set SQUEEZE_LONG=1")]

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402


def test_r20_100_steps_three_kernels_and_light_cone():
    w = I.TRIANGLE_R20
    with sq.Handle(w.fractal, w.r) as h:
        start = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        sq.squeeze_init_bernoulli(h.h, start, w.seed, I.p_q24(w.p))
        a = start.clone()
        b = torch.empty_like(a)
        sq.squeeze_step(h.h, a, b, w.n_steps, sq.SQUEEZE_STEP_TILED)
        ref = a if w.n_steps % 2 == 0 else b
        for kind in (sq.SQUEEZE_MAP_ALU, sq.SQUEEZE_MAP_TC_BF16):
            x = start.clone()
            y = torch.empty_like(x)
            sq.squeeze_step(h.h, x, y, w.n_steps, kind)
            got = x if w.n_steps % 2 == 0 else y
            assert torch.equal(got, ref), kind
            del x, y, got
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
        om = I.random_ints(I.R20_SAMPLE_SEED, 1 << 16, h.cells).astype(np.uint64)
        sample = ref[torch.from_numpy(om.astype(np.int64)).cuda()].cpu().numpy()
        xy = oracle.lam(w.fractal, w.r, om)
        want = oracle.lightcone(w.fractal, w.r, w.seed, I.p_q24(w.p), w.n_steps, xy)
        assert np.array_equal(sample, want)
