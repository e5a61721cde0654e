"""The full triangle workloads at r = 16 and r = 20, against the oracle.

r = 20, 100 steps: the tiled step, the per-cell integer-ALU step and the
per-cell tensor-core (tcgen05) step each run 100 B3/S23 steps over all
3,486,784,401 cells from the seeded Bernoulli(0.5) start; their final states
must be identical, and a seeded sample of 2^16 compact indices must match the
CPU oracle's light cone (the state of a cell after T steps depends only on
the start within Chebyshev distance T).

r = 16, 1000 steps (Bernoulli(0.3)): the tiled step equals the same-GPU
bounding-box kernel on the full state at steps 1, 10, 100 and 1000; the CPU
bounding-box oracle, run on the whole 65,536^2 box, equals the tiled step at
every step from 1 to 10; a few cells match the oracle's light cone at T = 1000.

Together about four minutes on a GB300 (the per-cell tensor-core step over
3.5e9 cells dominates) and 13 GB of host memory for the r = 16 box.
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


def test_r16_1000_steps_bb_and_cpu_box():
    w = I.TRIANGLE_R16
    f, r, pq = w.fractal, w.r, I.p_q24(w.p)
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
        # CPU oracle on the whole box, steps 1..10, against the tiled step
        member = oracle.member_grid(f, r)
        box = oracle.box_init(f, r, w.seed, pq)
        assert np.array_equal(oracle.box_to_compact(f, r, box), a.cpu().numpy())
        for t in range(1, 11):
            box = oracle.box_run(member, box, 1)
            sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)
            a, b = b, a
            assert np.array_equal(oracle.box_to_compact(f, r, box), a.cpu().numpy()), t
        del box, member
        # the same-GPU bounding box at 1, 10, 100, 1000 steps
        sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
        g0 = torch.empty(h.side * h.side, dtype=torch.uint8, device="cuda")
        g1 = torch.empty_like(g0)
        sq.squeeze_bb_init(h.h, g0, w.seed, pq)
        st = torch.empty_like(a)
        done = 0
        for t in (1, 10, 100, 1000):
            sq.squeeze_step(h.h, a, b, t - done, sq.SQUEEZE_STEP_TILED)
            sq.squeeze_bb_step(h.h, g0, g1, t - done)
            if (t - done) % 2:
                a, b = b, a
                g0, g1 = g1, g0
            done = t
            sq.squeeze_bb_to_compact(h.h, g0, st)
            assert torch.equal(a, st), t
        del g0, g1
        # light cone at T = 1000 on a few cells
        om = I.random_ints(22, 4, h.cells).astype(np.uint64)
        want = oracle.lightcone(f, r, w.seed, pq, 1000, oracle.lam(f, r, om))
        assert np.array_equal(a.cpu().numpy()[om.astype(np.int64)], want)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
