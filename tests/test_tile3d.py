"""The bit-sliced 3-D tile kernel on the GPU: equal to the per-cell kernel and
to the 3-D oracle.

squeeze_3d_step runs the tile kernel wherever it applies (tile rows of 8 or 16
cells: the Sierpinski tetrahedron, Cantor dust, the full cube) and the
per-cell kernel elsewhere (the Menger sponge).  The oracle comparisons at small
levels are in test_nbb3d.py, which now exercise the tile kernel too; here the
tile kernel is compared with the per-cell kernel on whole states at large
levels, with light-cone samples of the oracle at the tetrahedron's benchmark
level, and its level choice and fall-backs are checked.
"""
import numpy as np
import pytest

from oracle import nbb3d as O3
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402

DEV = torch.device("cuda:0")
RULES = [O3.LIFE_4555, ((1 << 0) | (1 << 6), (1 << 5) | (1 << 6) | (1 << 7))]


def run(h, start, steps, level=None):
    if level is not None:
        sq.squeeze_3d_set_tiled_level(h.h, level)
    a = start.clone()
    b = torch.empty_like(a)
    sq.squeeze_3d_step(h.h, a, b, steps)
    torch.cuda.synchronize()
    assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
    return (b if steps % 2 else a).clone()


@pytest.mark.parametrize("f,r,levels", [(I.TETRA, 12, (4, 5, 6)), (I.CANTOR_DUST, 7, (2, 3)),
                                        (I.FULL_CUBE, 8, (3,))],
                         ids=["tetrahedron12", "cantor_dust7", "full_cube8"])
@pytest.mark.parametrize("rule", RULES, ids=["4555", "b06s567"])
def test_tile_kernel_equals_per_cell_kernel(f, r, levels, rule):
    with sq.Handle3(f, r) as h:
        sq.squeeze_3d_set_rule(h.h, *rule)
        start = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        sq.squeeze_3d_init_bernoulli(h.h, start, 9 + r, I.p_q24(0.3))
        want = run(h, start, 3, level=0)
        for L in levels:
            assert torch.equal(run(h, start, 3, level=L), want), L
            assert sq.squeeze_3d_tiled_level(h.h) == L


def test_tile_kernel_at_the_benchmark_level_against_light_cones():
    f, r, seed, p, steps = I.TETRA, 15, 8, I.p_q24(0.35), 2
    with sq.Handle3(f, r) as h:
        assert sq.squeeze_3d_tiled_level(h.h) == 5
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        b = torch.empty_like(a)
        sq.squeeze_3d_init_bernoulli(h.h, a, seed, p)
        sq.squeeze_3d_step(h.h, a, b, steps)
        om = np.concatenate([I.random_ints(6, 2048, h.cells).astype(np.uint64),
                             np.array([0, h.cells - 1], dtype=np.uint64)])
        got = a[torch.from_numpy(om.astype(np.int64)).to(DEV)].cpu().numpy()
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
    want = O3.lightcone(f, r, seed, p, steps, O3.lam(f, r, om))
    assert np.array_equal(got, want)


def test_level_choice_and_fall_backs():
    with sq.Handle3(I.MENGER, 4) as h:          # rows of 20 cells: per-cell kernel
        assert sq.squeeze_3d_tiled_level(h.h) == 0
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_3d_set_tiled_level(h.h, 2)
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
    with sq.Handle3(I.TETRA, 8) as h:
        assert sq.squeeze_3d_tiled_level(h.h) == 5
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_3d_set_tiled_level(h.h, 9)    # above r
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_3d_set_tiled_level(h.h, 3)    # rows of 4 cells
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        # misaligned buffers take the per-cell kernel, with the same result
        c0 = O3.init_compact(I.TETRA, 8, 4, I.p_q24(0.4))
        raw_a = torch.zeros(h.cells + 16, dtype=torch.uint8, device=DEV)
        raw_b = torch.zeros(h.cells + 16, dtype=torch.uint8, device=DEV)
        a, b = raw_a[1:1 + h.cells], raw_b[1:1 + h.cells]
        a.copy_(torch.from_numpy(c0))
        sq.squeeze_3d_step(h.h, a, b, 1)
        assert np.array_equal(b.cpu().numpy(), O3.run_compact(I.TETRA, 8, c0, 1))
        # a new neighbourhood rebuilds the tile program
        sq.squeeze_3d_set_neighbourhood(h.h, O3.VON_NEUMANN3)
        x = torch.from_numpy(c0).to(DEV)
        y = torch.empty_like(x)
        sq.squeeze_3d_step(h.h, x, y, 1)
        want = O3.run_compact(I.TETRA, 8, c0, 1, O3.LIFE_4555, O3.VON_NEUMANN3)
        assert np.array_equal(y.cpu().numpy(), want)
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
