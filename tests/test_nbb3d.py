"""Three-dimensional NBB fractals on the GPU: lambda, nu, start and step, bit-exact.

The CUDA path (squeeze_3d_*) is compared with the 3-D oracle cell by cell at
levels the box oracle holds, by light-cone samples at large levels (the Menger
sponge at 6.4e7 cells, the tetrahedron at 2.7e8), and with the two-dimensional
step on the flat triangle slab, whose cells are those of the planar
triangle.
"""
import numpy as np
import pytest

import oracle
from oracle import nbb3d as O3
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402

DEV = torch.device("cuda:0")
MAX = np.uint64(2 ** 64 - 1)

SMALL = [(I.MENGER, 2), (I.MENGER, 3), (I.TETRA, 5), (I.TETRA, 7), (I.CANTOR_DUST, 3),
         (I.FULL_CUBE, 4), (I.FLAT_TRIANGLE, 6), (I.SINGLE3, 0), (I.SINGLE3, 4)]
FORWARD = sum(1 << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1) for dx, dy, dz in
              [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 1), (0, -1, -1), (1, 1, 1)])
RULES = [(O3.LIFE_4555, O3.MOORE3),
         (((1 << 6), (1 << 5) | (1 << 6) | (1 << 7)), O3.MOORE3),
         (((1 << 1) | (1 << 2), (1 << 1) | (1 << 3)), O3.VON_NEUMANN3),
         (((1 << 1) | (1 << 2), (1 << 1) | (1 << 3)), FORWARD)]


def ids(v):
    return getattr(v, "name", str(v))


def lam_gpu(h, om):
    d = torch.from_numpy(np.ascontiguousarray(om, dtype=np.uint64).view(np.int64)).to(DEV)
    xyz = torch.full((len(om), 3), 7, dtype=torch.int32, device=DEV)
    sq.squeeze_3d_lambda(h.h, d, xyz, len(om))
    return xyz.cpu().numpy().astype(np.int64)


def nu_gpu(h, pts):
    d = torch.from_numpy(np.ascontiguousarray(pts, dtype=np.int32)).to(DEV)
    o = torch.full((len(pts),), 7, dtype=torch.int64, device=DEV)
    sq.squeeze_3d_nu(h.h, d, o, len(pts))
    return o.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("f,r", SMALL, ids=ids)
def test_3d_maps_every_cell_and_box_point(f, r):
    with sq.Handle3(f, r) as h:
        assert (h.wx, h.wy, h.wz) == O3.extents(f, r) and h.cells == f.k ** r
        om = np.arange(f.k ** r + 3, dtype=np.uint64)       # 3 past the end
        assert np.array_equal(lam_gpu(h, om), O3.lam(f, r, om))
        n = f.s ** r
        z, y, x = np.mgrid[-1:n + 1, -1:n + 1, -1:n + 1]
        pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
        assert np.array_equal(nu_gpu(h, pts), O3.nu(f, r, pts))
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK


@pytest.mark.parametrize("f,r", [(I.MENGER, 7), (I.TETRA, 15), (I.CANTOR_DUST, 10),
                                 (I.FULL_CUBE, 12), (I.FLAT_TRIANGLE, 20)], ids=ids)
def test_3d_maps_sampled_at_large_levels(f, r):
    with sq.Handle3(f, r) as h:
        cells = f.k ** r
        om = np.concatenate([I.random_ints(31, 8192, cells).astype(np.uint64),
                             np.array([0, 1, cells - 1, cells, 2 ** 63], dtype=np.uint64)])
        xyz = lam_gpu(h, om)
        assert np.array_equal(xyz, O3.lam(f, r, om))
        good = xyz[:, 0] >= 0
        assert np.array_equal(nu_gpu(h, xyz[good]), om[good])
        moved = xyz[good] + [1, -1, 1]
        assert np.array_equal(nu_gpu(h, moved), O3.nu(f, r, moved))


def test_3d_start_matches_the_oracle():
    f, r = I.MENGER, 4
    with sq.Handle3(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        sq.squeeze_3d_init_bernoulli(h.h, a, 12, I.p_q24(0.3))
        assert np.array_equal(a.cpu().numpy(), O3.init_compact(f, r, 12, I.p_q24(0.3)))


@pytest.mark.parametrize("f,r", [(I.MENGER, 3), (I.TETRA, 6), (I.CANTOR_DUST, 3),
                                 (I.FULL_CUBE, 4), (I.FLAT_TRIANGLE, 6), (I.SINGLE3, 0),
                                 (I.SINGLE3, 3), (I.TETRA, 1)], ids=ids)
@pytest.mark.parametrize("case", range(len(RULES)), ids=["4555", "5766", "vonneumann", "forward"])
def test_3d_step_equals_the_oracle(f, r, case):
    rule, mask = RULES[case]
    c0 = O3.init_compact(f, r, 40 + r, I.p_q24(0.4))
    steps = 3 + (case % 2)                    # odd and even counts: both result buffers
    with sq.Handle3(f, r) as h:
        sq.squeeze_3d_set_rule(h.h, *rule)
        sq.squeeze_3d_set_neighbourhood(h.h, mask)
        a = torch.from_numpy(c0).to(DEV)
        b = torch.empty_like(a)
        sq.squeeze_3d_step(h.h, a, b, steps)
        got = (b if steps % 2 else a).cpu().numpy()
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
    assert np.array_equal(got, O3.run_compact(f, r, c0, steps, rule, mask))


@pytest.mark.parametrize("f,r", [(I.MENGER, 6), (I.TETRA, 14)], ids=ids)
def test_3d_step_at_large_levels_against_light_cones(f, r):
    seed, p, steps = 8, I.p_q24(0.35), 2
    with sq.Handle3(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        b = torch.empty_like(a)
        sq.squeeze_3d_init_bernoulli(h.h, a, seed, p)
        sq.squeeze_3d_step(h.h, a, b, steps)
        om = np.concatenate([I.random_ints(5, 2048, h.cells).astype(np.uint64),
                             np.array([0, h.cells - 1], dtype=np.uint64)])
        got = a[torch.from_numpy(om.astype(np.int64)).to(DEV)].cpu().numpy()
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
    want = O3.lightcone(f, r, seed, p, steps, O3.lam(f, r, om))
    assert np.array_equal(got, want)


@pytest.mark.parametrize("r", [8, 13])
def test_flat_triangle_slab_equals_the_planar_step(r):
    """The slab's cells are the planar triangle's; B3/S23 over the 26 neighbours
    of a slab cell counts exactly its 8 planar ones."""
    steps = 6
    with sq.Handle3(I.FLAT_TRIANGLE, r) as h3, sq.Handle(I.TRIANGLE, r) as h2:
        sq.squeeze_3d_set_rule(h3.h, 1 << 3, (1 << 2) | (1 << 3))
        a3 = torch.empty(h3.cells, dtype=torch.uint8, device=DEV)
        sq.squeeze_3d_init_bernoulli(h3.h, a3, 21, I.p_q24(0.5))
        # the same start in the planar compact order: omega_2d = nu_2d(x, y) of each slab cell
        xyz = lam_gpu(h3, np.arange(h3.cells, dtype=np.uint64))
        assert not xyz[:, 2].any()
        perm = oracle.nu(I.TRIANGLE, r, xyz[:, :2]).astype(np.int64)
        a2 = torch.empty(h2.cells, dtype=torch.uint8, device=DEV)
        a2[torch.from_numpy(perm).to(DEV)] = a3
        b3, b2 = torch.empty_like(a3), torch.empty_like(a2)
        sq.squeeze_3d_step(h3.h, a3, b3, steps)
        sq.squeeze_step(h2.h, a2, b2, steps, sq.SQUEEZE_STEP_AUTO)
        assert torch.equal(a2[torch.from_numpy(perm).to(DEV)], a3)
        assert sq.squeeze_3d_device_status(h3.h) == sq.SQUEEZE_OK


def test_3d_argument_checks():
    with sq.Handle3(I.TETRA, 3) as h:
        d = torch.zeros(64, dtype=torch.uint8, device=DEV)
        bad = [lambda: sq.squeeze_3d_set_rule(h.h, 1 << 27, 0),
               lambda: sq.squeeze_3d_set_neighbourhood(h.h, 1 << 13),
               lambda: sq.squeeze_3d_set_neighbourhood(h.h, 1 << 27),
               lambda: sq.squeeze_3d_step(h.h, d, d, 1),
               lambda: sq.squeeze_3d_lambda(h.h, d[1:], d, 1),
               lambda: sq.squeeze_3d_init_bernoulli(h.h, d, 0, (1 << 24) + 1)]
        for call in bad:
            with pytest.raises(sq.SqueezeError) as e:
                call()
            assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_3d_lambda(h.h, d, d, 0)       # zero points: nothing enqueued
        sq.squeeze_3d_step(h.h, d, d[32:], 0)    # zero steps
        assert sq.squeeze_3d_device_status(h.h) == sq.SQUEEZE_OK
