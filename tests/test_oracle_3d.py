"""Pins of the three-dimensional oracle (reading R15 of the paper's 3-D extension).

Each check compares the oracle with something other than itself: closed-form
membership of the Menger sponge, the Sierpinski tetrahedron and Cantor dust;
lambda at levels 3 and 4 written out by hand from the cycling of levels over
the compact axes; the hole-free cube against a convolution from scipy; the flat
triangle slab against the (separately pinned) two-dimensional oracle; a plain
Python step on a tiny fractal; and the light-cone sampler against the full box.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import nbb3d as O3
from paper_2201_00613_gb300 import inputs as I

FRACTALS = [I.MENGER, I.TETRA, I.CANTOR_DUST, I.FULL_CUBE, I.FLAT_TRIANGLE, I.SINGLE3]


def digits(v, s, r):
    return [(v // s ** j) % s for j in range(r)]


@pytest.mark.parametrize("f", FRACTALS, ids=lambda f: f.name)
def test_cell_count_is_k_to_the_r(f):
    for r in range(0, 4 if f.s == 3 else 5):
        assert int(O3.member_grid(f, r).sum()) == f.k ** r


def test_menger_membership_closed_form():
    # a point is in the sponge iff no base-3 position has two or more digits equal to 1
    r = 3
    n = 3 ** r
    m = O3.member_grid(I.MENGER, r)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    ok = np.ones_like(m, dtype=bool)
    for j in range(r):
        ones = sum(((c // 3 ** j) % 3 == 1).astype(int) for c in (x, y, z))
        ok &= ones <= 1
    assert np.array_equal(m.astype(bool), ok)


def test_tetrahedron_membership_closed_form():
    # no bit position holds a 1 in two of the three coordinates
    r = 5
    n = 2 ** r
    m = O3.member_grid(I.TETRA, r)
    z, y, x = np.mgrid[0:n, 0:n, 0:n]
    assert np.array_equal(m.astype(bool), ((x & y) | (y & z) | (x & z)) == 0)


def test_cantor_dust_is_a_product_of_cantor_sets():
    r = 3
    n = 3 ** r
    cantor = np.array([all(d != 1 for d in digits(v, 3, r)) for v in range(n)])
    want = cantor[:, None, None] & cantor[None, :, None] & cantor[None, None, :]
    assert np.array_equal(O3.member_grid(I.CANTOR_DUST, r).astype(bool), want)


def test_extents_follow_the_cycle_of_levels():
    for f in (I.MENGER, I.TETRA):
        for r in range(0, 9):
            wx, wy, wz = O3.extents(f, r)
            assert (wx, wy, wz) == (f.k ** -(-r // 3), f.k ** ((r + 1) // 3), f.k ** (r // 3))
            assert wx * wy * wz == f.k ** r


@pytest.mark.parametrize("f", [I.MENGER, I.TETRA, I.CANTOR_DUST], ids=lambda f: f.name)
def test_lambda_written_out_at_levels_three_and_four(f):
    tau = np.asarray(f.offsets)
    k, s = f.k, f.s
    # r = 3: one level per axis, omega = (w_z * k + w_y) * k + w_x
    om = np.arange(k ** 3)
    wx, wy, wz = om % k, (om // k) % k, om // k ** 2
    want = tau[wx] + s * tau[wy] + s * s * tau[wz]
    assert np.array_equal(O3.lam(f, 3, om), want)
    # r = 4: level 4 is the second digit of w_x; W_x = k^2, W_y = W_z = k
    om = np.arange(k ** 4)
    wx, wy, wz = om % k ** 2, (om // k ** 2) % k, om // k ** 3
    want = tau[wx % k] + s * tau[wy] + s ** 2 * tau[wz] + s ** 3 * tau[wx // k]
    assert np.array_equal(O3.lam(f, 4, om), want)
    # past the end
    assert np.array_equal(O3.lam(f, 3, [k ** 3]), [[-1, -1, -1]])


@pytest.mark.parametrize("f,r", [(I.MENGER, 2), (I.TETRA, 4), (I.CANTOR_DUST, 2),
                                 (I.FLAT_TRIANGLE, 4), (I.FULL_CUBE, 3), (I.SINGLE3, 3)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_nu_inverts_lambda_and_rejects_exactly_the_holes(f, r):
    n = f.s ** r
    om = np.arange(f.k ** r, dtype=np.uint64)
    xyz = O3.lam(f, r, om)
    assert np.array_equal(O3.nu(f, r, xyz), om)
    # every point of the box and a ring around it
    z, y, x = np.mgrid[-1:n + 1, -1:n + 1, -1:n + 1]
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    got = O3.nu(f, r, pts)
    inside = (pts >= 0).all(axis=1) & (pts < n).all(axis=1)
    m = O3.member_grid(f, r)
    is_cell = np.zeros(len(pts), dtype=bool)
    is_cell[inside] = m[pts[inside, 2], pts[inside, 1], pts[inside, 0]] == 1
    assert np.all(got[~is_cell] == np.uint64(2 ** 64 - 1))
    assert np.array_equal(np.sort(got[is_cell]), om)
    assert np.array_equal(O3.lam(f, r, got[is_cell]), pts[is_cell])


def conv_step(state, mask, rule):
    """One step on the full cube through scipy's convolution (zero outside)."""
    ndimage = pytest.importorskip("scipy.ndimage")
    kern = np.zeros((3, 3, 3), dtype=np.int32)
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        if (mask >> ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1)) & 1:
            kern[dz + 1, dy + 1, dx + 1] = 1   # symmetric masks only: orientation is moot
    c = ndimage.convolve(state.astype(np.int32), kern, mode="constant", cval=0)
    alive = state == 1
    born = (rule[0] >> c) & 1
    keep = (rule[1] >> c) & 1
    return np.where(alive, keep, born).astype(np.uint8)


@pytest.mark.parametrize("rule,mask", [(O3.LIFE_4555, O3.MOORE3),
                                       (((1 << 6), (1 << 5) | (1 << 6) | (1 << 7)), O3.MOORE3),
                                       (((1 << 1) | (1 << 3), (1 << 2) | (1 << 3)), O3.VON_NEUMANN3)],
                         ids=["4555", "5766", "vonneumann"])
def test_hole_free_cube_equals_convolution(rule, mask):
    f, r = I.FULL_CUBE, 4
    rng = np.random.default_rng(7)
    box = (rng.random((16, 16, 16)) < 0.35).astype(np.uint8)
    m = O3.member_grid(f, r)
    assert m.all()
    want = box
    for _ in range(3):
        want = conv_step(want, mask, rule)
    assert np.array_equal(O3.box_run(m, box, 3, rule, mask), want)


def test_flat_triangle_slab_equals_the_planar_oracle():
    # the 3-D Moore neighbourhood restricted to the plane z = 0 is the 2-D Moore one
    r = 6
    n = 2 ** r
    m3 = O3.member_grid(I.FLAT_TRIANGLE, r)
    m2 = oracle.member_grid(I.TRIANGLE, r)
    assert np.array_equal(m3[0], m2) and not m3[1:].any()
    box2 = oracle.box_init(I.TRIANGLE, r, 11, I.p_q24(0.45))
    box3 = np.zeros((n, n, n), dtype=np.uint8)
    box3[0] = box2
    want2 = oracle.box_run(m2, box2, 5)                   # B3/S23
    got3 = O3.box_run(m3, box3, 5, oracle.B3S23, O3.MOORE3)
    assert np.array_equal(got3[0], want2) and not got3[1:].any()


def mask_of(offsets):
    return sum(1 << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1) for dx, dy, dz in offsets)


FORWARD = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 1), (0, -1, -1)]


@pytest.mark.parametrize("offsets", [None, FORWARD], ids=["moore", "asymmetric"])
def test_tiny_step_against_plain_python(offsets):
    f, r = I.TETRA, 2
    n = 4
    if offsets is None:
        offsets = [d for d in itertools.product((-1, 0, 1), repeat=3) if d != (0, 0, 0)]
    member = lambda x, y, z: (0 <= min(x, y, z) and max(x, y, z) < n
                              and ((x & y) | (y & z) | (x & z)) == 0)
    rng = np.random.default_rng(3)
    box = np.zeros((n, n, n), dtype=np.uint8)
    for z, y, x in itertools.product(range(n), repeat=3):
        if member(x, y, z):
            box[z, y, x] = rng.random() < 0.6
    birth, survive = 1 << 2, (1 << 1) | (1 << 2)
    want = np.zeros_like(box)
    for z, y, x in itertools.product(range(n), repeat=3):
        if not member(x, y, z):
            continue
        c = sum(int(box[z + dz, y + dy, x + dx]) for dx, dy, dz in offsets
                if member(x + dx, y + dy, z + dz))
        want[z, y, x] = ((survive if box[z, y, x] else birth) >> c) & 1
    got = O3.box_run(O3.member_grid(f, r), box, 1, (birth, survive), mask_of(offsets))
    assert np.array_equal(got, want)


def test_flat_slab_with_a_one_sided_neighbourhood_equals_the_planar_oracle():
    # an asymmetric in-plane mask fixes the orientation of x and y against the 2-D oracle
    r = 5
    n = 2 ** r
    plane = [(1, 0), (1, 1), (0, -1), (-1, 1)]
    mask2 = sum(1 << ((dy + 1) * 3 + dx + 1) for dx, dy in plane)
    mask3 = mask_of([(dx, dy, 0) for dx, dy in plane] + [(0, 0, 1), (1, 0, -1)])
    rule = ((1 << 1) | (1 << 2), (1 << 1))
    box2 = oracle.box_init(I.TRIANGLE, r, 12, I.p_q24(0.5))
    box3 = np.zeros((n, n, n), dtype=np.uint8)
    box3[0] = box2
    want2 = oracle.box_run_nbhd(oracle.member_grid(I.TRIANGLE, r), box2, 4, rule, mask2)
    got3 = O3.box_run(O3.member_grid(I.FLAT_TRIANGLE, r), box3, 4, rule, mask3)
    assert np.array_equal(got3[0], want2) and not got3[1:].any()


def test_init_draws_are_keyed_by_the_compact_index():
    f, r, seed, p = I.MENGER, 3, 5, I.p_q24(0.3)
    c = O3.init_compact(f, r, seed, p)
    idx = [0, 1, 17, 4000, f.k ** r - 1]
    assert [int(c[i]) for i in idx] == [int((oracle.splitmix64(seed, i) >> 40) < p) for i in idx]
    assert abs(c.mean() - 0.3) < 0.01


@pytest.mark.parametrize("f,r,steps", [(I.MENGER, 2, 3), (I.TETRA, 4, 2), (I.FULL_CUBE, 3, 2)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_lightcone_equals_the_full_box(f, r, steps):
    seed, p = 9, I.p_q24(0.4)
    c0 = O3.init_compact(f, r, seed, p)
    want = O3.run_compact(f, r, c0, steps)
    om = np.arange(f.k ** r, dtype=np.uint64)
    got = O3.lightcone(f, r, seed, p, steps, O3.lam(f, r, om))
    assert np.array_equal(got, want)


def test_holes_are_dead_whatever_the_box_holds():
    f, r = I.MENGER, 2
    m = O3.member_grid(f, r)
    box = O3.compact_to_box(f, r, O3.init_compact(f, r, 4, I.p_q24(0.5)))
    junk = np.where(m == 1, box, 1).astype(np.uint8)     # every hole set alive
    assert np.array_equal(O3.box_run(m, junk, 2), O3.box_run(m, box, 2))
