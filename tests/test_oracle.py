"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each check compares the oracle with a closed form, an independent construction
(Kronecker powers, Lucas's theorem, a library convolution), brute force on tiny
levels, or a value printed in / worked by hand from the paper.  Together they
are chosen so that a dropped level, a swapped axis, an off-by-one digit or a
wrong rule bit in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy.signal import convolve2d

import oracle
from conftest import read_golden
from paper_2201_00613_gb300 import inputs as I

ALL = [I.TRIANGLE, I.TRIANGLE_PAPER, I.CARPET, I.VICSEK, I.FULL2, I.SINGLE]


def _popcount(v):
    return bin(v).count("1")


# --------------------------------------------------------------------------
# Membership: closed forms and independent constructions.

@pytest.mark.parametrize("r", range(0, 11))
def test_triangle_membership_closed_form(r):
    m = oracle.member_grid(I.TRIANGLE, r)
    n = 2 ** r
    y, x = np.mgrid[0:n, 0:n]
    assert np.array_equal(m, ((x & y) == 0).astype(np.uint8))
    assert int(m.sum()) == 3 ** r
    rows = m.sum(axis=1)
    for yy in range(n):
        assert rows[yy] == 2 ** (r - _popcount(yy))


@pytest.mark.parametrize("r", range(0, 7))
def test_triangle_is_pascal_mod_2(r):
    # Lucas: C(x+y, x) is odd iff x & y == 0.
    m = oracle.member_grid(I.TRIANGLE, r)
    n = 2 ** r
    for y in range(n):
        for x in range(n):
            assert m[y, x] == (math.comb(x + y, x) % 2)


@pytest.mark.parametrize("r", range(0, 9))
def test_paper_orientation_triangle(r):
    m = oracle.member_grid(I.TRIANGLE_PAPER, r)
    n = 2 ** r
    y, x = np.mgrid[0:n, 0:n]
    assert np.array_equal(m, ((x & ~y) == 0).astype(np.uint8))


def _kron_power(f, r):
    base = np.zeros((f.s, f.s), dtype=np.uint8)
    for tx, ty in f.offsets:
        base[ty, tx] = 1
    g = np.ones((1, 1), dtype=np.uint8)
    for _ in range(r):
        g = np.kron(g, base)
    return g


@pytest.mark.parametrize("f", [I.TRIANGLE, I.TRIANGLE_PAPER, I.CARPET, I.VICSEK, I.FULL2, I.SINGLE],
                         ids=lambda f: f.name)
@pytest.mark.parametrize("r", range(0, 6))
def test_membership_equals_kronecker_power(f, r):
    if f.s ** r > 729:
        pytest.skip("box too large for this check")
    m = oracle.member_grid(f, r)
    assert np.array_equal(m, _kron_power(f, r))
    assert int(m.sum()) == f.k ** r


def test_carpet_and_vicsek_digit_rules():
    r = 4
    n = 3 ** r
    mc = oracle.member_grid(I.CARPET, r)
    mv = oracle.member_grid(I.VICSEK, r)
    for y in range(n):
        for x in range(n):
            dx = [(x // 3 ** j) % 3 for j in range(r)]
            dy = [(y // 3 ** j) % 3 for j in range(r)]
            carpet = all(not (a == 1 and b == 1) for a, b in zip(dx, dy))
            vicsek = all(a == 1 or b == 1 for a, b in zip(dx, dy))
            assert mc[y, x] == carpet
            assert mv[y, x] == vicsek


def test_memory_table_and_mrf():
    """Compact sizes reproduce the paper's Table 'memory' and the 315x figure."""
    g = read_golden("memory_table_r16.txt")
    gib = float(2 ** 30)
    for rho, bb_gb, sq_gb, mrf in g["row"]:
        rho = int(rho)
        sq = oracle.state_bytes(I.TRIANGLE, 16, rho, cell_bytes=4)
        bb = oracle.box_bytes(I.TRIANGLE, 16, cell_bytes=4)
        assert round(bb / gib) == int(bb_gb)
        # printed to two decimals, rounded in some rows and truncated in others
        assert abs(sq / gib - float(sq_gb)) < 0.01
        assert abs(bb / sq - float(mrf)) < 0.06
    mrf20 = oracle.box_bytes(I.TRIANGLE, 20) / oracle.state_bytes(I.TRIANGLE, 20)
    assert round(mrf20) == int(g["r20_mrf"][0][0])
    assert round(oracle.box_bytes(I.TRIANGLE, 20, 4) / gib) == int(g["r20_bb_gb"][0][0])


@pytest.mark.parametrize("r", range(0, 9))
def test_compact_shape(r):
    for f in ALL:
        h, w = oracle.compact_shape(f, r)
        assert h * w == f.k ** r
        assert w == f.k ** ((r + 1) // 2)


# --------------------------------------------------------------------------
# lambda / nu: worked example and brute force.

def test_worked_lambda_nu_r3():
    g = read_golden("lambda_nu_worked_r3.txt")
    off = [int(v) for v in g["offsets"][0]]
    f = I.Fractal("t", 2, 3, tuple(zip(off[0::2], off[1::2])))
    r = int(g["r"][0][0])
    wx, wy = (int(v) for v in g["omega_xy"][0])
    ex, ey = (int(v) for v in g["expanded_xy"][0])
    h, w = oracle.compact_shape(f, r)
    assert (h, w) == (3, 9)
    xy = oracle.lam(f, r, [wy * w + wx])
    assert tuple(xy[0]) == (ex, ey)
    assert int(oracle.nu(f, r, [[ex, ey]])[0]) == wy * w + wx


def test_compact_layout_r2():
    g = read_golden("compact_layout_r2.txt")
    f = I.TRIANGLE
    xy = oracle.lam(f, 2, np.arange(9))
    for row in range(3):
        vals = [int(v) for v in g["row%d" % row][0]]
        expect = list(zip(vals[0::2], vals[1::2]))
        assert [tuple(p) for p in xy[3 * row: 3 * row + 3]] == expect


@pytest.mark.parametrize("f", ALL, ids=lambda f: f.name)
def test_lambda_nu_bijection_brute_force(f):
    for r in range(0, 9):
        if f.k ** r > 300000 or f.s ** r > 1024:
            break
        cells = f.k ** r
        n = f.s ** r
        xy = oracle.lam(f, r, np.arange(cells))
        m = oracle.member_grid(f, r)
        # lambda lands on fractal cells, injectively, and covers the fractal.
        assert np.all(m[xy[:, 1], xy[:, 0]] == 1)
        flat = xy[:, 1] * n + xy[:, 0]
        assert np.unique(flat).size == cells
        assert int(m.sum()) == cells
        # nu(lambda(w)) = w
        assert np.array_equal(oracle.nu(f, r, xy), np.arange(cells, dtype=np.uint64))
        # lambda(nu(p)) = p on the fractal; nu(hole) = sentinel.
        yy, xx = np.mgrid[0:n, 0:n]
        pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
        om = oracle.nu(f, r, pts)
        hole = m.ravel() == 0
        assert np.all(om[hole] == np.uint64(2 ** 64 - 1))
        back = oracle.lam(f, r, om[~hole])
        assert np.array_equal(back, pts[~hole])


def test_nu_outside_box_and_lambda_out_of_range():
    f = I.TRIANGLE
    r = 5
    n = 32
    pts = [[-1, 0], [0, -1], [n, 0], [0, n], [-1, -1], [n, n]]
    assert np.all(oracle.nu(f, r, pts) == np.uint64(2 ** 64 - 1))
    xy = oracle.lam(f, r, [3 ** r, 3 ** r + 7])
    assert np.all(xy == -1)


def test_replica_order_invariance():
    """Permuting the replica ids changes the compact order, not the fractal."""
    rng = np.random.default_rng(0)
    f = I.CARPET
    perm = rng.permutation(f.k)
    g = I.Fractal("carpet_perm", f.s, f.k, tuple(f.offsets[i] for i in perm))
    r = 3
    c = I.bernoulli_bytes(7, f.k ** r)
    box_f = oracle.compact_to_box(f, r, c)
    m = oracle.member_grid(f, r)
    assert np.array_equal(m, oracle.member_grid(g, r))
    out_f = oracle.box_run(m, box_f, 5)
    c_g = oracle.box_to_compact(g, r, box_f)
    out_g = oracle.run_compact(g, r, c_g, 5)
    assert np.array_equal(oracle.box_to_compact(g, r, out_f), out_g)


# --------------------------------------------------------------------------
# The automaton: textbook Life, hand-worked steps, degenerate cases.

def _textbook_life(grid, steps):
    k = np.ones((3, 3), dtype=np.int32)
    k[1, 1] = 0
    g = grid.astype(np.int32)
    for _ in range(steps):
        c = convolve2d(g, k, mode="same", boundary="fill", fillvalue=0)
        g = ((c == 3) | ((g == 1) & (c == 2))).astype(np.int32)
    return g.astype(np.uint8)


@pytest.mark.parametrize("steps", [1, 2, 7])
def test_full_box_equals_textbook_life(steps):
    f = I.FULL2
    r = 5
    m = oracle.member_grid(f, r)
    assert m.all()
    box = I.bernoulli_bytes(11 + steps, 32 * 32, 0.4).reshape(32, 32)
    assert np.array_equal(oracle.box_run(m, box, steps), _textbook_life(box, steps))


def test_full_box_patterns():
    f = I.FULL2
    r = 4
    m = oracle.member_grid(f, r)
    block = np.zeros((16, 16), np.uint8)
    block[5:7, 5:7] = 1
    assert np.array_equal(oracle.box_run(m, block, 3), block)
    blinker = np.zeros((16, 16), np.uint8)
    blinker[8, 7:10] = 1
    one = oracle.box_run(m, blinker, 1)
    assert one[7:10, 8].all() and one.sum() == 3
    assert np.array_equal(oracle.box_run(m, blinker, 2), blinker)
    glider = np.zeros((16, 16), np.uint8)
    for yy, xx in [(1, 2), (2, 3), (3, 1), (3, 2), (3, 3)]:
        glider[yy, xx] = 1
    moved = np.roll(np.roll(glider, 1, axis=0), 1, axis=1)
    assert np.array_equal(oracle.box_run(m, glider, 4), moved)


def test_hand_worked_r2_steps():
    g = read_golden("step_worked_r2.txt")
    f = I.TRIANGLE
    for case, steps in (("A", (1, 2)), ("B", (1,))):
        c0 = np.array([int(v) for v in g[case + "_step0"][0]], np.uint8)
        for t in steps:
            expect = np.array([int(v) for v in g["%s_step%d" % (case, t)][0]], np.uint8)
            assert np.array_equal(oracle.run_compact(f, 2, c0, t), expect), (case, t)


def test_single_cell_dies():
    f = I.SINGLE
    for r in range(0, 4):
        c = np.ones(1, np.uint8)
        assert oracle.run_compact(f, r, c, 1)[0] == 0


def test_rule_masks_are_used():
    # With birth on 0 neighbours an isolated dead cell is born.
    f = I.SINGLE
    c = np.zeros(1, np.uint8)
    assert oracle.run_compact(f, 3, c, 1, rule=(1, 0))[0] == 1


# --------------------------------------------------------------------------
# Initial states and the light cone.

def test_splitmix64_reference_outputs():
    g = read_golden("splitmix64_seed0.txt")
    seed = int(g["seed"][0][0])
    for i in range(3):
        assert oracle.splitmix64(seed, i) == int(g["out%d" % i][0][0], 16)


def test_bernoulli_density():
    f = I.TRIANGLE
    r = 10
    for p in (0.3, 0.5):
        c = oracle.compact_init(f, r, 1, I.p_q24(p))
        n = c.size
        sigma = math.sqrt(n * p * (1 - p))
        assert abs(int(c.sum()) - n * p) < 5 * sigma
        assert set(np.unique(c)) <= {0, 1}


def test_bernoulli_keyed_by_expanded_position():
    # The same expanded cell gets the same draw whatever the replica order.
    f = I.CARPET
    perm = tuple(f.offsets[i] for i in (3, 1, 7, 0, 2, 6, 5, 4))
    g = I.Fractal("carpet_perm", f.s, f.k, perm)
    assert np.array_equal(oracle.box_init(f, 3, 9, I.p_q24(0.5)),
                          oracle.box_init(g, 3, 9, I.p_q24(0.5)))


@pytest.mark.parametrize("f,r,T", [(I.TRIANGLE, 7, 6), (I.CARPET, 4, 5), (I.VICSEK, 4, 4)],
                         ids=["triangle", "carpet", "vicsek"])
def test_lightcone_matches_full_run(f, r, T):
    seed, pq = 3, I.p_q24(0.5)
    m = oracle.member_grid(f, r)
    full = oracle.box_run(m, oracle.box_init(f, r, seed, pq), T)
    om = I.random_ints(5, 200, f.k ** r)
    om[:3] = [0, f.k ** r - 1, f.k ** (r // 2)]
    xy = oracle.lam(f, r, om)
    got = oracle.lightcone(f, r, seed, pq, T, xy)
    assert np.array_equal(got, full[xy[:, 1], xy[:, 0]])


def test_light_cone_locality_of_box_step():
    f = I.TRIANGLE
    r = 7
    m = oracle.member_grid(f, r)
    a = oracle.box_init(f, r, 4, I.p_q24(0.5))
    ys, xs = np.nonzero(m)
    i = len(xs) // 2
    b = a.copy()
    b[ys[i], xs[i]] ^= 1
    T = 5
    da = oracle.box_run(m, a, T)
    db = oracle.box_run(m, b, T)
    yy, xx = np.nonzero(da != db)
    if yy.size:
        assert np.max(np.maximum(np.abs(yy - ys[i]), np.abs(xx - xs[i]))) <= T


def test_state_is_bit_zero_of_each_byte():
    """Reading R10: only bit 0 of a cell's byte is its state."""
    f, r = I.TRIANGLE, 6
    rng = np.random.default_rng(3)
    raw = rng.integers(0, 256, f.k ** r).astype(np.uint8)
    assert np.array_equal(oracle.run_compact(f, r, raw, 3), oracle.run_compact(f, r, raw & 1, 3))


# --------------------------------------------------------------------------
# Other neighbourhoods and the heat equation (Sec. 1: stencil simulations,
# cellular automata and PDE solvers on compact fractals)

PLUS = np.array([[0, 1, 0], [1, 0, 1], [0, 1, 0]])


def _brute_nbhd_step(member, box, birth, survive, offsets):
    n = member.shape[0]
    out = np.zeros_like(box)
    for y in range(n):
        for x in range(n):
            if not member[y, x]:
                continue
            c = 0
            for dx, dy in offsets:
                qx, qy = x + dx, y + dy
                if 0 <= qx < n and 0 <= qy < n and member[qy, qx] and box[qy, qx] & 1:
                    c += 1
            out[y, x] = ((survive if box[y, x] & 1 else birth) >> c) & 1
    return out


def test_moore_mask_equals_the_life_oracle():
    f, r = I.TRIANGLE, 6
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, 4, I.p_q24(0.5))
    assert np.array_equal(oracle.box_run_nbhd(m, box, 5, nbhd=oracle.MOORE), oracle.box_run(m, box, 5))


@pytest.mark.parametrize("rule", [oracle.B3S23, ((1 << 1) | (1 << 3), (1 << 1) | (1 << 2))],
                         ids=["b3s23", "b13s12"])
def test_von_neumann_on_the_full_box_is_the_textbook_stencil(rule):
    f, r = I.FULL2, 6
    n = f.s ** r
    m = oracle.member_grid(f, r)
    assert m.all()
    box = (np.random.default_rng(3).random((n, n)) < 0.4).astype(np.uint8)
    want = box.copy()
    for _ in range(4):
        c = convolve2d(want, PLUS, mode="same", boundary="fill")
        want = np.where(want == 1, (rule[1] >> c) & 1, (rule[0] >> c) & 1).astype(np.uint8)
    assert np.array_equal(oracle.box_run_nbhd(m, box, 4, rule, oracle.VON_NEUMANN), want)


def test_von_neumann_on_the_triangle_by_brute_force():
    f, r = I.TRIANGLE, 4
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, 9, I.p_q24(0.6))
    want = box.copy()
    for _ in range(3):
        want = _brute_nbhd_step(m, want, 1 << 2, (1 << 1) | (1 << 2), [(0, -1), (-1, 0), (1, 0), (0, 1)])
    assert np.array_equal(oracle.box_run_nbhd(m, box, 3, ((1 << 2), (1 << 1) | (1 << 2)),
                                              oracle.VON_NEUMANN), want)


def test_heat_constant_field_and_conservation():
    f, r = I.TRIANGLE, 7
    m = oracle.member_grid(f, r)
    u = np.where(m == 1, 2.5, 0.0)
    assert np.array_equal(oracle.heat_run(m, u, 10, 0.2), u)
    rng = np.random.default_rng(5)
    u = np.where(m == 1, rng.random(m.shape), 0.0)
    v = oracle.heat_run(m, u, 25, 0.2)
    assert abs(v.sum() - u.sum()) <= 1e-10 * u.sum()     # the graph Laplacian conserves heat
    assert np.all(v[m == 0] == 0.0)
    assert v[m == 1].max() <= u[m == 1].max() + 1e-12   # maximum principle for alpha * 4 <= 1
    assert v[m == 1].min() >= u[m == 1].min() - 1e-12


def test_heat_on_the_full_box_is_the_five_point_stencil():
    f, r = I.FULL2, 5
    n = f.s ** r
    m = oracle.member_grid(f, r)
    u = np.random.default_rng(6).random((n, n))
    alpha = 0.15
    want = u.copy()
    for _ in range(6):
        p = np.pad(want, 1)
        deg = np.pad(np.ones((n, n)), 1)
        flow = p[:-2, 1:-1] + p[2:, 1:-1] + p[1:-1, :-2] + p[1:-1, 2:]
        d = deg[:-2, 1:-1] + deg[2:, 1:-1] + deg[1:-1, :-2] + deg[1:-1, 2:]
        want = want + alpha * (flow - d * want)
    assert np.allclose(oracle.heat_run(m, u, 6, alpha), want, rtol=0, atol=1e-12)


def test_heat_on_the_triangle_by_brute_force():
    f, r = I.TRIANGLE, 3
    n = f.s ** r
    m = oracle.member_grid(f, r)
    u = np.where(m == 1, np.arange(n * n, dtype=np.float64).reshape(n, n) % 7, 0.0)
    want = u.copy()
    for _ in range(3):
        nxt = np.zeros_like(want)
        for y in range(n):
            for x in range(n):
                if not m[y, x]:
                    continue
                flow = sum(want[y + dy, x + dx] - want[y, x]
                           for dx, dy in ((0, -1), (-1, 0), (1, 0), (0, 1))
                           if 0 <= x + dx < n and 0 <= y + dy < n and m[y + dy, x + dx])
                nxt[y, x] = want[y, x] + 0.25 * flow
        want = nxt
    assert np.allclose(oracle.heat_run(m, u, 3, 0.25), want, rtol=0, atol=1e-12)


# Ising spins (Sec. 1: spin-model simulations), checkerboard Metropolis with
# counter-based draws.

def _energy(m, box):
    s = np.where(box & 1, 1, -1) * m
    return -int((s[:, 1:] * s[:, :-1]).sum() + (s[1:, :] * s[:-1, :]).sum())


def test_ising_infinite_temperature_flips_every_spin_once_per_sweep():
    f, r = I.TRIANGLE, 6
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, 2, I.p_q24(0.5))
    got = oracle.ising_run(m, box, 1, seed=8, temperature=1e300)
    assert np.array_equal(got, np.where(m == 1, 1 - box, 0))
    assert np.array_equal(oracle.ising_run(m, box, 2, seed=8, temperature=1e300), box)


def test_ising_zero_temperature():
    f, r = I.FULL2, 5
    n = f.s ** r
    m = oracle.member_grid(f, r)
    up = np.ones((n, n), dtype=np.uint8)
    assert np.array_equal(oracle.ising_run(m, up, 3, seed=1, temperature=0.0), up)
    one_down = up.copy()
    one_down[9, 14] = 0
    assert np.array_equal(oracle.ising_run(m, one_down, 1, seed=1, temperature=0.0), up)
    box = (np.random.default_rng(4).random((n, n)) < 0.5).astype(np.uint8)
    e = [_energy(m, box)]
    for _ in range(5):
        box = oracle.ising_run(m, box, 1, seed=len(e), temperature=0.0)
        e.append(_energy(m, box))
    assert all(b <= a for a, b in zip(e, e[1:]))


def test_ising_by_brute_force_on_the_triangle():
    f, r, T, seed = I.TRIANGLE, 3, 2.0, 77
    n = f.s ** r
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, 5, I.p_q24(0.5))
    thr = [2 ** 24] + [int(np.floor(np.exp(-2.0 * e / T) * 2 ** 24)) for e in range(1, 9)]
    want = box.copy()
    for t in range(2 * 3):
        d = oracle.splitmix64(seed, t)
        for y in range(n):
            for x in range(n):
                if (x + y) % 2 != t % 2 or not m[y, x]:
                    continue
                h = sum(1 if want[y + dy, x + dx] & 1 else -1
                        for dx, dy in ((0, -1), (-1, 0), (1, 0), (0, 1))
                        if 0 <= x + dx < n and 0 <= y + dy < n and m[y + dy, x + dx])
                e2 = (1 if want[y, x] & 1 else -1) * h
                if e2 <= 0 or (oracle.splitmix64(d, (y << 32) | x) >> 40) < thr[e2]:
                    want[y, x] ^= 1
    assert np.array_equal(oracle.ising_run(m, box, 3, seed, T), want)


def test_heat_two_cell_closed_form():
    """Two diagonal cells (s = 2, k = 2, r = 1): Moore joins them, von Neumann
    does not.  Under Moore their difference shrinks by (1 - 2 alpha) per step
    and their sum stays."""
    f = I.Fractal("diagonal2", 2, 2, ((0, 0), (1, 1)))
    m = oracle.member_grid(f, 1)
    assert m.tolist() == [[1, 0], [0, 1]]
    u = np.array([[1.0, 0.0], [0.0, 0.25]])
    alpha, steps = 0.1, 7
    got = oracle.heat_run(m, u, steps, alpha, oracle.MOORE)
    diff = 0.75 * (1 - 2 * alpha) ** steps
    assert got[0, 0] == pytest.approx((1.25 + diff) / 2, abs=1e-14)
    assert got[1, 1] == pytest.approx((1.25 - diff) / 2, abs=1e-14)
    assert np.array_equal(oracle.heat_run(m, u, steps, alpha, oracle.VON_NEUMANN), u)
