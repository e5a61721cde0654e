"""GPU parity: every CUDA kernel against the CPU oracle, bit for bit.

All work is integer, so the tolerance is zero.  Inputs are seeded; sizes span
several tile groups and ragged tails.  Calls go through the C ABI binding.
"""
import numpy as np
import pytest

import oracle
from paper_2201_00613_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # collected on CPU, skipped there
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2201_00613_gb300 as sq  # noqa: E402

DEV = torch.device("cuda:0")
FRACTALS = [I.TRIANGLE, I.TRIANGLE_PAPER, I.CARPET, I.VICSEK, I.FULL2, I.SINGLE]
KINDS = [sq.SQUEEZE_MAP_ALU, sq.SQUEEZE_STEP_TILED]


def levels_for(f, max_cells=600000):
    out = []
    for r in range(0, 12):
        if f.k ** r > max_cells or f.s ** r > 2048:
            break
        out.append(r)
    return out


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_steps(h, state0, steps, kind):
    a = to_dev(state0)
    b = torch.empty_like(a)
    sq.squeeze_step(h.h, a, b, steps, kind)
    torch.cuda.synchronize()
    return (b if steps % 2 else a).cpu().numpy()


def assert_status_ok(h):
    assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


# --------------------------------------------------------------------------
# lambda / nu


@pytest.mark.parametrize("f", FRACTALS, ids=lambda f: f.name)
def test_lambda_nu_match_oracle_all_cells(f):
    for r in levels_for(f, 200000):
        with sq.Handle(f, r) as h:
            cells = f.k ** r
            om = np.arange(cells + 3, dtype=np.uint64)  # three indices past the end
            xy = torch.empty((om.size, 2), dtype=torch.int32, device=DEV)
            sq.squeeze_lambda(h.h, to_dev(om.view(np.int64)), xy, om.size)
            got = xy.cpu().numpy().astype(np.int64)
            want = oracle.lam(f, r, om)
            assert np.array_equal(got, want), (f.name, r)
            # nu over every point of the box plus a ring outside it
            n = f.s ** r
            yy, xx = np.mgrid[-1:n + 1, -1:n + 1]
            pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
            o = torch.empty(pts.shape[0], dtype=torch.int64, device=DEV)
            sq.squeeze_nu(h.h, to_dev(pts.astype(np.int32)), o, pts.shape[0])
            assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.nu(f, r, pts)), (f.name, r)


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 20), (I.CARPET, 10), (I.VICSEK, 13)],
                         ids=["triangle20", "carpet10", "vicsek13"])
def test_lambda_nu_sampled_at_large_levels(f, r):
    with sq.Handle(f, r) as h:
        om = I.random_ints(17, 100000, f.k ** r).astype(np.uint64)
        xy = torch.empty((om.size, 2), dtype=torch.int32, device=DEV)
        sq.squeeze_lambda(h.h, to_dev(om.view(np.int64)), xy, om.size)
        got = xy.cpu().numpy().astype(np.int64)
        assert np.array_equal(got, oracle.lam(f, r, om))
        pts = np.concatenate([got, got + [1, 0], got + [0, 1], got - [1, 1]])
        o = torch.empty(pts.shape[0], dtype=torch.int64, device=DEV)
        sq.squeeze_nu(h.h, to_dev(pts.astype(np.int32)), o, pts.shape[0])
        assert np.array_equal(o.cpu().numpy().view(np.uint64), oracle.nu(f, r, pts))


def test_round_trip_all_omega_r16_on_device():
    f, r = I.TRIANGLE, 16
    with sq.Handle(f, r) as h:
        cells = h.cells
        om = torch.arange(cells, dtype=torch.int64, device=DEV)
        xy = torch.empty((cells, 2), dtype=torch.int32, device=DEV)
        back = torch.empty(cells, dtype=torch.int64, device=DEV)
        sq.squeeze_lambda(h.h, om, xy, cells)
        sq.squeeze_nu(h.h, xy, back, cells)
        assert torch.equal(back, om)
        # the image is exactly the fractal: x & y == 0 and all points distinct
        assert int(((xy[:, 0] & xy[:, 1]) != 0).sum()) == 0
        key = xy[:, 1].to(torch.int64) * h.side + xy[:, 0].to(torch.int64)
        assert torch.unique(key).numel() == cells
        idx = torch.from_numpy(I.random_ints(3, 4096, cells)).to(DEV)
        assert np.array_equal(xy[idx].cpu().numpy().astype(np.int64),
                              oracle.lam(f, r, idx.cpu().numpy().astype(np.uint64)))


# --------------------------------------------------------------------------
# initial state


@pytest.mark.parametrize("f", [I.TRIANGLE, I.CARPET, I.VICSEK], ids=lambda f: f.name)
def test_bernoulli_init_matches_oracle(f):
    r = max(levels_for(f, 300000))
    with sq.Handle(f, r) as h:
        st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        for seed, p in ((1, 0.5), (2, 0.3)):
            sq.squeeze_init_bernoulli(h.h, st, seed, I.p_q24(p))
            assert np.array_equal(st.cpu().numpy(), oracle.compact_init(f, r, seed, I.p_q24(p)))


# --------------------------------------------------------------------------
# the step


@pytest.mark.parametrize("kind", KINDS, ids=["alu", "tiled"])
@pytest.mark.parametrize("f", FRACTALS, ids=lambda f: f.name)
def test_step_matches_oracle_every_level(f, kind):
    for r in levels_for(f, 300000):
        if r == 0 and kind == sq.SQUEEZE_STEP_TILED:
            continue
        with sq.Handle(f, r) as h:
            c0 = I.bernoulli_bytes(100 + r, f.k ** r, 0.45)
            for steps in (1, 2, 5):
                got = run_steps(h, c0, steps, kind)
                want = oracle.run_compact(f, r, c0, steps)
                assert np.array_equal(got, want), (f.name, r, steps)
            assert_status_ok(h)


@pytest.mark.parametrize("level", [1, 2, 3, 4, 5, 6])
def test_tiled_every_tile_level_triangle(level):
    f, r = I.TRIANGLE, 9
    with sq.Handle(f, r) as h:
        sq.squeeze_set_tiled_level(h.h, level)
        assert sq.squeeze_tiled_level(h.h) == level
        c0 = I.bernoulli_bytes(7, h.cells, 0.5)
        want = oracle.run_compact(f, r, c0, 3)
        assert np.array_equal(run_steps(h, c0, 3, sq.SQUEEZE_STEP_TILED), want)
        assert_status_ok(h)


@pytest.mark.parametrize("f,r,levels", [(I.CARPET, 5, [1, 2]), (I.VICSEK, 6, [1, 2, 3, 4])],
                         ids=["carpet", "vicsek"])
def test_tiled_every_tile_level_s3(f, r, levels):
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(8, h.cells, 0.5)
        want = oracle.run_compact(f, r, c0, 4)
        for level in levels:
            sq.squeeze_set_tiled_level(h.h, level)
            assert np.array_equal(run_steps(h, c0, 4, sq.SQUEEZE_STEP_TILED), want), level
        assert_status_ok(h)


# Fractals whose tile rows are 8 or 16 cells wide, where 4 or 2 tile rows share
# one slot word, or 64 cells wide, where a row takes two slot words: a
# two-replica diagonal (k = 2: widths 8 at L = 5, 6, 16 at L = 7, 8 and 64 at
# L = 11, 12), the hole-free s = 2 fractal (k = 4: width 16 at L = 3, 4, 64 at
# L = 5), the hole-free s = 4 fractal (k = 16: width 16, one row at L = 1, 16
# rows at L = 2) and the carpet at r = 8 (width 8, 8 rows at L = 2; width 64 at
# L = 3; several groups per band, so a CTA's run hands row ends on).
DIAG2 = I.Fractal("diagonal2", 2, 2, ((0, 0), (1, 1)))
FULL4 = I.Fractal("full4", 4, 16, tuple((x, y) for y in range(4) for x in range(4)))


@pytest.mark.parametrize("f,r,levels", [(DIAG2, 12, [4, 5, 6, 7, 8, 11]), (I.FULL2, 9, [2, 3, 4, 5]),
                                        (FULL4, 5, [1, 2]), (I.CARPET, 8, [1, 2, 3])],
                         ids=["diagonal2", "full2", "full4", "carpet8"])
def test_tiled_shared_slot_words(f, r, levels):
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(9, h.cells, 0.5)
        want = oracle.run_compact(f, r, c0, 3)
        for level in levels:
            sq.squeeze_set_tiled_level(h.h, level)
            assert np.array_equal(run_steps(h, c0, 3, sq.SQUEEZE_STEP_TILED), want), level
            assert np.array_equal(run_steps(h, c0, 1, sq.SQUEEZE_STEP_TILED),
                                  oracle.run_compact(f, r, c0, 1)), level
        assert_status_ok(h)
        if f is DIAG2:
            # 64 rows of 64 cells: the staging buffers alone exceed one CTA's shared memory
            with pytest.raises(sq.SqueezeError) as e:
                sq.squeeze_set_tiled_level(h.h, 12)
            assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED


@pytest.mark.parametrize("rule", [(1 << 3, (1 << 2) | (1 << 3)), (1 << 2, 0), ((1 << 3) | (1 << 6), (1 << 2) | (1 << 3)),
                                  (0b000111000, 0b111000111), (1, 1 << 8)],
                         ids=["b3s23", "seeds", "highlife", "mixed", "b0s8"])
@pytest.mark.parametrize("kind", KINDS, ids=["alu", "tiled"])
def test_other_rules(rule, kind):
    for f, r in ((I.TRIANGLE, 8), (I.CARPET, 4), (I.FULL2, 6)):
        with sq.Handle(f, r) as h:
            sq.squeeze_set_rule(h.h, *rule)
            c0 = I.bernoulli_bytes(9, h.cells, 0.4)
            want = oracle.run_compact(f, r, c0, 3, rule=rule)
            assert np.array_equal(run_steps(h, c0, 3, kind), want), f.name


def test_only_bit_zero_of_a_byte_is_read():
    f, r = I.TRIANGLE, 8
    with sq.Handle(f, r) as h:
        noisy = np.random.default_rng(1).integers(0, 256, h.cells).astype(np.uint8)
        want = oracle.run_compact(f, r, noisy & 1, 1)
        assert np.array_equal(oracle.run_compact(f, r, noisy, 1), want)
        for kind in KINDS:
            assert np.array_equal(run_steps(h, noisy, 1, kind), want)


def test_config_r10_100_steps_bit_exact():
    """Triangle r = 10, Bernoulli(0.5) seed 1, checked at steps 1, 2, 10, 100."""
    w = I.TRIANGLE_R10
    f, r = w.fractal, w.r
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, w.seed, I.p_q24(w.p))
    with sq.Handle(f, r) as h:
        st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        sq.squeeze_init_bernoulli(h.h, st, w.seed, I.p_q24(w.p))
        c0 = st.cpu().numpy()
        assert np.array_equal(c0, oracle.box_to_compact(f, r, box))
        done = 0
        for t in (1, 2, 10, 100):
            box = oracle.box_run(m, box, t - done)
            done = t
            want = oracle.box_to_compact(f, r, box)
            for kind in KINDS:
                assert np.array_equal(run_steps(h, c0, t, kind), want), (t, kind)


def test_misaligned_buffers():
    f, r = I.TRIANGLE, 8
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(3, h.cells, 0.5)
        raw_a = torch.zeros(h.cells + 16, dtype=torch.uint8, device=DEV)
        raw_b = torch.zeros(h.cells + 16, dtype=torch.uint8, device=DEV)
        a, b = raw_a[1:1 + h.cells], raw_b[1:1 + h.cells]
        a.copy_(to_dev(c0))
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_TILED)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_STEP_AUTO)  # falls back to the ALU kernel
        assert sq.squeeze_last_step_info(h.h)[0] == sq.SQUEEZE_MAP_ALU   # ... observably
        assert np.array_equal(b.cpu().numpy(), oracle.run_compact(f, r, c0, 1))
        x = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        y = torch.empty_like(x)
        x.copy_(to_dev(c0))
        sq.squeeze_step(h.h, x, y, 1, sq.SQUEEZE_STEP_AUTO)   # aligned: the tiled kernel
        assert sq.squeeze_last_step_info(h.h)[0] == sq.SQUEEZE_STEP_TILED
        assert torch.equal(y, b)


def test_tile_level_limits():
    with sq.Handle(I.TRIANGLE, 9) as h:
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_set_tiled_level(h.h, 7)  # 81-cell tile rows
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_set_tiled_level(h.h, 10)  # above r
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        assert sq.squeeze_tiled_level(h.h) == 6


def test_unsupported_and_invalid_kinds():
    with sq.Handle(I.TRIANGLE, 6) as h:
        a = torch.zeros(h.cells, dtype=torch.uint8, device=DEV)
        b = torch.zeros_like(a)
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_step(h.h, a, b, 1, sq.SQUEEZE_MAP_TC_I8)
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_step(h.h, a, b, 1, 99)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_step(h.h, a, a, 1, sq.SQUEEZE_STEP_AUTO)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_step(h.h, a, b, 0, sq.SQUEEZE_STEP_AUTO)  # zero steps is a no-op


def test_step_host_round_trip():
    f, r = I.VICSEK, 6
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(4, h.cells, 0.5)
        hin = torch.from_numpy(c0).pin_memory()
        hout = torch.empty_like(hin).pin_memory()
        d0 = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        d1 = torch.empty_like(d0)
        for steps in (1, 4):
            sq.squeeze_step_host(h.h, hin, hout, d0, d1, steps)
            assert np.array_equal(hout.numpy(), oracle.run_compact(f, r, c0, steps))


# --------------------------------------------------------------------------
# bounding-box comparator


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 9), (I.TRIANGLE, 4), (I.CARPET, 5), (I.VICSEK, 5)],
                         ids=["triangle9", "triangle4", "carpet5", "vicsek5"])
def test_bb_matches_oracle(f, r):
    seed, pq = 6, I.p_q24(0.5)
    with sq.Handle(f, r) as h:
        n = h.side
        g0 = torch.empty(n * n, dtype=torch.uint8, device=DEV)
        g1 = torch.empty_like(g0)
        sq.squeeze_bb_init(h.h, g0, seed, pq)
        box = oracle.box_init(f, r, seed, pq)
        m = oracle.member_grid(f, r)
        got0 = g0.cpu().numpy().reshape(n, n)
        assert np.array_equal(got0 & 1, box) and np.array_equal(got0 >> 1, m)
        st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        for steps in (1, 3):
            g0c = g0.clone()
            sq.squeeze_bb_step(h.h, g0c, g1, steps)
            res = g1 if steps % 2 else g0c
            want = oracle.box_run(m, box, steps)
            got = res.cpu().numpy().reshape(n, n)
            assert np.array_equal(got & 1, want) and np.array_equal(got >> 1, m)
            sq.squeeze_bb_to_compact(h.h, res, st)
            assert np.array_equal(st.cpu().numpy(), oracle.box_to_compact(f, r, want))


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 10), (I.TRIANGLE, 3), (I.CARPET, 5), (I.VICSEK, 6),
                                 (I.TRIANGLE_PAPER, 8)],
                         ids=["triangle10", "triangle3", "carpet5", "vicsek6", "paper8"])
def test_lambda_approach_matches_oracle(f, r):
    """The lambda(omega) comparator: compact threads over the expanded box."""
    seed, pq = 11, I.p_q24(0.45)
    with sq.Handle(f, r) as h:
        n = h.side
        g0 = torch.empty(n * n, dtype=torch.uint8, device=DEV)
        sq.squeeze_bb_init(h.h, g0, seed, pq)
        g1 = g0.clone()                     # holes of the second box must be 0
        box = oracle.box_init(f, r, seed, pq)
        m = oracle.member_grid(f, r)
        st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        done = 0
        for steps in (1, 2, 7):
            sq.squeeze_lambda_step(h.h, g0, g1, steps - done)
            if (steps - done) % 2:
                g0, g1 = g1, g0
            done = steps
            want = oracle.box_run(m, box, steps)
            got = g0.cpu().numpy().reshape(n, n)
            assert np.array_equal(got & 1, want) and np.array_equal(got >> 1, m), steps
            sq.squeeze_bb_to_compact(h.h, g0, st)
            assert np.array_equal(st.cpu().numpy(), oracle.box_to_compact(f, r, want)), steps
        with pytest.raises(sq.SqueezeError):
            sq.squeeze_lambda_step(h.h, g0, g0, 1)
        assert_status_ok(h)


# --------------------------------------------------------------------------
# full-size levels: cross-kernel equality plus sampled light cones


def test_r16_compact_equals_bb_and_light_cone():
    w = I.TRIANGLE_R16
    f, r, pq = w.fractal, w.r, I.p_q24(w.p)
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
        c0 = a.clone()
        g0 = torch.empty(h.side * h.side, dtype=torch.uint8, device=DEV)
        g1 = torch.empty_like(g0)
        sq.squeeze_bb_init(h.h, g0, w.seed, pq)
        st = torch.empty_like(a)
        alu_a, alu_b = c0.clone(), torch.empty_like(a)
        l0 = g0.clone()          # the lambda(omega) approach on its own pair of boxes
        l1 = g0.clone()
        done = 0
        for t in (1, 10, 100):
            sq.squeeze_step(h.h, a, b, t - done, sq.SQUEEZE_STEP_TILED)
            sq.squeeze_bb_step(h.h, g0, g1, t - done)
            sq.squeeze_step(h.h, alu_a, alu_b, t - done, sq.SQUEEZE_MAP_ALU)
            sq.squeeze_lambda_step(h.h, l0, l1, t - done)
            if (t - done) % 2:
                a, b = b, a
                g0, g1 = g1, g0
                alu_a, alu_b = alu_b, alu_a
                l0, l1 = l1, l0
            done = t
            sq.squeeze_bb_to_compact(h.h, g0, st)
            assert torch.equal(a, st), t
            assert torch.equal(a, alu_a), t
            sq.squeeze_bb_to_compact(h.h, l0, st)
            assert torch.equal(a, st), t
        del l0, l1
        # light cone at T = 100 on sampled cells
        om = I.random_ints(21, 96, h.cells).astype(np.uint64)
        xy = oracle.lam(f, r, om)
        want = oracle.lightcone(f, r, w.seed, pq, 100, xy)
        assert np.array_equal(a.cpu().numpy()[om.astype(np.int64)], want)
        assert_status_ok(h)


def test_r20_tiled_against_light_cone_and_alu():
    w = I.TRIANGLE_R20
    f, r, pq = w.fractal, w.r, I.p_q24(w.p)
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, w.seed, pq)
        c0 = a.clone()
        # full-state cross check against the per-cell ALU kernel for 2 steps
        sq.squeeze_step(h.h, a, b, 2, sq.SQUEEZE_STEP_TILED)
        a2 = a.clone()
        a.copy_(c0)
        sq.squeeze_step(h.h, a, b, 2, sq.SQUEEZE_MAP_ALU)
        assert torch.equal(a, a2)
        del a2
        # 100 steps, light cone on a seeded uniform sample of omega
        a.copy_(c0)
        del c0
        sq.squeeze_step(h.h, a, b, w.n_steps, sq.SQUEEZE_STEP_TILED)
        om = I.random_ints(I.R20_SAMPLE_SEED, 256, h.cells).astype(np.uint64)
        xy = oracle.lam(f, r, om)
        want = oracle.lightcone(f, r, w.seed, pq, w.n_steps, xy)
        got = a[torch.from_numpy(om.astype(np.int64)).to(DEV)].cpu().numpy()
        assert np.array_equal(got, want)
        assert_status_ok(h)


TWO_STEP_RULES = [(1 << 3, (1 << 2) | (1 << 3)),                    # B3/S23
                  ((1 << 3) | (1 << 6), (1 << 2) | (1 << 3)),       # HighLife
                  ((1 << 0) | (1 << 3), (1 << 2) | (1 << 3))]       # B03/S23: births at 0


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 9), (I.TRIANGLE_PAPER, 8), (I.CARPET, 5),
                                 (I.VICSEK, 6), (I.FULL2, 7), (I.TRIANGLE, 4)],
                         ids=["triangle9", "triangle_paper8", "carpet5", "vicsek6", "full2-7",
                              "triangle4"])
@pytest.mark.parametrize("steps", [4, 6, 7, 12, 16, 21])
def test_multi_step_launches_match_the_oracle(f, r, steps):
    """The tiled kernel runs eight, four or two steps in one launch (the intermediate
    steps of the tile and of its halo rings in shared memory); every rule,
    including one with births at zero neighbours (which a missing adjacent
    tile must not feed), must give the oracle's states."""
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(31 + steps, h.cells, 0.4)
        box0 = oracle.compact_to_box(f, r, c0)
        m = oracle.member_grid(f, r)
        for rule in TWO_STEP_RULES:
            sq.squeeze_set_rule(h.h, *rule)
            got = run_steps(h, c0, steps, sq.SQUEEZE_STEP_TILED)
            kind, launches, by = sq.squeeze_last_step_info(h.h)
            assert kind == sq.SQUEEZE_STEP_TILED and sum(by[1:]) >= 1
            # one more launch writes the input's border records (tiles with a halo)
            assert launches - sum(by) in (0, 1) and sum(by) % 2 == steps % 2
            assert sum(c << i for i, c in enumerate(by)) == steps
            want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(m, box0, steps, rule,
                                                                   oracle.MOORE))
            assert np.array_equal(got, want), rule
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


@pytest.mark.parametrize("steps", [1, 2, 3, 4, 5, 6, 8, 10, 16, 17, 24, 100])
def test_launch_plan_puts_the_result_in_the_right_buffer(steps):
    f, r = I.TRIANGLE, 10
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(5, h.cells, 0.5)
        got = run_steps(h, c0, steps, sq.SQUEEZE_STEP_TILED)
        _, launches, by = sq.squeeze_last_step_info(h.h)
        # + the launch that writes the input's border records, when a launch
        # of several steps reads them
        assert launches == sum(by) + (1 if sum(by[1:]) else 0) and sum(by) % 2 == steps % 2
        assert sum(c << i for i, c in enumerate(by)) == steps
        assert np.array_equal(got, oracle.run_compact(f, r, c0, steps))


def test_handles_sharing_a_kernel_with_less_shared_memory_do_not_break_each_other():
    """The eight-ring program's two-step launches need more shared memory than
    a two-ring program's launches of the same kernel: preparing the smaller
    one after the larger must not take shared memory away from the larger."""
    f, r = I.TRIANGLE, 10
    c0 = I.bernoulli_bytes(77, f.k ** r, 0.5)
    want = oracle.run_compact(f, r, c0, 10)
    with sq.Handle(f, r) as big, sq.Handle(f, r) as small:
        assert np.array_equal(run_steps(big, c0, 10, sq.SQUEEZE_STEP_TILED), want)  # 8 + 2
        sq.squeeze_set_max_steps_per_launch(small.h, 2)
        assert np.array_equal(run_steps(small, c0, 10, sq.SQUEEZE_STEP_TILED), want)
        assert np.array_equal(run_steps(big, c0, 10, sq.SQUEEZE_STEP_TILED), want)
        assert sq.squeeze_last_step_info(big.h)[2][1] == 1   # the two-step launch ran
        assert_status_ok(big)
        assert_status_ok(small)
