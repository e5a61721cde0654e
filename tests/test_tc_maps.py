"""Tensor-core (tcgen05 kind::f16) lambda / nu sums and step: bit-exact.

The digit-times-weight sums run as bf16 MMAs with fp32 accumulation over
radix-256 weight limbs (Sec. 3.6).  Each result must equal the integer-ALU map
and the CPU oracle exactly: every column sum stays below 2^21 < 2^24.  The
cases include the largest digits the descriptor allows (s = 16, k = 255), so
every limb of the weights is exercised, holes, points off the box and
compact indices past the end.
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
TC = sq.SQUEEZE_MAP_TC_BF16

# s = 16 with every digit pair but (15, 15): k = 255, the largest replica id
# and the widest weights (k^r up to 255^7 ~ 2^56, seven and more limbs).
BIG = I.Fractal("s16_k255", 16, 255,
                tuple((x, y) for y in range(16) for x in range(16) if (x, y) != (15, 15)))
SMALL = [(I.TRIANGLE, 10), (I.TRIANGLE_PAPER, 9), (I.CARPET, 5), (I.VICSEK, 6), (I.FULL2, 8),
         (I.SINGLE, 3), (BIG, 2)]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def lam_both(h, om):
    """(ALU, TC) lambda of the uint64 array om."""
    d = to_dev(om.view(np.int64))
    out = []
    for tc in (False, True):
        xy = torch.full((om.size, 2), 7, dtype=torch.int32, device=DEV)
        if tc:
            sq.squeeze_map_tc(h.h, 0, d, xy, om.size, TC)
        else:
            sq.squeeze_lambda(h.h, d, xy, om.size)
        out.append(xy.cpu().numpy().astype(np.int64))
    return out


def nu_both(h, pts):
    d = to_dev(pts.astype(np.int32))
    out = []
    for tc in (False, True):
        o = torch.full((pts.shape[0],), 7, dtype=torch.int64, device=DEV)
        if tc:
            sq.squeeze_map_tc(h.h, 1, d, o, pts.shape[0], TC)
        else:
            sq.squeeze_nu(h.h, d, o, pts.shape[0])
        out.append(o.cpu().numpy().view(np.uint64))
    return out


@pytest.mark.parametrize("f,r", SMALL, ids=lambda v: getattr(v, "name", str(v)))
def test_tc_maps_every_cell_and_box_point(f, r):
    with sq.Handle(f, r) as h:
        om = np.arange(f.k ** r + 5, dtype=np.uint64)   # a ragged last tile, 5 past the end
        alu, tc = lam_both(h, om)
        assert np.array_equal(tc, alu)
        assert np.array_equal(tc, oracle.lam(f, r, om))
        n = f.s ** r
        yy, xx = np.mgrid[-1:n + 1, -1:n + 1]
        pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
        alu, tc = nu_both(h, pts)
        assert np.array_equal(tc, alu)
        assert np.array_equal(tc, oracle.nu(f, r, pts))
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 20), (I.TRIANGLE, 30), (I.CARPET, 10),
                                 (I.VICSEK, 13), (BIG, 7), (I.FULL2, 30)],
                         ids=["tri20", "tri30", "carpet10", "vicsek13", "s16k255r7", "full2r30"])
def test_tc_maps_sampled_at_large_levels(f, r):
    with sq.Handle(f, r) as h:
        cells = f.k ** r
        om = np.concatenate([I.random_ints(21, 65536, min(cells, 2 ** 62)).astype(np.uint64),
                             np.array([0, cells - 1, cells, 2 ** 64 - 1], dtype=np.uint64)])
        alu, tc = lam_both(h, om)
        assert np.array_equal(tc, alu)
        sub = slice(0, 4096)
        assert np.array_equal(tc[sub], oracle.lam(f, r, om[sub]))
        good = tc[:, 0] >= 0
        pts = np.concatenate([tc[good], tc[good] + [1, 0], tc[good] - [0, 1], tc[good] + [1, 1]])
        alu_o, tc_o = nu_both(h, pts)
        assert np.array_equal(tc_o, alu_o)
        # nu(lambda(omega)) = omega on the sample
        assert np.array_equal(tc_o[:int(good.sum())], om[good])
        assert np.array_equal(tc_o[:4096], oracle.nu(f, r, pts[:4096]))
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 7), (I.TRIANGLE, 12), (I.CARPET, 5), (I.VICSEK, 7),
                                 (I.TRIANGLE_PAPER, 9), (I.FULL2, 7), (BIG, 2)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_tc_step_equals_alu_and_oracle(f, r):
    with sq.Handle(f, r) as h:
        c0 = I.bernoulli_bytes(300 + r, f.k ** r, 0.4)
        out = {}
        for kind in (sq.SQUEEZE_MAP_ALU, TC):
            a = to_dev(c0)
            b = torch.empty_like(a)
            sq.squeeze_step(h.h, a, b, 5, kind)
            torch.cuda.synchronize()
            out[kind] = b.cpu().numpy()
        assert np.array_equal(out[TC], out[sq.SQUEEZE_MAP_ALU])
        if f.s ** r <= 4096:
            assert np.array_equal(out[TC], oracle.run_compact(f, r, c0, 5))
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


def test_tc_step_r20_two_steps_against_tiled():
    """Triangle r = 20: two TC steps equal two tiled steps everywhere."""
    f, r = I.TRIANGLE, 20
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        sq.squeeze_init_bernoulli(h.h, a, 3, I.p_q24(0.5))
        a2 = a.clone()
        b = torch.empty_like(a)
        sq.squeeze_step(h.h, a, b, 2, TC)
        sq.squeeze_step(h.h, a2, b, 2, sq.SQUEEZE_STEP_TILED)
        assert torch.equal(a, a2)
        del a2, b
        om = I.random_ints(I.R20_SAMPLE_SEED, 2048, h.cells).astype(np.uint64)
        xy = oracle.lam(f, r, om)
        want = oracle.lightcone(f, r, 3, I.p_q24(0.5), 2, xy)
        got = a[torch.from_numpy(om.astype(np.int64)).to(DEV)].cpu().numpy()
        assert np.array_equal(got, want)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


def test_tc_argument_checks():
    with sq.Handle(I.TRIANGLE, 6) as h:
        d = torch.zeros(16, dtype=torch.int64, device=DEV)
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_map_tc(h.h, 0, d, d, 4, sq.SQUEEZE_MAP_TC_I8)
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_map_tc(h.h, 2, d, d, 4, TC)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_map_tc(h.h, 0, d[1:].view(torch.uint8)[3:], d, 1, TC)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_map_tc(h.h, 1, d, d, 0, TC)   # zero points: nothing enqueued


def test_tc_step_other_rules_and_neighbourhood():
    f, r = I.TRIANGLE, 9
    c0 = I.bernoulli_bytes(31, f.k ** r, 0.5)
    with sq.Handle(f, r) as h:
        for rule, nbhd in ((((1 << 3) | (1 << 6), (1 << 2) | (1 << 3)), sq.SQUEEZE_MOORE),
                           (((1 << 1), (1 << 1) | (1 << 2)), sq.SQUEEZE_VON_NEUMANN)):
            sq.squeeze_set_rule(h.h, *rule)
            sq.squeeze_set_neighbourhood(h.h, nbhd)
            m = oracle.member_grid(f, r)
            want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(
                m, oracle.compact_to_box(f, r, c0), 4, rule, nbhd))
            a = to_dev(c0)
            b = torch.empty_like(a)
            sq.squeeze_step(h.h, a, b, 4, TC)
            assert np.array_equal(a.cpu().numpy(), want), (rule, nbhd)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
