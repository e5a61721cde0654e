"""Other neighbourhoods and the heat equation on compact fractals (Sec. 1).

Every step kernel counts over the handle's neighbourhood mask; each is
compared with the CPU oracle's masked box automaton.  The fp32 heat step is
compared with the oracle's fp64 heat equation within the bound derived from
the arithmetic: each step adds at most (2 * neighbours + 2) roundings of
size 2^-24 * max|u| to values that stay in [min u, max u] (the update is a
convex combination for alpha * neighbours <= 1, so earlier errors are not
amplified); over T steps |error| <= T * 10 * 2^-24 * max|u| < 1e-6 * T * max|u|.
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
DIAGONALS = (1 << 0) | (1 << 2) | (1 << 6) | (1 << 8)
MASKS = [sq.SQUEEZE_VON_NEUMANN, DIAGONALS, (1 << 1) | (1 << 5)]
CASES = [(I.TRIANGLE, 8), (I.CARPET, 5), (I.VICSEK, 5), (I.FULL2, 6), (I.TRIANGLE_PAPER, 7)]
KINDS = [sq.SQUEEZE_STEP_TILED, sq.SQUEEZE_MAP_ALU, sq.SQUEEZE_MAP_TC_BF16]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("mask", MASKS, ids=["von_neumann", "diagonals", "east_north"])
@pytest.mark.parametrize("f,r", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_compact_kernels_over_a_neighbourhood(f, r, mask):
    rule = ((1 << 1) | (1 << 2), (1 << 1) | (1 << 3))   # B12/S13
    c0 = I.bernoulli_bytes(17, f.k ** r, 0.4)
    m = oracle.member_grid(f, r)
    want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(m, oracle.compact_to_box(f, r, c0), 3,
                                                           rule, mask))
    with sq.Handle(f, r) as h:
        sq.squeeze_set_rule(h.h, *rule)
        sq.squeeze_set_neighbourhood(h.h, mask)
        for kind in KINDS:
            a = to_dev(c0)
            b = torch.empty_like(a)
            sq.squeeze_step(h.h, a, b, 3, kind)
            assert np.array_equal(b.cpu().numpy(), want), kind
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 7), (I.CARPET, 4), (I.VICSEK, 4)],
                         ids=["triangle", "carpet", "vicsek"])
def test_box_lambda_and_block_kernels_over_von_neumann(f, r):
    seed, pq = 19, I.p_q24(0.5)
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, seed, pq)
    want = oracle.box_run_nbhd(m, box, 4, oracle.B3S23, oracle.VON_NEUMANN)
    want_c = oracle.box_to_compact(f, r, want)
    with sq.Handle(f, r) as h:
        sq.squeeze_set_neighbourhood(h.h, sq.SQUEEZE_VON_NEUMANN)
        n = h.side
        g0 = torch.empty(n * n, dtype=torch.uint8, device=DEV)
        sq.squeeze_bb_init(h.h, g0, seed, pq)
        g1 = g0.clone()
        l0, l1 = g0.clone(), g0.clone()
        sq.squeeze_bb_step(h.h, g0, g1, 4)
        assert np.array_equal(g0.cpu().numpy().reshape(n, n) & 1, want)
        sq.squeeze_lambda_step(h.h, l0, l1, 4)
        assert np.array_equal(l0.cpu().numpy().reshape(n, n) & 1, want)
        st = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
        for b in range(0, 3):
            x = torch.empty(sq.squeeze_block_bytes(h.h, b), dtype=torch.uint8, device=DEV)
            y = torch.empty_like(x)
            sq.squeeze_block_init(h.h, b, x, seed, pq)
            sq.squeeze_block_step(h.h, b, x, y, 4)
            sq.squeeze_block_to_compact(h.h, b, x, st)
            assert np.array_equal(st.cpu().numpy(), want_c), b


def test_batch_mixes_neighbourhoods():
    mix = [I.Instance(I.TRIANGLE, 9, 1), I.Instance(I.CARPET, 5, 2), I.Instance(I.VICSEK, 6, 3)]
    handles = [sq.Handle(m.fractal, m.r) for m in mix]
    try:
        sq.squeeze_set_neighbourhood(handles[0].h, sq.SQUEEZE_VON_NEUMANN)
        sq.squeeze_set_neighbourhood(handles[2].h, DIAGONALS)
        bufs = []
        for m, h in zip(mix, handles):
            a = torch.empty(h.cells, dtype=torch.uint8, device=DEV)
            sq.squeeze_init_bernoulli(h.h, a, m.seed, I.p_q24(0.5))
            bufs.append((a, torch.empty_like(a), a.clone()))
        batch = sq.squeeze_batch_create([(h.h, a, b) for h, (a, b, _) in zip(handles, bufs)])
        sq.squeeze_batch_run(batch, 5)
        torch.cuda.synchronize()
        for h, (a, b, start) in zip(handles, bufs):
            y = torch.empty_like(start)
            sq.squeeze_step(h.h, start, y, 5, sq.SQUEEZE_STEP_TILED)
            assert torch.equal(b, y)
        sq.squeeze_batch_destroy(batch)
    finally:
        for h in handles:
            h.close()


def test_neighbourhood_argument_checks():
    with sq.Handle(I.TRIANGLE, 5) as h:
        for bad in (1 << 4, 1 << 9, sq.SQUEEZE_MOORE | (1 << 4)):
            with pytest.raises(sq.SqueezeError) as e:
                sq.squeeze_set_neighbourhood(h.h, bad)
            assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        sq.squeeze_set_neighbourhood(h.h, 0)   # no neighbours: every count is 0


def compact_from_box(f, r, box):
    xy = oracle.lam(f, r, np.arange(f.k ** r, dtype=np.uint64))
    return box[xy[:, 1], xy[:, 0]]


@pytest.mark.parametrize("f,r,mask,alpha", [(I.TRIANGLE, 9, sq.SQUEEZE_VON_NEUMANN, 0.25),
                                            (I.CARPET, 5, sq.SQUEEZE_VON_NEUMANN, 0.2),
                                            (I.VICSEK, 5, sq.SQUEEZE_MOORE, 0.1),
                                            (I.FULL2, 7, sq.SQUEEZE_VON_NEUMANN, 0.25)],
                         ids=["triangle", "carpet", "vicsek_moore", "full2"])
def test_heat_matches_the_fp64_oracle(f, r, mask, alpha):
    steps = 30
    rng = np.random.default_rng(23)
    u0 = rng.random(f.k ** r).astype(np.float32)
    m = oracle.member_grid(f, r)
    box = np.zeros(m.shape, dtype=np.float64)
    xy = oracle.lam(f, r, np.arange(f.k ** r, dtype=np.uint64))
    box[xy[:, 1], xy[:, 0]] = u0
    want = compact_from_box(f, r, oracle.heat_run(m, box, steps, alpha, mask))
    with sq.Handle(f, r) as h:
        sq.squeeze_set_neighbourhood(h.h, mask)
        a = to_dev(u0)
        b = torch.empty_like(a)
        sq.squeeze_heat_step(h.h, a, b, steps, alpha)
        got = a.cpu().numpy().astype(np.float64)   # steps is even
    bound = 1e-6 * steps * float(np.abs(u0).max())
    assert np.abs(got - want).max() <= bound
    assert abs(got.sum() - u0.astype(np.float64).sum()) <= bound * u0.size


def test_heat_constant_field_and_checks():
    with sq.Handle(I.TRIANGLE, 10) as h:
        a = torch.full((h.cells,), 0.75, dtype=torch.float32, device=DEV)
        b = torch.empty_like(a)
        sq.squeeze_heat_step(h.h, a, b, 7, 0.2)
        assert torch.equal(b, torch.full_like(b, 0.75))
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_heat_step(h.h, a, a, 1, 0.2)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG


@pytest.mark.parametrize("temperature", [0.0, 1.5, 2.269, 5.0, 1e300],
                         ids=["T0", "T1.5", "Tc", "T5", "Tinf"])
@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 8), (I.CARPET, 4), (I.VICSEK, 5), (I.FULL2, 6)],
                         ids=["triangle", "carpet", "vicsek", "full2"])
def test_ising_sweeps_match_the_oracle(f, r, temperature):
    """Metropolis decisions are integers (24-bit thresholds from the same double
    formula on both sides), so every spin must agree."""
    seed = 1234
    m = oracle.member_grid(f, r)
    box = oracle.box_init(f, r, 21, I.p_q24(0.5))
    want = oracle.box_to_compact(f, r, oracle.ising_run(m, box, 4, seed, temperature))
    with sq.Handle(f, r) as h:
        sq.squeeze_set_neighbourhood(h.h, sq.SQUEEZE_VON_NEUMANN)
        st = to_dev(oracle.box_to_compact(f, r, box))
        sq.squeeze_ising_sweep(h.h, st, 4, seed, temperature)
        assert np.array_equal(st.cpu().numpy(), want)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK


def test_ising_checks():
    with sq.Handle(I.TRIANGLE, 6) as h:
        st = torch.zeros(h.cells, dtype=torch.uint8, device=DEV)
        with pytest.raises(sq.SqueezeError) as e:   # Moore joins cells of equal parity
            sq.squeeze_ising_sweep(h.h, st, 1, 1, 2.0)
        assert e.value.code == sq.SQUEEZE_ERR_UNSUPPORTED
        sq.squeeze_set_neighbourhood(h.h, sq.SQUEEZE_VON_NEUMANN)
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_ising_sweep(h.h, st, 1, 1, -1.0)
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
