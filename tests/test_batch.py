"""Batched mixed-fractal steps: every instance equals its own run, bit for bit.

Instances of different NBB fractals and levels are stepped together (one
persistent launch per step, replayed from a CUDA graph).  Each result is
compared with the instance stepped alone through squeeze_step, and with the
CPU oracle (full box where it fits, light-cone samples otherwise).
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
from paper_2201_00613_gb300.batch import MixedBatch, autotune  # noqa: E402


def solo(inst, steps, level=None):
    with sq.Handle(inst.fractal, inst.r) as h:
        if level:
            sq.squeeze_set_tiled_level(h.h, level)
        a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, inst.seed, I.p_q24(inst.p))
        sq.squeeze_step(h.h, a, b, steps, sq.SQUEEZE_STEP_TILED)
        torch.cuda.synchronize()
        return (b if steps % 2 else a).clone()


def small_mix():
    mix = []
    for i, (f, r) in enumerate([(I.TRIANGLE, 8), (I.CARPET, 4), (I.VICSEK, 5), (I.TRIANGLE, 11),
                                (I.CARPET, 5), (I.VICSEK, 7), (I.TRIANGLE, 3), (I.TRIANGLE_PAPER, 9),
                                (I.TRIANGLE, 14), (I.VICSEK, 6), (I.CARPET, 3), (I.FULL2, 6)]):
        mix.append(I.Instance(f, r, 1000 + i))
    return mix


@pytest.mark.parametrize("use_graph", [True, False], ids=["graph", "direct"])
def test_small_mix_matches_solo_and_oracle(use_graph):
    mix = small_mix()
    with MixedBatch(mix, use_graph=use_graph) as mb:
        mb.run(3)
        mb.run(4)  # 7 steps in two runs (two graphs)
        torch.cuda.synchronize()
        for i, inst in enumerate(mix):
            got = mb.state(i)
            assert torch.equal(got, solo(inst, 7)), inst
            if inst.fractal.cells(inst.r) <= 200000 and inst.fractal.side(inst.r) <= 1024:
                c0 = oracle.compact_init(inst.fractal, inst.r, inst.seed, I.p_q24(inst.p))
                want = oracle.run_compact(inst.fractal, inst.r, c0, 7)
                assert np.array_equal(got.cpu().numpy(), want), inst


def test_batch_rule_mix_and_levels():
    mix = small_mix()[:6]
    handles = [sq.Handle(m.fractal, m.r) for m in mix]
    bufs = []
    try:
        for j, (m, h) in enumerate(zip(mix, handles)):
            if j % 2:
                sq.squeeze_set_rule(h.h, (1 << 3) | (1 << 6), (1 << 2) | (1 << 3))  # HighLife
            a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
            b = torch.empty_like(a)
            sq.squeeze_init_bernoulli(h.h, a, m.seed, I.p_q24(0.5))
            bufs.append((a, b))
        ref = [x[0].clone() for x in bufs]
        batch = sq.squeeze_batch_create([(h.h, a, b) for h, (a, b) in zip(handles, bufs)])
        sq.squeeze_batch_configure(batch, 192, 2, True)
        grid, threads, smem = sq.squeeze_batch_info(batch)
        assert threads == 192 and grid >= 1 and smem > 0
        sq.squeeze_batch_run(batch, 5)
        torch.cuda.synchronize()
        for (h, (a, b), r0, m) in zip(handles, bufs, ref, mix):
            x, y = r0.clone(), torch.empty_like(r0)
            sq.squeeze_step(h.h, x, y, 5, sq.SQUEEZE_STEP_TILED)
            assert torch.equal(b, y), m
        sq.squeeze_batch_destroy(batch)
    finally:
        for h in handles:
            h.close()


def test_batch_rejects_bad_items():
    with sq.Handle(I.TRIANGLE, 6) as h:
        a = torch.zeros(h.cells + 16, dtype=torch.uint8, device="cuda")
        with pytest.raises(sq.SqueezeError) as e:
            sq.squeeze_batch_create([(h.h, a, a)])
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
        with pytest.raises(sq.SqueezeError):
            sq.squeeze_batch_create([(h.h, a[1:], a[8:])])


def test_config4_mix_50_steps():
    """256 instances (triangle r 8-14, carpet r 4-8, Vicsek r 5-9), 50 steps.

    Every instance equals its solo run; instances whose bounding box has at
    most 1024^2 cells equal the full oracle run, the others light-cone samples."""
    mix = I.batch_mix(5, 256)
    steps = 50
    full = 0
    with MixedBatch(mix) as mb:
        mb.run(steps)
        torch.cuda.synchronize()
        rng = np.random.default_rng(7)
        for i, inst in enumerate(mix):
            got = mb.state(i)
            assert torch.equal(got, solo(inst, steps)), inst
            f, r = inst.fractal, inst.r
            pq = I.p_q24(inst.p)
            if f.side(r) <= 1024:
                c0 = oracle.compact_init(f, r, inst.seed, pq)
                assert np.array_equal(got.cpu().numpy(), oracle.run_compact(f, r, c0, steps)), inst
                full += 1
            else:
                om = rng.integers(0, f.cells(r), size=4).astype(np.uint64)
                want = oracle.lightcone(f, r, inst.seed, pq, steps, oracle.lam(f, r, om))
                idx = torch.from_numpy(om.astype(np.int64)).cuda()
                assert np.array_equal(got[idx].cpu().numpy(), want), inst
    assert full >= 64


def test_autotuner_picks_a_valid_shape(tmp_path, monkeypatch):
    from paper_2201_00613_gb300 import batch as B
    monkeypatch.setattr(B, "_CACHE", str(tmp_path / "autotune.json"))
    mix = small_mix()[:5]
    res = autotune(mix)
    assert res["threads"] in (0, 192, 256, 288) and res["seconds_per_step"] > 0
    again = autotune(mix)  # from the cache
    assert again["threads"] == res["threads"] and again["levels"] == res["levels"]
    with MixedBatch(mix, levels=res["levels"], threads=res["threads"],
                    ctas_per_sm=res["ctas_per_sm"]) as mb:
        mb.run(3)
        torch.cuda.synchronize()
        for i, inst in enumerate(mix):
            assert torch.equal(mb.state(i), solo(inst, 3)), inst


@pytest.mark.parametrize("steps", [1, 6, 9])
def test_items_sharing_a_handle_keep_their_own_states(steps):
    """Several items of one batch on the same handle (the request loop shares a
    handle per fractal and level): each keeps its own states and border
    records, so each must equal its own solo run."""
    shapes = [(I.CARPET, 6), (I.CARPET, 6), (I.CARPET, 6), (I.TRIANGLE, 9), (I.TRIANGLE, 9)]
    handles = {}
    bufs, items, insts = [], [], []
    try:
        for i, (f, r) in enumerate(shapes):
            h = handles.setdefault((f.name, r), sq.Handle(f, r))
            inst = I.Instance(f, r, 700 + i)
            a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
            b = torch.empty_like(a)
            sq.squeeze_init_bernoulli(h.h, a, inst.seed, I.p_q24(inst.p))
            bufs.append((a, b))
            items.append((h.h, a, b))
            insts.append(inst)
        batch = sq.squeeze_batch_create(items)
        sq.squeeze_batch_run(batch, steps)
        torch.cuda.synchronize()
        for (a, b), inst in zip(bufs, insts):
            assert torch.equal(b if steps % 2 else a, solo(inst, steps)), inst
        sq.squeeze_batch_destroy(batch)
        for h in handles.values():
            assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
    finally:
        for h in handles.values():
            h.close()


def test_runs_reuse_current_records_and_states_written_renews_them():
    """A second run of a batch reads the records its first run left (no
    records launch); after the caller rewrites a state and says so, the next
    run writes the records again: every result equals the solo run of the
    state the batch was given."""
    shapes = [(I.TRIANGLE, 10), (I.CARPET, 6), (I.VICSEK, 7)]
    handles = [sq.Handle(f, r) for f, r in shapes]
    try:
        bufs = []
        for i, h in enumerate(handles):
            a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
            bufs.append((a, torch.empty_like(a)))
            sq.squeeze_init_bernoulli(h.h, a, 40 + i, I.p_q24(0.5))
        start = [a.clone() for a, _ in bufs]
        batch = sq.squeeze_batch_create([(h.h, a, b) for h, (a, b) in zip(handles, bufs)])
        sq.squeeze_batch_run(batch, 5)
        sq.squeeze_batch_run(batch, 6)          # 11 steps, state in buffer 1
        torch.cuda.synchronize()
        for h, (a, b), s0, (f, r) in zip(handles, bufs, start, shapes):
            want = solo_from(h, s0, 11)
            assert torch.equal(b, want), f.name
        # rewrite the states (in buffer 1, where the batch keeps them now)
        for i, (h, (a, b)) in enumerate(zip(handles, bufs)):
            sq.squeeze_init_bernoulli(h.h, b, 90 + i, I.p_q24(0.4))
        fresh = [b.clone() for _, b in bufs]
        sq.squeeze_batch_states_written(batch)
        sq.squeeze_batch_run(batch, 7)          # 18 steps in all, state in buffer 0
        torch.cuda.synchronize()
        for h, (a, b), s0, (f, r) in zip(handles, bufs, fresh, shapes):
            assert torch.equal(a, solo_from(h, s0, 7)), f.name
        sq.squeeze_batch_destroy(batch)
        with pytest.raises(sq.SqueezeError):
            sq.squeeze_batch_states_written(None)
    finally:
        for h in handles:
            h.close()


def solo_from(h, state, steps):
    a = state.clone()
    b = torch.empty_like(a)
    sq.squeeze_step(h.h, a, b, steps, sq.SQUEEZE_STEP_TILED)
    torch.cuda.synchronize()
    return (b if steps % 2 else a).clone()


def test_batch_with_caller_records_matches_solo_runs():
    """Items whose border records the caller keeps (written once by
    squeeze_write_records, then kept current by the runs) give the same
    results as solo runs, across runs and a rebuilt batch."""
    shapes = [(I.CARPET, 6), (I.TRIANGLE, 9), (I.VICSEK, 7), (I.SINGLE, 3)]
    handles = [sq.Handle(f, r) for f, r in shapes]
    try:
        states, recs, starts = [], [], []
        for i, h in enumerate(handles):
            a = torch.empty(h.cells, dtype=torch.uint8, device="cuda")
            b = torch.empty_like(a)
            sq.squeeze_init_bernoulli(h.h, a, 500 + i, I.p_q24(0.5))
            n = sq.squeeze_record_bytes(h.h)
            assert n % 4 == 0 and (n > 0) == (shapes[i][0] is not I.SINGLE)
            ra = torch.empty(max(n, 4) // 4, dtype=torch.int32, device="cuda") if n else None
            rb = torch.empty_like(ra) if n else None
            if n:
                sq.squeeze_write_records(h.h, a, ra)
            states.append([a, b])
            recs.append([ra, rb])
            starts.append(a.clone())
        done = 0
        for run in (5, 8, 3):   # a new batch each time, buffers swapped after odd runs
            batch = sq.squeeze_batch_create_with_records(
                [(h.h, s[0], s[1]) for h, s in zip(handles, states)], [tuple(r) for r in recs])
            sq.squeeze_batch_run(batch, run)
            torch.cuda.synchronize()
            sq.squeeze_batch_destroy(batch)
            done += run
            if run % 2:
                for s, r in zip(states, recs):
                    s.reverse()
                    r.reverse()
            for h, s, s0, (f, rr) in zip(handles, states, starts, shapes):
                assert torch.equal(s[0], solo_from(h, s0, done)), (f.name, done)
        with pytest.raises(sq.SqueezeError):   # a program with records needs its buffers
            sq.squeeze_batch_create_with_records([(handles[0].h, states[0][0], states[0][1])],
                                                 [(None, None)])
    finally:
        for h in handles:
            h.close()
