"""The tiled step's host-built neighbour program, emulated on the CPU.

The tiled kernel never evaluates lambda or nu per cell: the host builds, once
per fractal and tile level, a program that gives every local cell of a tile
(a level-L sub-replica) 8 references into a word array of the tile's own
cells, halo cells of the adjacent tiles (by direction) and a zero word.  This
test builds that program with the library's own host code
(tests/tile_host.cu), runs one step with it in numpy over every tile of a
level-r fractal, and compares the result with the oracle's box step, for
every tile width the kernel instantiates (3, 9, 25, 27, shared 8- and 16-wide
slot words, 64-wide rows split in two) and several neighbourhoods.  The adjacent tiles come from
the kernel's own carry walk (host-callable), which is also compared with the
tiles the oracle's lambda and nu give.  No GPU is needed.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_2201_00613_gb300 import build as B
from paper_2201_00613_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
P = ctypes.c_void_p
MAX = np.uint64(2 ** 64 - 1)

DIAG2 = I.Fractal("diag2", 2, 2, ((0, 0), (1, 1)))
VON_NEUMANN = 0xAA
ONE_SIDED = sum(1 << ((dy + 1) * 3 + dx + 1) for dx, dy in [(1, 0), (1, 1), (0, -1), (-1, 1)])


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = B._nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("tile_host") / "libtile_host.so")
    cmd = [nvcc] + B.ARCH + ["-O1", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                             "-fPIC", "-shared", "-I", B.INCLUDE, "-I", B.CSRC,
                             os.path.join(HERE, "tile_host.cu"), "-o", out, "-lcudart"]
    subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(out)


def ptr(a):
    return a.ctypes.data_as(P)


def program(lib, f, r, L, nbhd, passes=1):
    off = np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)
    caps = np.zeros(3, dtype=np.uint64)
    assert lib.tile_sizes(f.s, f.k, ptr(off), r, L, ptr(caps)) == 0
    cells, slots, halo = (int(v) for v in caps)
    info = np.zeros(18, dtype=np.uint32)
    slot = np.zeros(cells, dtype=np.uint32)
    X = np.zeros(cells, dtype=np.uint32)
    Y = np.zeros(cells, dtype=np.uint32)
    refs16 = np.zeros((slots + halo) * 8, dtype=np.uint16)
    halo_off = np.zeros(halo, dtype=np.uint32)
    halo_dir = np.zeros(halo, dtype=np.uint8)
    dir_list = np.zeros(9, dtype=np.uint8)
    rc = lib.tile_program(f.s, f.k, ptr(off), r, L, nbhd, passes, ptr(info), ptr(slot), ptr(X),
                          ptr(Y), ptr(refs16), ptr(halo_off), ptr(halo_dir), ptr(dir_list))
    if rc and passes > 1:
        return None     # rings deeper than the box is wide: the library builds fewer passes
    assert rc == 0, rc
    TW, TH, rpw, wpr, ncell, nslot, nhalo, ndirs, npass = (int(v) for v in info[:9])
    ring_end = [int(v) for v in info[9:18]]
    nrows = nslot + ring_end[npass - 1]
    return dict(TW=TW, TH=TH, rpw=rpw, wpr=wpr, cells=ncell, slots=nslot, nhalo=nhalo,
                passes=npass, ring_end=ring_end, nhalo1=ring_end[1],
                slot=slot[:ncell].astype(np.int64), X=X[:ncell].astype(np.int64),
                Y=Y[:ncell].astype(np.int64), refs=(refs16[:nrows * 8] // 4).astype(np.int64),
                halo_off=halo_off[:nhalo].astype(np.int64), halo_dir=halo_dir[:nhalo],
                dir_list=dir_list[:ndirs])


def tile_bases(f, r, prog):
    W, H = oracle.compact_shape(f, r)[::-1]
    ty, tx = np.mgrid[0:H // prog["TH"], 0:W // prog["TW"]]
    return (ty.ravel() * prog["TH"] * W + tx.ravel() * prog["TW"]).astype(np.int64)


def oracle_adjacency(f, r, L, prog):
    """Base of the tile adjacent to each tile in each program direction (-1:
    none), from the oracle's lambda and nu of the tiles' first cells."""
    bases, side = tile_bases(f, r, prog), f.s ** L
    origin = oracle.lam(f, r, bases.astype(np.uint64)) - [prog["X"][0], prog["Y"][0]]
    adj = np.full((len(bases), len(prog["dir_list"])), -1, dtype=np.int64)
    for j, d in enumerate(prog["dir_list"]):
        bx, by = int(d) % 3 - 1, int(d) // 3 - 1
        q = origin + [bx * side + prog["X"][0], by * side + prog["Y"][0]]
        om = oracle.nu(f, r, q)
        ok = om != MAX
        adj[ok, j] = om[ok].astype(np.int64)        # cell 0 of a tile is its base
    return adj


def library_adjacency(lib, f, r, L, prog):
    """The same from the kernel's carry walk (tile indices turned into bases)."""
    off = np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)
    bases = tile_bases(f, r, prog)
    adj = np.full((len(bases), len(prog["dir_list"])), -1, dtype=np.int64)
    for j, d in enumerate(prog["dir_list"]):
        t = np.zeros(len(bases), dtype=np.uint32)
        assert lib.tile_adjacency(f.s, f.k, ptr(off), r, L, int(d), ptr(t)) == 0
        ok = t != np.uint32(2 ** 32 - 1)
        adj[ok, j] = bases[t[ok].astype(np.int64)]
    return adj


def emulate_step(f, r, L, prog, state, adj, rule=oracle.B3S23):
    """One step of every tile through the program's word array (numpy)."""
    W = oracle.compact_shape(f, r)[1]
    TW = prog["TW"]
    bases = tile_bases(f, r, prog)
    loff = (np.arange(prog["cells"]) // TW) * W + np.arange(prog["cells"]) % TW
    words = np.zeros((len(bases), prog["slots"] + prog["nhalo"] + 1), dtype=np.int64)
    own = state[bases[:, None] + loff[None, :]].astype(np.int64) & 1
    words[:, prog["slot"]] = own
    for i in range(prog["nhalo"]):
        a = adj[:, prog["halo_dir"][i]]
        ok = a >= 0
        words[ok, prog["slots"] + i] = state[a[ok] + prog["halo_off"][i]] & 1
    refs = prog["refs"].reshape(-1, 8)[prog["slot"]]          # (cells, 8)
    count = words[:, refs].sum(axis=2)                        # (tiles, cells)
    nxt = np.where(own == 1, (rule[1] >> count) & 1, (rule[0] >> count) & 1)
    out = np.zeros_like(state)
    out[bases[:, None] + loff[None, :]] = nxt
    return out


def emulate_passes(f, r, L, prog, state, adj, rule=oracle.B3S23, mask=True):
    """P = prog["passes"] steps of every tile through the program, as one
    launch runs them: the tile's words and halo rings 1..P from the state,
    then for t = 1 .. P-1 step t of the slots and of rings 1..P-t (a ring cell
    of a missing tile stays dead), then step P of the tile from those."""
    W = oracle.compact_shape(f, r)[1]
    TW, slots, P = prog["TW"], prog["slots"], prog["passes"]
    bases = tile_bases(f, r, prog)
    loff = (np.arange(prog["cells"]) // TW) * W + np.arange(prog["cells"]) % TW
    nw = slots + prog["nhalo"] + 1
    x = np.zeros((len(bases), nw), dtype=np.int64)
    x[:, prog["slot"]] = state[bases[:, None] + loff[None, :]].astype(np.int64) & 1
    exists = np.zeros((len(bases), prog["nhalo"]), dtype=np.int64)
    for i in range(prog["nhalo"]):
        a = adj[:, prog["halo_dir"][i]]
        ok = a >= 0
        x[ok, slots + i] = state[a[ok] + prog["halo_off"][i]] & 1
        exists[:, i] = ok
    refs = prog["refs"].reshape(-1, 8)                        # rows: slots, then the first ring

    def rule_rows(words, rows):
        count = words[:, refs[rows]].sum(axis=2)
        own = words[:, rows]
        return np.where(own == 1, (rule[1] >> count) & 1, (rule[0] >> count) & 1)

    for t in range(1, P):
        n = prog["ring_end"][P - t]
        y = np.zeros_like(x)
        y[:, prog["slot"]] = rule_rows(x, prog["slot"])
        ring = np.arange(slots, slots + n)
        y[:, ring] = rule_rows(x, ring) & (exists[:, :n] if mask else 1)
        x = y
    nxt = rule_rows(x, prog["slot"])
    out = np.zeros_like(state)
    out[bases[:, None] + loff[None, :]] = nxt
    return out


CASES = [
    (I.TRIANGLE, 8, 2, oracle.MOORE), (I.TRIANGLE, 8, 3, oracle.MOORE),
    (I.TRIANGLE, 8, 5, oracle.MOORE), (I.TRIANGLE, 9, 6, oracle.MOORE),
    (I.TRIANGLE, 9, 6, VON_NEUMANN), (I.TRIANGLE, 9, 6, ONE_SIDED),
    (I.TRIANGLE_PAPER, 8, 6, oracle.MOORE),
    (I.CARPET, 5, 2, oracle.MOORE), (I.CARPET, 5, 3, oracle.MOORE), (I.CARPET, 5, 3, ONE_SIDED),
    (I.VICSEK, 6, 3, oracle.MOORE), (I.VICSEK, 6, 4, oracle.MOORE),
    (I.FULL2, 8, 3, oracle.MOORE), (I.FULL2, 8, 4, oracle.MOORE), (I.FULL2, 8, 5, oracle.MOORE),
    (DIAG2, 10, 5, oracle.MOORE), (DIAG2, 10, 7, oracle.MOORE), (DIAG2, 10, 9, VON_NEUMANN),
    (I.TRIANGLE, 6, 6, oracle.MOORE), (I.CARPET, 3, 3, oracle.MOORE),   # one tile: no neighbours
]


@pytest.mark.parametrize("f,r,L,nbhd", CASES,
                         ids=["%s-r%d-L%d-%x" % (f.name, r, L, m) for f, r, L, m in CASES])
def test_program_step_equals_the_oracle(lib, f, r, L, nbhd):
    prog = program(lib, f, r, L, nbhd)
    assert prog["cells"] == f.k ** L
    state = I.bernoulli_bytes(100 + r + L, f.k ** r, 0.45)
    m = oracle.member_grid(f, r)
    want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(
        m, oracle.compact_to_box(f, r, state), 1, oracle.B3S23, nbhd))
    adj = library_adjacency(lib, f, r, L, prog)
    assert np.array_equal(adj, oracle_adjacency(f, r, L, prog))
    assert np.array_equal(emulate_step(f, r, L, prog, state, adj), want)


def test_program_shapes_cover_every_kernel_width(lib):
    seen = set()
    for f, r, L, nbhd in CASES:
        p = program(lib, f, r, L, nbhd)
        seen.add((p["TW"], p["rpw"], p["wpr"]))
    assert {(27, 1, 1), (25, 1, 1), (8, 4, 1), (16, 2, 1), (64, 1, 2)} <= seen


TWO_STEP_RULES = [oracle.B3S23, ((1 << 3) | (1 << 6), (1 << 2) | (1 << 3)),   # Life, HighLife
                  ((1 << 0) | (1 << 3), (1 << 2) | (1 << 3))]                 # B03/S23: birth at 0


@pytest.mark.parametrize("passes", [2, 4, 8])
@pytest.mark.parametrize("f,r,L,nbhd", CASES,
                         ids=["%s-r%d-L%d-%x" % (f.name, r, L, m) for f, r, L, m in CASES])
def test_multi_step_program_equals_oracle_steps(lib, f, r, L, nbhd, passes):
    prog = program(lib, f, r, L, nbhd, passes=passes)
    one = program(lib, f, r, L, nbhd)
    if prog is None:
        assert f.s ** L < passes    # the only reason the builder refuses more passes
        return
    assert prog["passes"] == passes
    # ring 1, its order and the slots' references are the one-step program's
    assert prog["nhalo1"] == one["nhalo"] and prog["nhalo"] >= prog["nhalo1"]
    assert np.array_equal(prog["halo_off"][:prog["nhalo1"]], one["halo_off"])
    zero1, zero2 = one["slots"] + one["nhalo"], prog["slots"] + prog["nhalo"]
    r1 = one["refs"].copy()
    r1[r1 == zero1] = zero2
    assert np.array_equal(prog["refs"][:prog["slots"] * 8], r1)
    state = I.bernoulli_bytes(200 + r + L, f.k ** r, 0.45)
    m = oracle.member_grid(f, r)
    adj = library_adjacency(lib, f, r, L, prog)
    for rule in TWO_STEP_RULES:
        want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(
            m, oracle.compact_to_box(f, r, state), passes, rule, nbhd))
        assert np.array_equal(emulate_passes(f, r, L, prog, state, adj, rule), want), rule


def test_multi_step_emulation_catches_a_dropped_existence_mask(lib):
    # Without the mask a ring cell of a missing tile can be born (rule B03
    # births at 0 neighbours) and feed the next step: the result must differ.
    f, r, L = I.TRIANGLE, 8, 3
    for passes in (2, 4, 8):
        prog = program(lib, f, r, L, oracle.MOORE, passes=passes)
        adj = library_adjacency(lib, f, r, L, prog)
        state = I.bernoulli_bytes(7, f.k ** r, 0.45)
        rule = TWO_STEP_RULES[2]
        want = oracle.box_to_compact(f, r, oracle.box_run_nbhd(
            oracle.member_grid(f, r), oracle.compact_to_box(f, r, state), passes, rule,
            oracle.MOORE))
        assert np.array_equal(emulate_passes(f, r, L, prog, state, adj, rule), want)
        assert not np.array_equal(emulate_passes(f, r, L, prog, state, adj, rule, mask=False),
                                  want)


CHUNK_CASES = [(I.CARPET, 5, 3, oracle.MOORE), (I.CARPET, 6, 3, VON_NEUMANN),
               (I.CARPET, 6, 3, ONE_SIDED), (I.FULL2, 7, 5, oracle.MOORE),
               (I.TRIANGLE, 8, 6, oracle.MOORE)]


def chunk_table(lib, f, r, L, nbhd, passes):
    off = np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)
    caps = np.zeros(3, dtype=np.uint64)
    assert lib.tile_sizes(f.s, f.k, ptr(off), r, L, ptr(caps)) == 0
    slots, halo = int(caps[1]), int(caps[2])
    info = np.zeros(23, dtype=np.uint32)
    table = np.zeros(5 * halo + slots // 2 + 300, dtype=np.uint32)
    hoff = np.zeros(halo, dtype=np.uint32)
    hdir = np.zeros(halo, dtype=np.uint8)
    rc = lib.tile_chunks(f.s, f.k, ptr(off), r, L, nbhd, passes, ptr(info), ptr(table), ptr(hoff),
                         ptr(hdir))
    return rc, info, table, hoff, hdir


@pytest.mark.parametrize("passes", [1, 2, 4, 8])
@pytest.mark.parametrize("f,r,L,nbhd", CHUNK_CASES,
                         ids=["%s-r%d-L%d-%x" % (f.name, r, L, m) for f, r, L, m in CHUNK_CASES])
def test_halo_chunk_table_serves_every_halo_cell(lib, f, r, L, nbhd, passes):
    """64-wide rows gather the halo by 16-byte chunks of the adjacent tile: the
    table must hold every halo word exactly once, in the chunk and at the byte
    of its offset, under its own direction; other widths carry no table."""
    prog = program(lib, f, r, L, nbhd, passes=passes)
    if prog is None:
        return
    rc, info, table, hoff, hdir = chunk_table(lib, f, r, L, nbhd, passes)
    assert rc == 0
    nhalo, ndirs, W = prog["nhalo"], len(prog["dir_list"]), f.k ** ((r + 1) // 2)
    assert np.array_equal(hoff[:nhalo], prog["halo_off"])
    nch, cs = int(info[0]), info[1:11].astype(np.int64)
    if prog["TW"] != 64:
        assert nch == 0
        return
    assert nch > 0 and cs[0] == 0 and cs[ndirs] == nch and np.all(np.diff(cs) >= 0)
    assert np.all(cs[ndirs:] == nch)
    coff = table[:nch].astype(np.int64)
    cstart = table[nch:2 * nch + 1].astype(np.int64)
    cells = table[2 * nch + 1:2 * nch + 1 + nhalo].astype(np.int64)
    assert cstart[0] == 0 and cstart[-1] == nhalo and np.all(np.diff(cstart) > 0)
    assert np.all(coff % 16 == 0)
    assert np.all(coff // W < prog["TH"]) and np.all(coff % W + 16 <= prog["TW"])
    seen = np.zeros(nhalo, dtype=np.int64)
    for j in range(ndirs):
        assert np.all(np.diff(coff[cs[j]:cs[j + 1]]) > 0)   # distinct, increasing
        for c in range(cs[j], cs[j + 1]):
            ent = cells[cstart[c]:cstart[c + 1]]
            h, byte = ent & 0xFFFF, ent >> 16
            assert np.all(np.diff(h) > 0)                    # ring by ring
            assert np.all(hdir[h] == j)
            assert np.all(coff[c] + byte == prog["halo_off"][h])
            seen[h] += 1
    assert np.all(seen == 1)


RECORD_CASES = CHUNK_CASES + [(I.VICSEK, 7, 4, oracle.MOORE), (I.TRIANGLE, 9, 5, VON_NEUMANN),
                              (I.TRIANGLE, 8, 3, ONE_SIDED), (I.FULL2, 6, 4, oracle.MOORE),
                              (DIAG2, 8, 4, oracle.MOORE)]


@pytest.mark.parametrize("passes", [1, 4, 8])
@pytest.mark.parametrize("f,r,L,nbhd", RECORD_CASES,
                         ids=["%s-r%d-L%d-%x" % (f.name, r, L, m) for f, r, L, m in RECORD_CASES])
def test_border_records_carry_every_halo_word(lib, f, r, L, nbhd, passes):
    """The tiled step reads its halo from the adjacent tiles' border records:
    emulate a launch writing every tile's record from its final words (kept
    for the exported cells only) and the next reading them (its halo words),
    and compare each halo word with the direct gather through halo_off."""
    prog = program(lib, f, r, L, nbhd, passes=passes)
    if prog is None:
        return
    rc, info, table, hoff, hdir = chunk_table(lib, f, r, L, nbhd, passes)
    assert rc == 0
    nhalo, ndirs, nch = prog["nhalo"], len(prog["dir_list"]), int(info[0])
    R, seg, nexp = int(info[11]), info[12:22].astype(np.int64), int(info[22])
    if nhalo == 0:
        assert R == 0
        return
    assert R > 0 and seg[0] == 0 and seg[ndirs] == R and np.all(seg[ndirs:] == R)
    base = 2 * nch + 1 + nhalo if nch else 0
    rtab = table[base:base + 32 * R].astype(np.int64)
    exp_slot = table[base + 32 * R:base + 32 * R + nexp].astype(np.int64)
    packed = table[base + 32 * R + nexp:base + 32 * R + nexp + (prog["slots"] + 1) // 2]
    exp_of = np.stack([packed & 0xFFFF, packed >> 16], axis=1).reshape(-1)[:prog["slots"]]
    pad = rtab == 0xFFFFFFFF
    e_of, h_of = rtab & 0xFFFF, rtab >> 16
    # the exported cells: distinct slots, each mapped back to its number
    assert 0 < nexp <= nhalo and len(set(exp_slot.tolist())) == nexp
    assert np.array_equal(exp_of[exp_slot], np.arange(nexp))
    assert np.sum(exp_of != 0xFFFF) == nexp and np.all(e_of[~pad] < nexp)
    slot_of = np.where(pad, 0, exp_slot[np.where(pad, 0, e_of)])
    # every halo word once, in its own direction's segment, ring by ring
    assert sorted(h_of[~pad].tolist()) == list(range(nhalo))
    for j in range(ndirs):
        hs = h_of[32 * seg[j]:32 * seg[j + 1]][~pad[32 * seg[j]:32 * seg[j + 1]]]
        assert np.all(hdir[hs] == j) and np.all(np.diff(hs) > 0)
        assert seg[j + 1] - seg[j] == -(-len(hs) // 32)
    # emulation over every tile of a random state
    W, TW, TH = f.k ** ((r + 1) // 2), prog["TW"], prog["TH"]
    tiles_x, tiles_y = W // TW, f.k ** (r // 2) // TH
    state = I.bernoulli_bytes(41 + r, f.k ** r, 0.5).reshape(-1, W)
    tiles = state.reshape(tiles_y, TH, tiles_x, TW).transpose(0, 2, 1, 3).reshape(-1, TH * TW)
    words = np.zeros((len(tiles), prog["slots"]), dtype=np.int64)   # slot word per tile
    words[:, prog["slot"]] = tiles[:, :prog["cells"]] & 1
    rec = np.where(pad, 0, words[:, np.where(pad, 0, slot_of)])   # record bits per tile
    adj = library_adjacency(lib, f, r, L, prog)     # base of the adjacent tile, or -1
    for j in range(ndirs):
        base = adj[:, j]
        ok = base >= 0
        b = np.where(ok, base, 0)
        t = (b // (TH * W)) * tiles_x + (b % W) // TW
        for pos in range(32 * seg[j], 32 * seg[j + 1]):
            if pad[pos]:
                continue
            h = h_of[pos]
            got = np.where(ok, rec[t, pos], 0)
            want = np.where(ok, state.reshape(-1)[b + prog["halo_off"][h]] & 1, 0)
            assert np.array_equal(got, want), (j, h)
