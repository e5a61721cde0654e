"""The three-dimensional tile kernel's host-built program, emulated on the CPU.

The 3-D tile kernel (tile3d.cu) evaluates no lambda or nu per cell: the host
builds, once per fractal and tile level, 26 references per local cell of a
tile (a level-L sub-replica) into a word array of the tile's cells, halo
cells of the 26 adjacent tiles (by direction) and a zero word.  This test
builds that program with the library's own host code (tests/tile3_host.cu),
runs one step with it in numpy over every tile of a level-r fractal, and
compares the result with the 3-D oracle's box step, for both tile-row widths
the kernel instantiates (8 and 16 cells) and several neighbourhoods and
rules.  The adjacent tiles come from the kernel's own rule (lambda of a
tile's first cell, moved by one block, nu back), which is checked against
tiles found by brute force from the oracle's maps.  No GPU is needed.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import nbb3d as O3
from paper_2201_00613_gb300 import build as B
from paper_2201_00613_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
P = ctypes.c_void_p
MAX = np.uint64(2 ** 64 - 1)
FORWARD = sum(1 << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1) for dx, dy, dz in
              [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 1), (0, -1, -1), (1, 1, 1)])


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = B._nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("tile3_host") / "libtile3_host.so")
    cmd = [nvcc] + B.ARCH + ["-O1", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                             "-fPIC", "-shared", "-I", B.INCLUDE, "-I", B.CSRC,
                             os.path.join(HERE, "tile3_host.cu"), "-o", out, "-lcudart"]
    subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(out)


def ptr(a):
    return a.ctypes.data_as(P)


def offsets(f):
    return np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)


def program(lib, f, r, L, nbhd):
    info = np.zeros(7, dtype=np.uint32)
    cap = 1 << 20
    refs = np.zeros(cap, dtype=np.uint16)
    halo_off = np.zeros(1 << 16, dtype=np.uint32)
    dirs = np.zeros(27, dtype=np.uint8)
    hs = np.zeros(28, dtype=np.uint32)
    rc = lib.tile3_program(f.s, f.k, ptr(offsets(f)), r, L, nbhd, ptr(info), ptr(refs),
                           ctypes.c_uint64(cap), ptr(halo_off), ctypes.c_uint64(len(halo_off)),
                           ptr(dirs), ptr(hs))
    assert rc == 0, rc
    TX, TY, TZ, slots, nhalo, ndirs, default = (int(v) for v in info)
    return dict(TX=TX, TY=TY, TZ=TZ, slots=slots, nhalo=nhalo, default=default,
                refs=(refs[:slots * 32] // 4).astype(np.int64).reshape(slots, 32),
                halo_off=halo_off[:nhalo].astype(np.int64), dirs=dirs[:ndirs].astype(np.int64),
                halo_start=hs.astype(np.int64))


def geometry(f, r, prog):
    Wx, Wy, Wz = O3.extents(f, r)
    TX, TY, TZ = prog["TX"], prog["TY"], prog["TZ"]
    tz, ty, tx = np.mgrid[0:Wz // TZ, 0:Wy // TY, 0:Wx // TX]
    bases = (tz.ravel() * TZ * Wx * Wy + ty.ravel() * TY * Wx + tx.ravel() * TX).astype(np.int64)
    c = np.arange(TX * TY * TZ)
    lx, ly, lz = c % TX, (c // TX) % TY, c // (TX * TY)
    loff = (lz * Wx * Wy + ly * Wx + lx).astype(np.int64)
    rpw = 32 // TX
    row = c // TX
    pos = (row % rpw) * TX + c % TX
    slot = (row // rpw) * 32 + 8 * (pos & 3) + (pos >> 2)
    return bases, loff, slot


def library_adjacency(lib, f, r, L, prog, nt):
    adj = np.full((nt, len(prog["dirs"])), -1, dtype=np.int64)
    for j, d in enumerate(prog["dirs"]):
        t = np.zeros(nt, dtype=np.uint32)
        assert lib.tile3_adjacency(f.s, f.k, ptr(offsets(f)), r, L, int(d), ptr(t)) == 0
        ok = t != np.uint32(2 ** 32 - 1)
        adj[ok, j] = t[ok]
    return adj


def oracle_adjacency(f, r, L, prog, bases):
    """Tile next to each tile in each direction: nu of any cell of the tile
    moved by one block, mapped to the tile holding it; the cell used is the
    tile's first cell (tile index from its compact coordinates)."""
    Wx, Wy, Wz = O3.extents(f, r)
    TX, TY, TZ = prog["TX"], prog["TY"], prog["TZ"]
    side = f.s ** L
    xyz = O3.lam(f, r, bases.astype(np.uint64))
    adj = np.full((len(bases), len(prog["dirs"])), -1, dtype=np.int64)
    for j, d in enumerate(prog["dirs"]):
        move = np.array([d % 3 - 1, (d // 3) % 3 - 1, d // 9 - 1]) * side
        om = O3.nu(f, r, xyz + move)
        ok = om != MAX
        o = om[ok].astype(np.int64)
        wx, wy, wz = o % Wx, (o // Wx) % Wy, o // (Wx * Wy)
        adj[ok, j] = ((wz // TZ) * (Wy // TY) + wy // TY) * (Wx // TX) + wx // TX
    return adj


def emulate_step(f, r, prog, state, adj, rule):
    bases, loff, slot = geometry(f, r, prog)
    slots, nhalo = prog["slots"], prog["nhalo"]
    words = np.zeros((len(bases), slots + nhalo + 1), dtype=np.int64)
    own = state[bases[:, None] + loff[None, :]].astype(np.int64) & 1
    words[:, slot] = own
    hs = prog["halo_start"]
    for j in range(len(prog["dirs"])):
        for h in range(hs[j], hs[j + 1]):
            a = adj[:, j]
            ok = a >= 0
            words[ok, slots + h] = state[bases[a[ok]] + prog["halo_off"][h]] & 1
    refs = prog["refs"][slot][:, :26]                 # (cells, 26)
    count = words[:, refs].sum(axis=2)
    nxt = np.where(own == 1, (rule[1] >> count) & 1, (rule[0] >> count) & 1)
    out = np.zeros_like(state)
    out[bases[:, None] + loff[None, :]] = nxt
    return out


CASES = [(I.TETRA, 4, 4, O3.MOORE3), (I.TETRA, 6, 4, O3.MOORE3), (I.TETRA, 6, 5, O3.MOORE3),
         (I.TETRA, 6, 6, FORWARD), (I.TETRA, 7, 5, O3.VON_NEUMANN3),
         (I.CANTOR_DUST, 4, 2, O3.MOORE3), (I.CANTOR_DUST, 4, 3, FORWARD),
         (I.FULL_CUBE, 4, 3, O3.MOORE3), (I.FULL_CUBE, 5, 2, O3.MOORE3),
         (I.TETRA, 5, 5, O3.MOORE3)]    # one tile per band of the box's size
RULES = [O3.LIFE_4555, ((1 << 0) | (1 << 6), (1 << 5) | (1 << 6) | (1 << 7))]


@pytest.mark.parametrize("f,r,L,nbhd", CASES,
                         ids=["%s-r%d-L%d-%x" % (f.name, r, L, m) for f, r, L, m in CASES])
def test_3d_program_step_equals_the_oracle(lib, f, r, L, nbhd):
    prog = program(lib, f, r, L, nbhd)
    bases, loff, slot = geometry(f, r, prog)
    assert len(loff) == f.k ** L and len(np.unique(slot)) == len(slot)
    adj = library_adjacency(lib, f, r, L, prog, len(bases))
    assert np.array_equal(adj, oracle_adjacency(f, r, L, prog, bases))
    state = O3.init_compact(f, r, 17 + r + L, I.p_q24(0.4))
    for rule in RULES:
        want = O3.run_compact(f, r, state, 1, rule, nbhd)
        assert np.array_equal(emulate_step(f, r, prog, state, adj, rule), want), rule


def test_3d_program_emulation_catches_a_shifted_halo_offset(lib):
    f, r, L = I.TETRA, 6, 4
    prog = program(lib, f, r, L, O3.MOORE3)
    bases, _, _ = geometry(f, r, prog)
    adj = library_adjacency(lib, f, r, L, prog, len(bases))
    state = O3.init_compact(f, r, 3, I.p_q24(0.5))
    want = O3.run_compact(f, r, state, 1, O3.LIFE_4555, O3.MOORE3)
    bad = dict(prog)
    bad["halo_off"] = prog["halo_off"] + 1
    assert not np.array_equal(emulate_step(f, r, bad, state, adj, O3.LIFE_4555), want)


def test_3d_tile_levels_the_kernel_takes(lib):
    # tile rows of 8 or 16 cells only; the Menger sponge (20) and the flat
    # triangle (powers of 3) stay on the per-cell kernel
    assert program(lib, I.TETRA, 15, 5, O3.MOORE3)["default"] == 5
    assert program(lib, I.CANTOR_DUST, 6, 3, O3.MOORE3)["default"] == 3
    info = np.zeros(7, dtype=np.uint32)
    refs = np.zeros(1 << 16, dtype=np.uint16)
    hoff = np.zeros(1 << 12, dtype=np.uint32)
    dirs = np.zeros(27, dtype=np.uint8)
    hs = np.zeros(28, dtype=np.uint32)
    for f, r, L in [(I.MENGER, 4, 2), (I.FLAT_TRIANGLE, 9, 3), (I.TETRA, 6, 7)]:
        rc = lib.tile3_program(f.s, f.k, ptr(offsets(f)), r, L, O3.MOORE3, ptr(info), ptr(refs),
                               ctypes.c_uint64(len(refs)), ptr(hoff), ctypes.c_uint64(len(hoff)),
                               ptr(dirs), ptr(hs))
        assert rc != 0
