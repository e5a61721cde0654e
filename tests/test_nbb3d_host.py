"""The 3-D step's per-cell arithmetic, run on the CPU, against the 3-D oracle.

The functions of nbb3d.cuh (compact split, lambda, nu, the neighbour walk) are
host-callable; tests/nbb3d_host.cu compiles them, with the kernel's per-cell
loop, into a host library.  Compared with the oracle: every cell and every box
point at small levels under symmetric and asymmetric neighbourhoods, and the
26 neighbour indices of sampled cells at 1e9 to 7e10 cells, where the walk
crosses up to 20 levels and compact indices pass 2^32.  No GPU is needed;
nvcc is (it compiles the file's kernels too).
"""
import ctypes
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import nbb3d as O3
from paper_2201_00613_gb300 import build as B
from paper_2201_00613_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
MAX = np.uint64(2 ** 64 - 1)
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def host(tmp_path_factory):
    nvcc = B._nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("nbb3d_host") / "libnbb3d_host.so")
    cmd = [nvcc] + B.ARCH + ["-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                             "-fPIC", "-shared", "-I", B.INCLUDE, "-I", B.CSRC,
                             os.path.join(HERE, "nbb3d_host.cu"), "-o", out, "-lcudart"]
    subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(out)


def ptr(a):
    return a.ctypes.data_as(P)


def offs(f):
    return np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)


def lam(L, f, r, om):
    om = np.ascontiguousarray(om, dtype=np.uint64)
    xyz = np.empty((om.size, 3), np.int32)
    assert L.h3_lambda(f.s, f.k, ptr(offs(f)), r, ptr(om), ptr(xyz), ctypes.c_uint64(om.size)) == 0
    return xyz.astype(np.int64)


def nu(L, f, r, pts):
    p = np.ascontiguousarray(pts, dtype=np.int32)
    o = np.empty(len(p), np.uint64)
    assert L.h3_nu(f.s, f.k, ptr(offs(f)), r, ptr(p), ptr(o), ctypes.c_uint64(len(p))) == 0
    return o


def step(L, f, r, state, rule, mask):
    st = np.ascontiguousarray(state, dtype=np.uint8)
    out = np.empty_like(st)
    bad = ctypes.c_uint64(7)
    assert L.h3_step(f.s, f.k, ptr(offs(f)), r, mask, rule[0], rule[1], ptr(st), ptr(out), None,
                     ctypes.c_uint64(0), ctypes.byref(bad)) == 0
    assert bad.value == 0
    return out


FORWARD = sum(1 << ((dz + 1) * 9 + (dy + 1) * 3 + dx + 1) for dx, dy, dz in
              [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (-1, 0, 1), (0, -1, -1), (1, 1, 1)])
CASES = [(O3.LIFE_4555, O3.MOORE3), (((1 << 1) | (1 << 2), (1 << 1) | (1 << 3)), O3.VON_NEUMANN3),
         (((1 << 1) | (1 << 2), (1 << 1) | (1 << 3)), FORWARD)]


@pytest.mark.parametrize("f,r", [(I.MENGER, 0), (I.MENGER, 2), (I.MENGER, 3), (I.TETRA, 1),
                                 (I.TETRA, 6), (I.CANTOR_DUST, 3), (I.FULL_CUBE, 4),
                                 (I.FLAT_TRIANGLE, 7), (I.SINGLE3, 4)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_host_per_cell_step_equals_the_oracle(host, f, r):
    info = np.zeros(5, dtype=np.uint64)
    assert host.h3_info(f.s, f.k, ptr(offs(f)), r, ptr(info)) == 0
    assert tuple(int(v) for v in info[1:4]) == O3.extents(f, r)
    om = np.arange(f.k ** r + 3, dtype=np.uint64)
    assert np.array_equal(lam(host, f, r, om), O3.lam(f, r, om))
    n = f.s ** r
    z, y, x = np.mgrid[-1:n + 1, -1:n + 1, -1:n + 1]
    pts = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    assert np.array_equal(nu(host, f, r, pts), O3.nu(f, r, pts))
    c0 = O3.init_compact(f, r, 5 + r, I.p_q24(0.4))
    for rule, mask in CASES:
        assert np.array_equal(step(host, f, r, c0, rule, mask),
                              O3.run_compact(f, r, c0, 1, rule, mask)), (rule, mask)


@pytest.mark.parametrize("f,r", [(I.MENGER, 7), (I.TETRA, 20), (I.CANTOR_DUST, 12),
                                 (I.FULL_CUBE, 12), (I.FLAT_TRIANGLE, 20)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_host_neighbour_walk_at_large_levels(host, f, r):
    cells = f.k ** r
    om = np.unique(np.concatenate([I.random_ints(r, 2000, cells).astype(np.uint64),
                                   np.array([0, 1, cells - 2, cells - 1], dtype=np.uint64)]))
    xyz = O3.lam(f, r, om)
    assert np.array_equal(lam(host, f, r, om), xyz)
    got = np.empty((om.size, 27), dtype=np.uint64)
    assert host.h3_neighbours(f.s, f.k, ptr(offs(f)), r, ptr(om), ctypes.c_uint64(om.size),
                              ptr(got)) == 0
    for d, (dz, dy, dx) in enumerate(itertools.product((-1, 0, 1), repeat=3)):
        want = O3.nu(f, r, xyz + [dx, dy, dz]) if d != 13 else np.full(om.size, MAX)
        assert np.array_equal(got[:, d], want), d
