"""The two-dimensional per-cell maps, run on the CPU, against the oracle.

lambda_alu, nu_alu and neighbour_omega (the carry walk of nu from a cell's own
digits) are what the per-cell step, the heat and Ising kernels, the block
layout and the lambda(omega) approach compute on the GPU.  They are
host-callable; tests/maps_host.cu compiles them into a host library.  Compared
with the oracle: every cell, every box point and a ring around the box at
small levels, and sampled cells up to level 30 (2e14 cells) and the s = 16,
k = 255 fractal's widest weights.  No GPU is needed.
"""
import ctypes
import itertools
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
BIG = I.Fractal("s16_k255", 16, 255,
                tuple((x, y) for y in range(16) for x in range(16) if (x, y) != (15, 15)))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = B._nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("maps_host") / "libmaps_host.so")
    cmd = [nvcc] + B.ARCH + ["-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                             "-fPIC", "-shared", "-I", B.INCLUDE, "-I", B.CSRC,
                             os.path.join(HERE, "maps_host.cu"), "-o", out, "-lcudart"]
    subprocess.run(cmd, check=True, capture_output=True)
    return ctypes.CDLL(out)


def ptr(a):
    return a.ctypes.data_as(P)


def call(lib, name, f, r, *arrays):
    off = np.ascontiguousarray(f.offsets_array(), dtype=np.uint8)
    args = [ptr(a) if isinstance(a, np.ndarray) else ctypes.c_uint64(a) for a in arrays]
    assert getattr(lib, name)(f.s, f.k, ptr(off), r, *args) == 0


def lam(lib, f, r, om):
    om = np.ascontiguousarray(om, dtype=np.uint64)
    xy = np.empty((om.size, 2), dtype=np.int64)
    call(lib, "h2_lambda", f, r, om, xy, om.size)
    return xy


def nu(lib, f, r, pts):
    p = np.ascontiguousarray(pts, dtype=np.int64)
    om = np.empty(len(p), dtype=np.uint64)
    call(lib, "h2_nu", f, r, p, om, len(p))
    return om


def neighbours(lib, f, r, om):
    om = np.ascontiguousarray(om, dtype=np.uint64)
    out = np.empty((om.size, 9), dtype=np.uint64)
    call(lib, "h2_neighbours", f, r, om, om.size, out)
    return out


def check_neighbours(lib, f, r, om):
    xy = oracle.lam(f, r, om)
    got = neighbours(lib, f, r, om)
    for d, (dy, dx) in enumerate(itertools.product((-1, 0, 1), repeat=2)):
        want = oracle.nu(f, r, xy + [dx, dy]) if d != 4 else np.full(om.size, MAX)
        assert np.array_equal(got[:, d], want), d


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 7), (I.TRIANGLE_PAPER, 6), (I.CARPET, 4),
                                 (I.VICSEK, 5), (I.FULL2, 6), (I.SINGLE, 4), (DIAG2, 9), (BIG, 2),
                                 (I.TRIANGLE, 0), (I.CARPET, 1), (BIG, 1)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_maps_and_walk_on_every_cell(lib, f, r):
    om = np.arange(f.k ** r + 3, dtype=np.uint64)
    assert np.array_equal(lam(lib, f, r, om), oracle.lam(f, r, om))
    n = f.s ** r
    yy, xx = np.mgrid[-1:n + 1, -1:n + 1]
    pts = np.stack([xx.ravel(), yy.ravel()], axis=1)
    assert np.array_equal(nu(lib, f, r, pts), oracle.nu(f, r, pts))
    check_neighbours(lib, f, r, np.arange(f.k ** r, dtype=np.uint64))


@pytest.mark.parametrize("f,r", [(I.TRIANGLE, 20), (I.TRIANGLE, 30), (I.CARPET, 10),
                                 (I.VICSEK, 13), (I.FULL2, 30), (DIAG2, 30), (BIG, 7)],
                         ids=lambda v: getattr(v, "name", str(v)))
def test_maps_and_walk_sampled_at_large_levels(lib, f, r):
    cells = f.k ** r
    om = np.unique(np.concatenate([I.random_ints(r + 7, 3000, min(cells, 2 ** 62)).astype(np.uint64),
                                   np.array([0, 1, cells - 2, cells - 1], dtype=np.uint64)]))
    xy = lam(lib, f, r, om)
    assert np.array_equal(xy, oracle.lam(f, r, om))
    assert np.array_equal(nu(lib, f, r, xy), om)
    check_neighbours(lib, f, r, om)
