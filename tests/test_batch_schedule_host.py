"""The batched step's work schedule (host code in batch.cu), on the CPU.

One launch of the batched kernel steps every instance once; CTA c walks the
schedule entries start[c] .. start[c + 1] - 1, each a run of tile groups of one
instance.  Checked: every group of every instance is in exactly one entry, the
entries run in (instance, group) order, every CTA's share of cells is within
one group of the even share, and the offsets are consistent, for random
mixes, the benchmark's 256-instance mix and edge cases (more CTAs than
groups, one instance, one group per instance).  No GPU is needed.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2201_00613_gb300 import build as B
from paper_2201_00613_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    nvcc = B._nvcc()
    if not (os.path.isabs(nvcc) and os.path.exists(nvcc)) and shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    out = str(tmp_path_factory.mktemp("batch_host") / "libbatch_host.so")
    cmd = [nvcc] + B.ARCH + ["-O1", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler",
                             "-fPIC", "-shared", "-I", B.INCLUDE, "-I", B.CSRC,
                             os.path.join(HERE, "batch_host.cu"), "-o", out, "-lcudart"]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(out)
    L.batch_schedule.restype = ctypes.c_int64
    return L


def schedule(lib, cells, groups, grid, strided=False):
    cells = np.ascontiguousarray(cells, dtype=np.uint64)
    groups = np.ascontiguousarray(groups, dtype=np.uint64)
    cap = int(groups.sum()) + len(cells) * grid + 1
    work = np.zeros((cap, 4), dtype=np.uint64)
    start = np.zeros(grid + 1, dtype=np.uint32)
    n = lib.batch_schedule(cells.ctypes.data_as(P), groups.ctypes.data_as(P), len(cells), grid,
                           int(strided), work.ctypes.data_as(P), ctypes.c_uint64(cap),
                           start.ctypes.data_as(P))
    assert n >= 0
    return work[:n].astype(np.int64), start.astype(np.int64)


def check(cells, groups, grid, work, start):
    cells, groups = np.asarray(cells, dtype=np.int64), np.asarray(groups, dtype=np.int64)
    assert start[0] == 0 and start[-1] == len(work) and np.all(np.diff(start) >= 0)
    # exact cover; contiguous runs come in (instance, group) order
    covered = [np.zeros(g, dtype=np.int64) for g in groups]
    prev = (-1, -1)
    for inst, g0, g1, step in work:
        assert 0 <= g0 < g1 <= groups[inst] and step >= 1
        if np.all(work[:, 3] == 1):
            assert (inst, g0) > prev
            prev = (inst, g1 - 1)
        covered[inst][g0:g1:step] += 1
    assert all(np.all(c == 1) for c in covered)
    # balance: each CTA's cells are within one group of total / grid
    per_group = cells / groups
    total = cells.sum()
    for c in range(grid):
        load = sum(len(range(g0, g1, step)) * per_group[inst]
                   for inst, g0, g1, step in work[start[c]:start[c + 1]])
        assert abs(load - total / grid) <= 2 * per_group.max() + 1e-6, (c, load, total / grid)


@pytest.mark.parametrize("seed", range(6))
def test_random_mixes(lib, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 60))
    groups = rng.integers(1, 400, n)
    cells = groups * rng.integers(1, 5000, n)
    grid = int(rng.choice([1, 7, 152, 304, 608]))
    work, start = schedule(lib, cells, groups, grid)
    check(cells, groups, grid, work, start)
    assert np.all(work[:, 3] == 1)
    work, start = schedule(lib, cells, groups, grid, strided=True)
    check(cells, groups, grid, work, start)


def test_benchmark_mix_shape(lib):
    # the 256-instance mix: cells k^r, groups from 27x27, 64x8 and 25x25 tiles, 32 per group
    mix = I.batch_mix()
    tile = {"sierpinski_triangle": 729, "sierpinski_carpet": 512, "vicsek": 625}
    cells = [i.fractal.cells(i.r) for i in mix]
    groups = [max(1, -(-c // tile[i.fractal.name] // 32)) for c, i in zip(cells, mix)]
    for grid in (304, 608):
        for strided in (False, True):
            work, start = schedule(lib, cells, groups, grid, strided)
            check(cells, groups, grid, work, start)
    # the large carpets are shared by runs of CTAs, which the strided form interleaves
    assert np.any(work[:, 3] > 1)


@pytest.mark.parametrize("cells,groups,grid", [
    ([1000], [3], 608),                 # more CTAs than groups
    ([5, 7, 9], [1, 1, 1], 2),          # one group per instance
    ([10 ** 9], [4096], 152),           # one large instance
    ([6561] * 300, [1] * 300, 152),     # many one-group instances
], ids=["few-groups", "one-group-each", "one-instance", "many-small"])
def test_edge_cases(lib, cells, groups, grid):
    for strided in (False, True):
        work, start = schedule(lib, cells, groups, grid, strided)
        check(cells, groups, grid, work, start)


def test_strided_runs_interleave_one_instance(lib):
    # one instance of 1000 groups over 7 CTAs: CTA q takes q, q + 7, ...
    work, start = schedule(lib, [10 ** 6], [1000], 7, strided=True)
    assert len(work) == 7 and np.all(np.diff(start) == 1)
    assert [tuple(w) for w in work] == [(0, q, 1000, 7) for q in range(7)]
