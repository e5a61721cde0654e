"""Seeded synthetic inputs: fractal descriptors, random cell states, workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds *inputs only*: replica-offset tables that define each NBB fractal, seeded
random draws, and the workload recipes (level, step count, seed, density).  It
contains none of the method's arithmetic (no lambda/nu map, no membership test,
no cellular-automaton rule) and imports neither the CUDA library nor the oracle.

Fractal notation follows Sec. 3: an NBB fractal F_n^{k,s} replicates itself k
times per level, each replica translated by an offset tau(beta) in [0, s)^2
(Eq. tau); the level-r fractal lives in an n x n box with n = s^r.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Fractal:
    """An NBB fractal: growth factor s, replica count k, offsets tau[0..k-1]."""

    name: str
    s: int
    k: int
    offsets: tuple  # k pairs (tau_x, tau_y), each coordinate in [0, s)

    def offsets_array(self) -> np.ndarray:
        """Offsets as a (k, 2) uint8 array, row beta = (tau_x, tau_y)."""
        return np.asarray(self.offsets, dtype=np.uint8).reshape(self.k, 2)

    def cells(self, r: int) -> int:
        """k^r, the fractal volume V at level r (Sec. 3, Eq. V)."""
        return self.k ** r

    def side(self, r: int) -> int:
        """n = s^r, side of the expanded bounding box."""
        return self.s ** r


# Sierpinski triangle in the orientation used by the workloads:
# replicas at (0,0), (1,0), (0,1); membership is (x & y) == 0.
TRIANGLE = Fractal("sierpinski_triangle", 2, 3, ((0, 0), (1, 0), (0, 1)))

# Sierpinski triangle in the orientation printed in Sec. 3.3 / Sec. 4:
# tau(0)=(0,0) top, tau(1)=(0,1) middle, tau(2)=(1,1) right.
TRIANGLE_PAPER = Fractal("sierpinski_triangle_paper", 2, 3, ((0, 0), (0, 1), (1, 1)))

# Sierpinski carpet F^{8,3}: the 3x3 grid minus its centre, raster order
# (y-major, x fastest).
CARPET = Fractal(
    "sierpinski_carpet", 3, 8,
    ((0, 0), (1, 0), (2, 0), (0, 1), (2, 1), (0, 2), (1, 2), (2, 2)),
)

# Vicsek cross F^{5,3}: centre plus the four edge centres, raster order.
VICSEK = Fractal("vicsek", 3, 5, ((1, 0), (0, 1), (1, 1), (2, 1), (1, 2)))

# s = 2 with all four offsets: no holes, the fractal is the whole box.
FULL2 = Fractal("full_box_s2", 2, 4, ((0, 0), (1, 0), (0, 1), (1, 1)))

# One cell per level: the level-r fractal is a single cell.
SINGLE = Fractal("single_cell", 2, 1, ((0, 0),))

MIX = (TRIANGLE, CARPET, VICSEK)


@dataclasses.dataclass(frozen=True)
class Fractal3:
    """A three-dimensional NBB fractal: offsets tau in [0, s)^3 (the paper's
    extension to three dimensions, abstract and Sec. 7)."""

    name: str
    s: int
    k: int
    offsets: tuple  # k triples (tau_x, tau_y, tau_z), each coordinate in [0, s)

    def offsets_array(self) -> np.ndarray:
        """Offsets as a (k, 3) uint8 array, row beta = (tau_x, tau_y, tau_z)."""
        return np.asarray(self.offsets, dtype=np.uint8).reshape(self.k, 3)

    def cells(self, r: int) -> int:
        return self.k ** r

    def side(self, r: int) -> int:
        return self.s ** r


# Menger sponge F^{20,3}: the 3x3x3 cube minus its centre and the six face
# centres, raster order (z-major, then y, x fastest).
MENGER = Fractal3("menger_sponge", 3, 20, tuple(
    (x, y, z) for z in range(3) for y in range(3) for x in range(3)
    if (x == 1) + (y == 1) + (z == 1) <= 1))

# Sierpinski tetrahedron on the cube's corner (s = 2): the origin and its
# three axis neighbours.
TETRA = Fractal3("sierpinski_tetrahedron", 2, 4, ((0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1)))

# Cantor dust F^{8,3}: the eight corners of the 3x3x3 cube.
CANTOR_DUST = Fractal3("cantor_dust", 3, 8, tuple(
    (x, y, z) for z in (0, 2) for y in (0, 2) for x in (0, 2)))

# s = 2 with all eight octants: no holes, the fractal is the whole cube.
FULL_CUBE = Fractal3("full_cube_s2", 2, 8, tuple(
    (x, y, z) for z in range(2) for y in range(2) for x in range(2)))

# The Sierpinski triangle in the plane z = 0: a 3-D fractal with a flat slab.
FLAT_TRIANGLE = Fractal3("flat_triangle", 2, 3, ((0, 0, 0), (1, 0, 0), (0, 1, 0)))

# One cell per level.
SINGLE3 = Fractal3("single_cell_3d", 2, 1, ((0, 0, 0),))

# Level ranges of the batched mixed workload, per fractal type.
MIX_LEVELS = {"sierpinski_triangle": (8, 14), "sierpinski_carpet": (4, 8), "vicsek": (5, 9)}


def p_q24(p: float) -> int:
    """Alive probability p as a 24-bit fixed-point threshold floor(p * 2^24)."""
    return int(math.floor(p * (1 << 24)))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One single-fractal workload: Bernoulli(p) initial state, n_steps steps."""

    name: str
    fractal: Fractal
    r: int
    p: float
    seed: int
    n_steps: int

    @property
    def cells(self) -> int:
        return self.fractal.cells(self.r)


# Triangle r = 10, Bernoulli(0.5), seed 1, 100 steps.
TRIANGLE_R10 = Workload("sierpinski_triangle_r10", TRIANGLE, 10, 0.5, 1, 100)
# Triangle r = 16, Bernoulli(0.3), seed 2, 1000 steps.
TRIANGLE_R16 = Workload("sierpinski_triangle_r16", TRIANGLE, 16, 0.3, 2, 1000)
# Triangle r = 20, Bernoulli(0.5), seed 3, 100 steps.
TRIANGLE_R20 = Workload("sierpinski_triangle_r20", TRIANGLE, 20, 0.5, 3, 100)
# Seed for the uniform sample of compact indices checked at r = 20.
R20_SAMPLE_SEED = 4


def bernoulli_bytes(seed: int, count: int, p: float = 0.5) -> np.ndarray:
    """count uint8 cells in {0, 1}, each 1 with probability p (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    return (rng.random(count) < p).astype(np.uint8)


def random_ints(seed: int, count: int, high: int) -> np.ndarray:
    """count uniform int64 draws from [0, high)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, high, size=count, dtype=np.int64)


@dataclasses.dataclass(frozen=True)
class Instance:
    """One member of a batched mix: a fractal, its level and its own seed."""

    fractal: Fractal
    r: int
    seed: int
    p: float = 0.5


def batch_mix(seed: int = 5, count: int = 256, levels: dict | None = None) -> list:
    """count instances, type uniform over MIX, level uniform over its range."""
    levels = levels or MIX_LEVELS
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        f = MIX[int(rng.integers(0, len(MIX)))]
        lo, hi = levels[f.name]
        r = int(rng.integers(lo, hi + 1))
        out.append(Instance(f, r, int(rng.integers(0, 2**31 - 1))))
    return out


# Largest level per type with k^r <= 3^18 cells.
REQUEST_LEVELS = {"sierpinski_triangle": (8, 18), "sierpinski_carpet": (4, 9), "vicsek": (5, 12)}


@dataclasses.dataclass(frozen=True)
class Request:
    """One simulation request of the request loop."""

    rid: int
    arrival_s: float
    instance: Instance
    n_steps: int


def request_stream(seed: int = 6, count: int = 10000, rate_per_s: float = 1000.0,
                   levels: dict | None = None, steps: tuple = (10, 500)) -> list:
    """Poisson arrivals at rate_per_s; type uniform; level uniform; steps uniform."""
    levels = levels or REQUEST_LEVELS
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        f = MIX[int(rng.integers(0, len(MIX)))]
        lo, hi = levels[f.name]
        r = int(rng.integers(lo, hi + 1))
        n_steps = int(rng.integers(steps[0], steps[1] + 1))
        out.append(Request(i, t, Instance(f, r, int(rng.integers(0, 2**31 - 1))), n_steps))
    return out
