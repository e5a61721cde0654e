"""Plain CPU oracle for the compact-fractal cellular automaton (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline use this package.  It wraps ``squeeze_oracle.c`` (plain C, OpenMP over
rows) through ctypes and shares nothing with the CUDA library: it neither
imports the product package nor loads its shared object.

Every function restates a definition of the paper (arXiv 2201.00613):
membership of an NBB fractal (Sec. 3), lambda (Sec. 3.3), nu (Sec. 3.4), the
bounding-box Game-of-Life step over fractal cells (Sec. 4), plus the SplitMix64
initial-state generator and a light-cone sampler for levels too large for the
box.  The readings of garbled passages are listed at the top of the C file.
The three-dimensional extension (``oracle.nbb3d``, ``nbb3d_oracle.c``) lives
in the same library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "squeeze_oracle.c")
_SOURCES = [_SRC, os.path.join(_HERE, "nbb3d_oracle.c")]
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

B3S23 = (1 << 3, (1 << 2) | (1 << 3))  # (birth mask, survive mask) over counts 0..8


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) if missing or stale."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or any(os.path.getmtime(_LIB_PATH) < os.path.getmtime(src) for src in _SOURCES))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp] + _SOURCES + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64
            p = ctypes.c_void_p
            lib.orc_member.argtypes = [u32, u32, p, u32, i64, i64]
            lib.orc_member.restype = ctypes.c_int
            lib.orc_member_grid.argtypes = [u32, u32, p, u32, p]
            lib.orc_lambda_many.argtypes = [u32, u32, p, u32, p, p, i64]
            lib.orc_nu_many.argtypes = [u32, u32, p, u32, p, p, i64]
            lib.orc_compact_to_box.argtypes = [u32, u32, p, u32, p, p]
            lib.orc_box_to_compact.argtypes = [u32, u32, p, u32, p, p]
            lib.orc_box_step.argtypes = [i64, p, p, p, u32, u32]
            lib.orc_box_run.argtypes = [i64, p, p, p, i64, u32, u32]
            lib.orc_splitmix64.argtypes = [u64, u64]
            lib.orc_splitmix64.restype = u64
            lib.orc_box_init.argtypes = [u32, u32, p, u32, u64, u32, p]
            lib.orc_lightcone.argtypes = [u32, u32, p, u32, u64, u32, i64, u32, u32, p, i64, p]
            lib.orc_threads.restype = ctypes.c_int
            lib.orc_box_run_nbhd.argtypes = [i64, p, p, p, i64, u32, u32, u32]
            lib.orc_heat_run.argtypes = [i64, p, p, p, i64, ctypes.c_double, u32]
            lib.orc_ising_run.argtypes = [i64, p, p, i64, u64, ctypes.c_double, u32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _tau(fractal) -> np.ndarray:
    return np.ascontiguousarray(fractal.offsets_array(), dtype=np.uint8)


def threads() -> int:
    """Number of OpenMP threads the oracle uses."""
    return int(_load().orc_threads())


def compact_shape(fractal, r: int) -> tuple:
    """(H, W) of the compact rectangle: W = k^ceil(r/2) columns, H = k^floor(r/2) rows."""
    return fractal.k ** (r // 2), fractal.k ** ((r + 1) // 2)


def member(fractal, r: int, x: int, y: int) -> bool:
    """Per-level NBB membership of one point (Sec. 3)."""
    t = _tau(fractal)
    return bool(_load().orc_member(fractal.s, fractal.k, _ptr(t), r, int(x), int(y)))


def member_grid(fractal, r: int) -> np.ndarray:
    """n x n uint8 membership grid (row y, column x)."""
    n = fractal.s ** r
    out = np.zeros((n, n), dtype=np.uint8)
    t = _tau(fractal)
    _load().orc_member_grid(fractal.s, fractal.k, _ptr(t), r, _ptr(out))
    return out


def lam(fractal, r: int, omega) -> np.ndarray:
    """lambda over linear compact indices -> (count, 2) int64 (x, y); -1 if out of range."""
    om = np.ascontiguousarray(omega, dtype=np.uint64).reshape(-1)
    xy = np.empty((om.size, 2), dtype=np.int64)
    t = _tau(fractal)
    _load().orc_lambda_many(fractal.s, fractal.k, _ptr(t), r, _ptr(om), _ptr(xy), om.size)
    return xy


def nu(fractal, r: int, xy) -> np.ndarray:
    """nu over (count, 2) expanded points -> linear compact indices; holes -> 2^64-1."""
    p = np.ascontiguousarray(xy, dtype=np.int64).reshape(-1, 2)
    om = np.empty(p.shape[0], dtype=np.uint64)
    t = _tau(fractal)
    _load().orc_nu_many(fractal.s, fractal.k, _ptr(t), r, _ptr(p), _ptr(om), p.shape[0])
    return om


def compact_to_box(fractal, r: int, compact: np.ndarray) -> np.ndarray:
    """Scatter a compact buffer (k^r bytes, row-major) into a zeroed n x n box."""
    n = fractal.s ** r
    c = np.ascontiguousarray(compact, dtype=np.uint8).reshape(-1)
    assert c.size == fractal.k ** r
    box = np.zeros((n, n), dtype=np.uint8)
    t = _tau(fractal)
    _load().orc_compact_to_box(fractal.s, fractal.k, _ptr(t), r, _ptr(c), _ptr(box))
    return box


def box_to_compact(fractal, r: int, box: np.ndarray) -> np.ndarray:
    """Gather the fractal cells of an n x n box into compact order."""
    b = np.ascontiguousarray(box, dtype=np.uint8)
    out = np.empty(fractal.k ** r, dtype=np.uint8)
    t = _tau(fractal)
    _load().orc_box_to_compact(fractal.s, fractal.k, _ptr(t), r, _ptr(b), _ptr(out))
    return out


def box_run(member_box: np.ndarray, box: np.ndarray, steps: int, rule=B3S23) -> np.ndarray:
    """`steps` synchronous B/S steps of the box automaton over fractal cells."""
    n = member_box.shape[0]
    m = np.ascontiguousarray(member_box, dtype=np.uint8)
    a = np.array(box, dtype=np.uint8, order="C", copy=True)
    b = np.empty_like(a)
    _load().orc_box_run(n, _ptr(m), _ptr(a), _ptr(b), int(steps), rule[0], rule[1])
    return a


MOORE = 0x1EF
VON_NEUMANN = 0xAA


def box_run_nbhd(member_box: np.ndarray, box: np.ndarray, steps: int, rule=B3S23,
                 nbhd: int = MOORE) -> np.ndarray:
    """box_run counting only the neighbours in `nbhd` (bit (dy+1)*3+(dx+1))."""
    n = member_box.shape[0]
    m = np.ascontiguousarray(member_box, dtype=np.uint8)
    a = np.array(box, dtype=np.uint8, order="C", copy=True)
    b = np.empty_like(a)
    _load().orc_box_run_nbhd(n, _ptr(m), _ptr(a), _ptr(b), int(steps), rule[0], rule[1], nbhd)
    return a


def heat_run(member_box: np.ndarray, u: np.ndarray, steps: int, alpha: float,
             nbhd: int = VON_NEUMANN) -> np.ndarray:
    """Explicit heat steps on the fractal graph in fp64 (n x n box, holes 0)."""
    n = member_box.shape[0]
    m = np.ascontiguousarray(member_box, dtype=np.uint8)
    a = np.array(u, dtype=np.float64, order="C", copy=True)
    b = np.empty_like(a)
    _load().orc_heat_run(n, _ptr(m), _ptr(a), _ptr(b), int(steps), float(alpha), nbhd)
    return a


def ising_run(member_box: np.ndarray, box: np.ndarray, sweeps: int, seed: int,
              temperature: float, nbhd: int = VON_NEUMANN) -> np.ndarray:
    """Checkerboard Metropolis sweeps of Ising spins (bit 0 = up) on the fractal graph."""
    n = member_box.shape[0]
    m = np.ascontiguousarray(member_box, dtype=np.uint8)
    a = np.array(box, dtype=np.uint8, order="C", copy=True)
    _load().orc_ising_run(n, _ptr(m), _ptr(a), int(sweeps), seed & (2**64 - 1),
                          float(temperature), nbhd)
    return a


def splitmix64(seed: int, i: int) -> int:
    """Output number i of the SplitMix64 stream seeded with `seed`."""
    return int(_load().orc_splitmix64(seed & (2**64 - 1), i & (2**64 - 1)))


def box_init(fractal, r: int, seed: int, p_q24: int) -> np.ndarray:
    """Bernoulli initial box: fractal cell (x, y) alive iff SplitMix64 draw < p."""
    n = fractal.s ** r
    box = np.zeros((n, n), dtype=np.uint8)
    t = _tau(fractal)
    _load().orc_box_init(fractal.s, fractal.k, _ptr(t), r, seed, p_q24, _ptr(box))
    return box


def compact_init(fractal, r: int, seed: int, p_q24: int) -> np.ndarray:
    """The Bernoulli initial state in compact order."""
    return box_to_compact(fractal, r, box_init(fractal, r, seed, p_q24))


def run_compact(fractal, r: int, compact0: np.ndarray, steps: int, rule=B3S23) -> np.ndarray:
    """Expand a compact state into the box, run `steps` box steps, compact it again."""
    m = member_grid(fractal, r)
    box = compact_to_box(fractal, r, compact0)
    return box_to_compact(fractal, r, box_run(m, box, steps, rule))


def lightcone(fractal, r: int, seed: int, p_q24: int, steps: int, xy, rule=B3S23) -> np.ndarray:
    """State after `steps` steps at each fractal cell of xy, from the Bernoulli start."""
    p = np.ascontiguousarray(xy, dtype=np.int64).reshape(-1, 2)
    out = np.empty(p.shape[0], dtype=np.uint8)
    t = _tau(fractal)
    _load().orc_lightcone(fractal.s, fractal.k, _ptr(t), r, seed, p_q24, int(steps),
                          rule[0], rule[1], _ptr(p), p.shape[0], _ptr(out))
    return out


def state_bytes(fractal, r: int, rho: int = 1, cell_bytes: int = 1) -> int:
    """Bytes of one compact state buffer (Sec. 3.1, Sec. 3.5).

    At thread level (rho = 1) the compact rectangle holds k^r cells.  With
    block-level compaction each rho x rho block is one coarse cell of a level
    r_b = r - log_s(rho) fractal and stores its rho^2 expanded cells, holes
    included, so the buffer holds k^(r_b) * rho^2 cells.
    """
    rb = r
    side = 1
    while side < rho:
        side *= fractal.s
        rb -= 1
    if side != rho or rb < 0:
        raise ValueError("rho must be a power of s no larger than s^r")
    return fractal.k ** rb * rho * rho * cell_bytes


def box_bytes(fractal, r: int, cell_bytes: int = 1) -> int:
    """Bytes of the expanded n x n bounding box, n = s^r."""
    return (fractal.s ** r) ** 2 * cell_bytes
