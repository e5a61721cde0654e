"""Plain CPU oracle for three-dimensional NBB fractals (test infrastructure).

Wraps ``nbb3d_oracle.c`` (linked into the oracle library) through ctypes.  The
paper (arXiv 2201.00613, abstract and Sec. 7) names the extension to three
dimensions without defining it; reading R15 at the top of the C file carries
Secs. 3.1-3.4 and 4 over to a third axis: offsets tau in [0, s)^3, the levels
cycling over the compact axes x, y, z, the 26-cell Moore neighbourhood by
default, and the initial state keyed by the compact index.
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import _load, _ptr

MOORE3 = ((1 << 27) - 1) & ~(1 << 13)          # all 26 offsets
VON_NEUMANN3 = ((1 << 4) | (1 << 10) | (1 << 12) | (1 << 14) | (1 << 16) | (1 << 22))
LIFE_4555 = (1 << 5, (1 << 4) | (1 << 5))      # B5/S45 (Bays' three-dimensional Life)

_lock = threading.Lock()
_ready = False


def _lib():
    global _ready
    lib = _load()
    with _lock:
        if not _ready:
            u32, u64, i64, p = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p
            lib.o3_extents.argtypes = [u32, u32, p, p, p]
            lib.o3_member.argtypes = [u32, u32, p, u32, i64, i64, i64]
            lib.o3_member.restype = ctypes.c_int
            lib.o3_member_grid.argtypes = [u32, u32, p, u32, p]
            lib.o3_lambda_many.argtypes = [u32, u32, p, u32, p, p, i64]
            lib.o3_nu_many.argtypes = [u32, u32, p, u32, p, p, i64]
            lib.o3_compact_to_box.argtypes = [u32, u32, p, u32, p, p]
            lib.o3_box_to_compact.argtypes = [u32, u32, p, u32, p, p]
            lib.o3_box_step.argtypes = [i64, p, p, p, u32, u32, u32]
            lib.o3_box_run.argtypes = [i64, p, p, p, i64, u32, u32, u32]
            lib.o3_init_compact.argtypes = [u64, u32, i64, p]
            lib.o3_lightcone.argtypes = [u32, u32, p, u32, u64, u32, i64, u32, u32, u32, p, i64, p]
            _ready = True
    return lib


def _tau(fractal) -> np.ndarray:
    return np.ascontiguousarray(fractal.offsets_array(), dtype=np.uint8)


def extents(fractal, r: int) -> tuple:
    """(W_x, W_y, W_z) of the compact box (R15b)."""
    v = [ctypes.c_uint64() for _ in range(3)]
    _lib().o3_extents(fractal.k, r, *[ctypes.byref(x) for x in v])
    return tuple(int(x.value) for x in v)


def member(fractal, r: int, x: int, y: int, z: int) -> bool:
    t = _tau(fractal)
    return bool(_lib().o3_member(fractal.s, fractal.k, _ptr(t), r, int(x), int(y), int(z)))


def member_grid(fractal, r: int) -> np.ndarray:
    """n x n x n uint8 membership box, indexed [z, y, x]."""
    n = fractal.s ** r
    out = np.zeros((n, n, n), dtype=np.uint8)
    t = _tau(fractal)
    _lib().o3_member_grid(fractal.s, fractal.k, _ptr(t), r, _ptr(out))
    return out


def lam(fractal, r: int, omega) -> np.ndarray:
    """lambda over compact indices -> (count, 3) int64 (x, y, z); -1s past the end."""
    om = np.ascontiguousarray(omega, dtype=np.uint64).reshape(-1)
    xyz = np.empty((om.size, 3), dtype=np.int64)
    t = _tau(fractal)
    _lib().o3_lambda_many(fractal.s, fractal.k, _ptr(t), r, _ptr(om), _ptr(xyz), om.size)
    return xyz


def nu(fractal, r: int, xyz) -> np.ndarray:
    """nu over (count, 3) points -> compact indices; holes and off-box -> 2^64-1."""
    p = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3)
    om = np.empty(p.shape[0], dtype=np.uint64)
    t = _tau(fractal)
    _lib().o3_nu_many(fractal.s, fractal.k, _ptr(t), r, _ptr(p), _ptr(om), p.shape[0])
    return om


def compact_to_box(fractal, r: int, compact) -> np.ndarray:
    n = fractal.s ** r
    c = np.ascontiguousarray(compact, dtype=np.uint8).reshape(-1)
    assert c.size == fractal.k ** r
    box = np.zeros((n, n, n), dtype=np.uint8)
    t = _tau(fractal)
    _lib().o3_compact_to_box(fractal.s, fractal.k, _ptr(t), r, _ptr(c), _ptr(box))
    return box


def box_to_compact(fractal, r: int, box) -> np.ndarray:
    b = np.ascontiguousarray(box, dtype=np.uint8)
    out = np.empty(fractal.k ** r, dtype=np.uint8)
    t = _tau(fractal)
    _lib().o3_box_to_compact(fractal.s, fractal.k, _ptr(t), r, _ptr(b), _ptr(out))
    return out


def box_run(member_box, box, steps: int, rule=LIFE_4555, nbhd: int = MOORE3) -> np.ndarray:
    """`steps` synchronous steps of the box automaton over fractal cells (R15d)."""
    n = member_box.shape[0]
    m = np.ascontiguousarray(member_box, dtype=np.uint8)
    a = np.array(box, dtype=np.uint8, order="C", copy=True)
    b = np.empty_like(a)
    _lib().o3_box_run(n, _ptr(m), _ptr(a), _ptr(b), int(steps), rule[0], rule[1], nbhd)
    return a


def init_compact(fractal, r: int, seed: int, p_q24: int) -> np.ndarray:
    """The Bernoulli start in compact order (R15e)."""
    cells = fractal.k ** r
    out = np.empty(cells, dtype=np.uint8)
    _lib().o3_init_compact(seed & (2**64 - 1), p_q24, cells, _ptr(out))
    return out


def run_compact(fractal, r: int, compact0, steps: int, rule=LIFE_4555,
                nbhd: int = MOORE3) -> np.ndarray:
    """Expand a compact state into the box, run `steps` steps, compact it again."""
    m = member_grid(fractal, r)
    box = compact_to_box(fractal, r, compact0)
    return box_to_compact(fractal, r, box_run(m, box, steps, rule, nbhd))


def lightcone(fractal, r: int, seed: int, p_q24: int, steps: int, xyz, rule=LIFE_4555,
              nbhd: int = MOORE3) -> np.ndarray:
    """State after `steps` steps at each sample cell, from the Bernoulli start."""
    p = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3)
    out = np.empty(p.shape[0], dtype=np.uint8)
    t = _tau(fractal)
    _lib().o3_lightcone(fractal.s, fractal.k, _ptr(t), r, seed & (2**64 - 1), p_q24, int(steps),
                        rule[0], rule[1], nbhd, _ptr(p), p.shape[0], _ptr(out))
    return out
