"""ctypes binding of libsqueeze.so (include/squeeze.h), same names as the C ABI.

Argument marshalling only: tensors are passed as raw device/host pointers,
streams as ``cudaStream_t`` values.  Every computation runs in the library's
CUDA kernels; there is no Python or CPU fallback.  If the shared library is
missing and cannot be built, importing the binding raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

SQUEEZE_OK = 0
SQUEEZE_ERR_INVALID_ARG = -1
SQUEEZE_ERR_UNSUPPORTED = -2
SQUEEZE_ERR_OOM = -3
SQUEEZE_ERR_CUDA = -4
SQUEEZE_ERR_DEVICE_TIMEOUT = -5
SQUEEZE_ERR_DEVICE_BOUNDS = -6
SQUEEZE_ERR_IO = -7
SQUEEZE_ERR_DEVICE_UNSAFE = -8

SQUEEZE_FAULT_WITHHOLD_LOADS = 1

SQUEEZE_STEP_AUTO = 0
SQUEEZE_STEP_TILED = 1
SQUEEZE_MAP_ALU = 2
SQUEEZE_MAP_TC_BF16 = 3
SQUEEZE_MAP_TC_I8 = 4

SQUEEZE_MOORE = 0x1EF
SQUEEZE_VON_NEUMANN = 0xAA
SQUEEZE_3D_MOORE = ((1 << 27) - 1) & ~(1 << 13)
SQUEEZE_3D_VON_NEUMANN = (1 << 4) | (1 << 10) | (1 << 12) | (1 << 14) | (1 << 16) | (1 << 22)

_lock = threading.Lock()
_lib = None


class SqueezeError(RuntimeError):
    """A non-zero status returned by the library."""

    def __init__(self, code: int, where: str):
        self.code = code
        lib = _load()
        msg = lib.squeeze_status_string(code).decode()
        cuda = lib.squeeze_last_cuda_error().decode()
        super().__init__("%s: %s (%d)%s" % (where, msg, code, (" [" + cuda + "]") if cuda else ""))


_SIGS = {
    "squeeze_create": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
                        ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "squeeze_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_info": ([ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_uint64)] * 4, ctypes.c_int),
    "squeeze_set_rule": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32], ctypes.c_int),
    "squeeze_lambda": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                        ctypes.c_void_p], ctypes.c_int),
    "squeeze_nu": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                    ctypes.c_void_p], ctypes.c_int),
    "squeeze_map_tc": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                        ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "squeeze_init_bernoulli": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "squeeze_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                      ctypes.c_int, ctypes.c_void_p], ctypes.c_int),
    "squeeze_step_host": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p],
                          ctypes.c_int),
    "squeeze_tiled_level": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_set_tiled_level": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_bb_init": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32,
                         ctypes.c_void_p], ctypes.c_int),
    "squeeze_bb_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                         ctypes.c_void_p], ctypes.c_int),
    "squeeze_bb_to_compact": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p], ctypes.c_int),
    "squeeze_lambda_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                             ctypes.c_void_p], ctypes.c_int),
    "squeeze_set_neighbourhood": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_ising_sweep": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                             ctypes.c_double, ctypes.c_void_p], ctypes.c_int),
    "squeeze_heat_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                           ctypes.c_float, ctypes.c_void_p], ctypes.c_int),
    "squeeze_block_bytes": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64)],
                            ctypes.c_int),
    "squeeze_block_init": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64,
                            ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "squeeze_block_step": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_uint64, ctypes.c_void_p], ctypes.c_int),
    "squeeze_block_to_compact": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "squeeze_batch_create": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)],
                             ctypes.c_int),
    "squeeze_batch_configure": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int],
                                ctypes.c_int),
    "squeeze_batch_info": ([ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_uint32)] * 3, ctypes.c_int),
    "squeeze_batch_run": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p], ctypes.c_int),
    "squeeze_batch_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_batch_states_written": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_batch_create_with_records": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p,
                                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "squeeze_record_bytes": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "squeeze_write_records": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
                              ctypes.c_int),
    "squeeze_step_noalloc": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
                              ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.POINTER(ctypes.c_int), ctypes.c_void_p], ctypes.c_int),
    "squeeze_checkpoint_write": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                  ctypes.c_uint32, ctypes.c_uint64, ctypes.c_void_p,
                                  ctypes.c_char_p], ctypes.c_int),
    "squeeze_checkpoint_read": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p,
                                 ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.c_void_p, ctypes.c_char_p], ctypes.c_int),
    "squeeze_3d_create": ([ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint32,
                           ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "squeeze_3d_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_3d_info": ([ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_uint64)] * 5, ctypes.c_int),
    "squeeze_3d_set_rule": ([ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32], ctypes.c_int),
    "squeeze_3d_set_neighbourhood": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_3d_lambda": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                           ctypes.c_void_p], ctypes.c_int),
    "squeeze_3d_nu": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                       ctypes.c_void_p], ctypes.c_int),
    "squeeze_3d_init_bernoulli": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_void_p], ctypes.c_int),
    "squeeze_3d_step": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64,
                         ctypes.c_void_p], ctypes.c_int),
    "squeeze_3d_device_status": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "squeeze_3d_set_tiled_level": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_3d_tiled_level": ([ctypes.c_void_p], ctypes.c_int),
    "squeeze_device_status": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "squeeze_set_wait_limit": ([ctypes.c_void_p, ctypes.c_uint64], ctypes.c_int),
    "squeeze_set_max_steps_per_launch": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_set_fault_injection": ([ctypes.c_void_p, ctypes.c_uint32], ctypes.c_int),
    "squeeze_last_step_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)],
                               ctypes.c_int),
    "squeeze_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "squeeze_last_cuda_error": ([], ctypes.c_char_p),
}


def exported_names() -> list:
    """Names of every entry point the binding expects the library to export."""
    return list(_SIGS)


def library_path() -> str:
    return _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if _build.stale() else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError("libsqueeze.so is missing and could not be built")
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


def lib():
    """The loaded ctypes library."""
    return _load()


def _check(code: int, where: str):
    if code != SQUEEZE_OK:
        raise SqueezeError(code, where)


def _ptr(x):
    """Raw pointer of a torch tensor, a numpy array or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError("cannot take a pointer of %r" % type(x))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---- entry points (same names and argument order as the C ABI) ----------------

def squeeze_create(s: int, k: int, offsets, r: int):
    """Create a handle for the level-r NBB fractal; offsets = k (tau_x, tau_y) pairs."""
    flat = bytes(int(v) for pair in offsets for v in pair)
    if len(flat) != 2 * k:
        raise ValueError("need k offset pairs")
    buf = ctypes.create_string_buffer(flat, len(flat))
    out = ctypes.c_void_p()
    _check(_load().squeeze_create(s, k, buf, r, ctypes.byref(out)), "squeeze_create")
    return out.value


def squeeze_destroy(h):
    _check(_load().squeeze_destroy(h), "squeeze_destroy")


def squeeze_info(h):
    """(n_cells, width W, height H, side n)."""
    v = [ctypes.c_uint64() for _ in range(4)]
    _check(_load().squeeze_info(h, *[ctypes.byref(x) for x in v]), "squeeze_info")
    return tuple(int(x.value) for x in v)


def squeeze_set_rule(h, birth: int, survive: int):
    _check(_load().squeeze_set_rule(h, birth, survive), "squeeze_set_rule")


def squeeze_lambda(h, d_omega, d_xy, count: int, stream=None):
    _check(_load().squeeze_lambda(h, _ptr(d_omega), _ptr(d_xy), count, _stream(stream)),
           "squeeze_lambda")


def squeeze_nu(h, d_xy, d_omega, count: int, stream=None):
    _check(_load().squeeze_nu(h, _ptr(d_xy), _ptr(d_omega), count, _stream(stream)), "squeeze_nu")


def squeeze_map_tc(h, direction: int, d_in, d_out, count: int, kind: int, stream=None):
    _check(_load().squeeze_map_tc(h, direction, _ptr(d_in), _ptr(d_out), count, kind,
                                  _stream(stream)), "squeeze_map_tc")


def squeeze_init_bernoulli(h, d_state, seed: int, p_q24: int, stream=None):
    _check(_load().squeeze_init_bernoulli(h, _ptr(d_state), seed, p_q24, _stream(stream)),
           "squeeze_init_bernoulli")


def squeeze_step(h, d_buf0, d_buf1, n_steps: int, kind: int = SQUEEZE_STEP_AUTO, stream=None):
    _check(_load().squeeze_step(h, _ptr(d_buf0), _ptr(d_buf1), n_steps, kind, _stream(stream)),
           "squeeze_step")


def squeeze_step_host(h, h_in, h_out, d_buf0, d_buf1, n_steps: int,
                      kind: int = SQUEEZE_STEP_AUTO, stream=None):
    _check(_load().squeeze_step_host(h, _ptr(h_in), _ptr(h_out), _ptr(d_buf0), _ptr(d_buf1),
                                     n_steps, kind, _stream(stream)), "squeeze_step_host")


def squeeze_tiled_level(h) -> int:
    return int(_load().squeeze_tiled_level(h))


def squeeze_set_tiled_level(h, level: int):
    _check(_load().squeeze_set_tiled_level(h, level), "squeeze_set_tiled_level")


def squeeze_bb_init(h, d_grid, seed: int, p_q24: int, stream=None):
    _check(_load().squeeze_bb_init(h, _ptr(d_grid), seed, p_q24, _stream(stream)),
           "squeeze_bb_init")


def squeeze_bb_step(h, d_grid0, d_grid1, n_steps: int, stream=None):
    _check(_load().squeeze_bb_step(h, _ptr(d_grid0), _ptr(d_grid1), n_steps, _stream(stream)),
           "squeeze_bb_step")


def squeeze_block_bytes(h, b: int) -> int:
    out = ctypes.c_uint64(0)
    _check(_load().squeeze_block_bytes(h, b, ctypes.byref(out)), "squeeze_block_bytes")
    return out.value


def squeeze_block_init(h, b: int, d_blocks, seed: int, p_q24: int, stream=None):
    _check(_load().squeeze_block_init(h, b, _ptr(d_blocks), seed, p_q24, _stream(stream)),
           "squeeze_block_init")


def squeeze_block_step(h, b: int, d_blocks0, d_blocks1, n_steps: int, stream=None):
    _check(_load().squeeze_block_step(h, b, _ptr(d_blocks0), _ptr(d_blocks1), n_steps,
                                      _stream(stream)), "squeeze_block_step")


def squeeze_block_to_compact(h, b: int, d_blocks, d_state, stream=None):
    _check(_load().squeeze_block_to_compact(h, b, _ptr(d_blocks), _ptr(d_state),
                                            _stream(stream)), "squeeze_block_to_compact")


def squeeze_set_neighbourhood(h, mask: int):
    _check(_load().squeeze_set_neighbourhood(h, mask), "squeeze_set_neighbourhood")


def squeeze_ising_sweep(h, d_state, n_sweeps: int, seed: int, temperature: float, stream=None):
    _check(_load().squeeze_ising_sweep(h, _ptr(d_state), n_sweeps, seed & (2**64 - 1),
                                       temperature, _stream(stream)), "squeeze_ising_sweep")


def squeeze_heat_step(h, d_u0, d_u1, n_steps: int, alpha: float, stream=None):
    _check(_load().squeeze_heat_step(h, _ptr(d_u0), _ptr(d_u1), n_steps, alpha, _stream(stream)),
           "squeeze_heat_step")


def squeeze_lambda_step(h, d_grid0, d_grid1, n_steps: int, stream=None):
    _check(_load().squeeze_lambda_step(h, _ptr(d_grid0), _ptr(d_grid1), n_steps,
                                       _stream(stream)), "squeeze_lambda_step")


def squeeze_bb_to_compact(h, d_grid, d_state, stream=None):
    _check(_load().squeeze_bb_to_compact(h, _ptr(d_grid), _ptr(d_state), _stream(stream)),
           "squeeze_bb_to_compact")


class _BatchItem(ctypes.Structure):
    _fields_ = [("h", ctypes.c_void_p), ("d_buf0", ctypes.c_void_p), ("d_buf1", ctypes.c_void_p)]


def squeeze_batch_create(items):
    """items: sequence of (handle, d_buf0, d_buf1); returns the batch pointer."""
    arr = (_BatchItem * len(items))(*[_BatchItem(h, _ptr(a), _ptr(b)) for h, a, b in items])
    out = ctypes.c_void_p()
    _check(_load().squeeze_batch_create(ctypes.cast(arr, ctypes.c_void_p), len(items),
                                        ctypes.byref(out)), "squeeze_batch_create")
    return out.value


def squeeze_batch_create_with_records(items, records):
    """items: sequence of (handle, d_buf0, d_buf1); records: sequence of
    (d_rec0, d_rec1) per item (None where the program has no records), the
    records of d_buf0 current; returns the batch pointer."""
    arr = (_BatchItem * len(items))(*[_BatchItem(h, _ptr(a), _ptr(b)) for h, a, b in items])
    recs = (ctypes.c_void_p * (2 * len(items)))(
        *[_ptr(r) if r is not None else None for pair in records for r in pair])
    out = ctypes.c_void_p()
    _check(_load().squeeze_batch_create_with_records(ctypes.cast(arr, ctypes.c_void_p), len(items),
                                                     ctypes.cast(recs, ctypes.c_void_p),
                                                     ctypes.byref(out)),
           "squeeze_batch_create_with_records")
    return out.value


def squeeze_record_bytes(h) -> int:
    v = ctypes.c_uint64()
    _check(_load().squeeze_record_bytes(h, ctypes.byref(v)), "squeeze_record_bytes")
    return int(v.value)


def squeeze_write_records(h, d_state, d_rec, stream=None):
    _check(_load().squeeze_write_records(h, _ptr(d_state), _ptr(d_rec), _stream(stream)),
           "squeeze_write_records")


def squeeze_batch_configure(b, threads: int, ctas_per_sm: int = 0, use_graph: bool = True):
    _check(_load().squeeze_batch_configure(b, threads, ctas_per_sm, int(use_graph)),
           "squeeze_batch_configure")


def squeeze_batch_info(b):
    """(grid, threads per CTA, shared-memory bytes per CTA)."""
    v = [ctypes.c_uint32() for _ in range(3)]
    _check(_load().squeeze_batch_info(b, *[ctypes.byref(x) for x in v]), "squeeze_batch_info")
    return tuple(int(x.value) for x in v)


def squeeze_batch_run(b, n_steps: int, stream=None):
    _check(_load().squeeze_batch_run(b, n_steps, _stream(stream)), "squeeze_batch_run")


def squeeze_batch_states_written(b):
    _check(_load().squeeze_batch_states_written(b), "squeeze_batch_states_written")


def squeeze_batch_destroy(b):
    _check(_load().squeeze_batch_destroy(b), "squeeze_batch_destroy")


def squeeze_step_noalloc(s: int, k: int, offsets, r: int, birth: int, survive: int,
                         d_in, d_out, wait_status: bool = True, stream=None):
    """One tiled step that allocates no memory (see include/squeeze.h).

    Returns the device status when wait_status is true, else None.
    """
    flat = bytes(int(v) for pair in offsets for v in pair)
    buf = ctypes.create_string_buffer(flat, len(flat))
    st = ctypes.c_int(-99)
    _check(_load().squeeze_step_noalloc(s, k, buf, r, birth, survive, _ptr(d_in), _ptr(d_out),
                                        ctypes.byref(st) if wait_status else None,
                                        _stream(stream)), "squeeze_step_noalloc")
    return int(st.value) if wait_status else None


def _offsets_buffer(offsets, k: int):
    flat = bytes(int(v) for pair in offsets for v in pair)
    if len(flat) != 2 * k:
        raise ValueError("need k offset pairs")
    return ctypes.create_string_buffer(flat, len(flat))


def squeeze_checkpoint_write(s: int, k: int, offsets, r: int, step: int, h_state, path):
    """Write a host state (k^r bytes, e.g. a numpy array) and its step count to `path`."""
    _check(_load().squeeze_checkpoint_write(s, k, _offsets_buffer(offsets, k), r, step,
                                            _ptr(h_state), os.fsencode(path)),
           "squeeze_checkpoint_write")


def squeeze_checkpoint_read(s: int, k: int, offsets, r: int, h_state, path) -> int:
    """Read a checkpoint into a host buffer of k^r bytes; returns its step count."""
    step = ctypes.c_uint64(0)
    _check(_load().squeeze_checkpoint_read(s, k, _offsets_buffer(offsets, k), r,
                                           ctypes.byref(step), _ptr(h_state), os.fsencode(path)),
           "squeeze_checkpoint_read")
    return int(step.value)


def squeeze_3d_create(s: int, k: int, offsets, r: int):
    """Create a handle for the level-r 3-D NBB fractal; offsets = k (x, y, z) triples."""
    flat = bytes(int(v) for t in offsets for v in t)
    if len(flat) != 3 * k:
        raise ValueError("need k offset triples")
    buf = ctypes.create_string_buffer(flat, len(flat))
    out = ctypes.c_void_p()
    _check(_load().squeeze_3d_create(s, k, buf, r, ctypes.byref(out)), "squeeze_3d_create")
    return out.value


def squeeze_3d_destroy(h):
    _check(_load().squeeze_3d_destroy(h), "squeeze_3d_destroy")


def squeeze_3d_info(h):
    """(n_cells, W_x, W_y, W_z, side n)."""
    v = [ctypes.c_uint64() for _ in range(5)]
    _check(_load().squeeze_3d_info(h, *[ctypes.byref(x) for x in v]), "squeeze_3d_info")
    return tuple(int(x.value) for x in v)


def squeeze_3d_set_rule(h, birth: int, survive: int):
    _check(_load().squeeze_3d_set_rule(h, birth, survive), "squeeze_3d_set_rule")


def squeeze_3d_set_neighbourhood(h, mask: int):
    _check(_load().squeeze_3d_set_neighbourhood(h, mask), "squeeze_3d_set_neighbourhood")


def squeeze_3d_lambda(h, d_omega, d_xyz, count: int, stream=None):
    _check(_load().squeeze_3d_lambda(h, _ptr(d_omega), _ptr(d_xyz), count, _stream(stream)),
           "squeeze_3d_lambda")


def squeeze_3d_nu(h, d_xyz, d_omega, count: int, stream=None):
    _check(_load().squeeze_3d_nu(h, _ptr(d_xyz), _ptr(d_omega), count, _stream(stream)),
           "squeeze_3d_nu")


def squeeze_3d_init_bernoulli(h, d_state, seed: int, p_q24: int, stream=None):
    _check(_load().squeeze_3d_init_bernoulli(h, _ptr(d_state), seed & (2**64 - 1), p_q24,
                                             _stream(stream)), "squeeze_3d_init_bernoulli")


def squeeze_3d_step(h, d_buf0, d_buf1, n_steps: int, stream=None):
    _check(_load().squeeze_3d_step(h, _ptr(d_buf0), _ptr(d_buf1), n_steps, _stream(stream)),
           "squeeze_3d_step")


def squeeze_3d_set_tiled_level(h, level: int) -> None:
    _check(_load().squeeze_3d_set_tiled_level(h, level), "squeeze_3d_set_tiled_level")


def squeeze_3d_tiled_level(h) -> int:
    rc = _load().squeeze_3d_tiled_level(h)
    if rc < 0:
        raise SqueezeError(rc, "squeeze_3d_tiled_level")
    return rc


def squeeze_3d_device_status(h) -> int:
    v = ctypes.c_int()
    _check(_load().squeeze_3d_device_status(h, ctypes.byref(v)), "squeeze_3d_device_status")
    return int(v.value)


def squeeze_device_status(h) -> int:
    v = ctypes.c_int()
    _check(_load().squeeze_device_status(h, ctypes.byref(v)), "squeeze_device_status")
    return int(v.value)


def squeeze_set_max_steps_per_launch(h, steps: int) -> None:
    _check(_load().squeeze_set_max_steps_per_launch(h, steps), "squeeze_set_max_steps_per_launch")


def squeeze_set_wait_limit(h, ns: int) -> None:
    _check(_load().squeeze_set_wait_limit(h, ns), "squeeze_set_wait_limit")


def squeeze_set_fault_injection(h, flags: int) -> None:
    _check(_load().squeeze_set_fault_injection(h, flags), "squeeze_set_fault_injection")


def squeeze_last_step_info(h) -> tuple:
    """(kind, launches, [launches of 1, 2, 4 and 8 steps]) of the handle's
    last squeeze_step."""
    kind, launches = ctypes.c_int(), ctypes.c_uint64()
    by = (ctypes.c_uint64 * 4)()
    _check(_load().squeeze_last_step_info(h, ctypes.byref(kind), ctypes.byref(launches), by),
           "squeeze_last_step_info")
    return int(kind.value), int(launches.value), [int(v) for v in by]


def squeeze_status_string(code: int) -> str:
    return _load().squeeze_status_string(code).decode()


def squeeze_last_cuda_error() -> str:
    return _load().squeeze_last_cuda_error().decode()


class Handle:
    """Owns one squeeze handle; closes it on ``close()`` or at context exit."""

    def __init__(self, fractal, r: int):
        self.fractal = fractal
        self.r = r
        self.h = squeeze_create(fractal.s, fractal.k, fractal.offsets, r)
        self.cells, self.width, self.height, self.side = squeeze_info(self.h)

    def close(self):
        if self.h:
            squeeze_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Handle3:
    """Owns one 3-D squeeze handle; closes it on ``close()`` or at context exit."""

    def __init__(self, fractal, r: int):
        self.fractal = fractal
        self.r = r
        self.h = squeeze_3d_create(fractal.s, fractal.k, fractal.offsets, r)
        self.cells, self.wx, self.wy, self.wz, self.side = squeeze_3d_info(self.h)

    def close(self):
        if self.h:
            squeeze_3d_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
