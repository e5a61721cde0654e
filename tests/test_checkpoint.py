"""Checkpoint and resume of a compact state (squeeze_checkpoint_write / _read).

The file functions are host code, so everything but the last test runs without
a GPU: the round trip, the header layout, the FNV-1a hashes (the state's
against published test vectors), rejection of another fractal or level
(INVALID_ARG) and of a damaged, truncated, over-long or foreign file (IO), any
single damaged byte, and atomic replacement.
The GPU test checks that a run stopped halfway, written out, read back and
resumed ends bit for bit where the uninterrupted run ends.
"""
import os
import struct

import numpy as np
import pytest

import paper_2201_00613_gb300 as sq
from paper_2201_00613_gb300 import inputs as I


def fnv1a64(data: bytes) -> int:
    """FNV-1a, 64-bit (Fowler, Noll, Vo), written out for the test."""
    h = 0xCBF29CE484222325
    for b in data:
        h = ((h ^ b) * 0x100000001B3) & (2 ** 64 - 1)
    return h


def write(f, r, step, state, path):
    sq.squeeze_checkpoint_write(f.s, f.k, f.offsets, r, step, state, path)


def read(f, r, path):
    out = np.full(f.k ** r, 0xEE, dtype=np.uint8)
    step = sq.squeeze_checkpoint_read(f.s, f.k, f.offsets, r, out, path)
    return step, out


def code_of(call):
    with pytest.raises(sq.SqueezeError) as e:
        call()
    return e.value.code


def test_round_trip_and_header_layout(tmp_path):
    f, r = I.TRIANGLE, 7
    state = I.bernoulli_bytes(3, f.k ** r, 0.5)
    path = str(tmp_path / "tri7.ckpt")
    write(f, r, 12345, state, path)
    step, back = read(f, r, path)
    assert step == 12345 and np.array_equal(back, state)
    raw = open(path, "rb").read()
    magic, version, hbytes, s, k, rr, dims, st, nbytes, shash, hhash = struct.unpack(
        "<8sIIIIIIQQQQ", raw[:64])
    assert (magic, version, hbytes, s, k, rr, dims) == (b"SQZSTATE", 1, 72, 2, 3, 7, 2)
    assert (st, nbytes) == (12345, 3 ** 7)
    assert raw[64:72] == bytes([0, 0, 1, 0, 0, 1, 0, 0])        # offsets, zero-padded
    assert len(raw) == 72 + 3 ** 7 and raw[72:] == state.tobytes()
    assert shash == fnv1a64(state.tobytes())
    assert hhash == fnv1a64(raw[:56] + bytes(8) + raw[64:72])   # header (this word as 0), offsets
    assert not [p for p in os.listdir(tmp_path) if ".tmp" in p]


@pytest.mark.parametrize("f,r,data,want", [
    (I.SINGLE, 0, b"a", 0xAF63DC4C8601EC8C),
    (I.Fractal("six", 3, 6, ((0, 0), (1, 0), (2, 0), (0, 1), (1, 1), (2, 1))), 1, b"foobar",
     0x85944171F73967E8),
], ids=["a", "foobar"])
def test_state_hash_is_fnv1a_64(tmp_path, f, r, data, want):
    # published FNV-1a 64-bit test vectors
    path = str(tmp_path / "h.ckpt")
    write(f, r, 0, np.frombuffer(data, dtype=np.uint8).copy(), path)
    assert struct.unpack("<Q", open(path, "rb").read()[48:56])[0] == want


def test_another_fractal_or_level_is_an_argument_error(tmp_path):
    f, r = I.TRIANGLE, 5
    path = str(tmp_path / "t.ckpt")
    write(f, r, 1, np.ones(f.k ** r, dtype=np.uint8), path)
    assert code_of(lambda: read(I.TRIANGLE, 6, path)) == sq.SQUEEZE_ERR_INVALID_ARG
    assert code_of(lambda: read(I.TRIANGLE_PAPER, 5, path)) == sq.SQUEEZE_ERR_INVALID_ARG
    assert code_of(lambda: read(I.Fractal("t", 2, 3, ((1, 0), (0, 0), (0, 1))), 5, path)) \
        == sq.SQUEEZE_ERR_INVALID_ARG                       # same cells, other replica order
    assert code_of(lambda: read(I.FULL2, 5, path)) == sq.SQUEEZE_ERR_INVALID_ARG


@pytest.mark.parametrize("damage", ["flip", "truncate", "append", "magic", "version", "garbage",
                                    "missing", "empty", "step", "offsets", "state_hash"])
def test_damaged_files_are_io_errors(tmp_path, damage):
    f, r = I.CARPET, 3
    path = str(tmp_path / "c.ckpt")
    write(f, r, 7, I.bernoulli_bytes(4, f.k ** r, 0.5), path)
    raw = bytearray(open(path, "rb").read())
    if damage == "flip":
        raw[-100] ^= 1
    elif damage == "truncate":
        raw = raw[:-1]
    elif damage == "append":
        raw += b"\0"
    elif damage == "magic":
        raw[0:8] = b"SQZSTATF"
    elif damage == "version":
        raw[8] = 2
    elif damage == "garbage":
        raw = bytearray(b"not a checkpoint at all")
    elif damage == "empty":
        raw = bytearray()
    elif damage == "step":
        raw[32] ^= 4                     # step count 7 -> 3
    elif damage == "offsets":
        raw[64] ^= 1
    elif damage == "state_hash":
        raw[48] ^= 0x80
    if damage == "missing":
        os.remove(path)
    else:
        open(path, "wb").write(bytes(raw))
    assert code_of(lambda: read(f, r, path)) == sq.SQUEEZE_ERR_IO
    assert sq.squeeze_last_cuda_error()          # the reason is recorded


def test_any_single_damaged_byte_is_caught(tmp_path):
    f, r = I.TRIANGLE, 4
    path = str(tmp_path / "t.ckpt")
    write(f, r, 99, I.bernoulli_bytes(6, f.k ** r, 0.5), path)
    raw = open(path, "rb").read()
    rng = np.random.default_rng(0)
    for pos in sorted(set(rng.integers(0, len(raw), 200).tolist()) | {8, 12, 32, 48, 56, 64}):
        bad = bytearray(raw)
        bad[pos] ^= int(rng.integers(1, 256))
        open(path, "wb").write(bytes(bad))
        code = code_of(lambda: read(f, r, path))
        assert code in (sq.SQUEEZE_ERR_IO, sq.SQUEEZE_ERR_INVALID_ARG), (pos, code)


def test_writes_replace_atomically_and_failures_leave_nothing(tmp_path):
    f, r = I.VICSEK, 4
    path = str(tmp_path / "v.ckpt")
    a = I.bernoulli_bytes(5, f.k ** r, 0.5)
    write(f, r, 1, a, path)
    write(f, r, 2, 1 - a, path)
    step, back = read(f, r, path)
    assert step == 2 and np.array_equal(back, 1 - a)
    bad = str(tmp_path / "no_such_dir" / "v.ckpt")
    assert code_of(lambda: write(f, r, 3, a, bad)) == sq.SQUEEZE_ERR_IO
    assert sorted(os.listdir(tmp_path)) == ["v.ckpt"]
    # a bad descriptor is rejected before any file is touched
    assert code_of(lambda: sq.squeeze_checkpoint_write(2, 3, ((0, 0), (1, 0), (1, 0)), 4, 0, a,
                                                       str(tmp_path / "x"))) \
        == sq.SQUEEZE_ERR_INVALID_ARG
    assert sorted(os.listdir(tmp_path)) == ["v.ckpt"]


@pytest.mark.gpu
def test_resumed_run_equals_the_uninterrupted_run(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    dev = torch.device("cuda:0")
    f, r, half = I.TRIANGLE, 12, 15
    path = str(tmp_path / "run.ckpt")
    with sq.Handle(f, r) as h:
        a = torch.empty(h.cells, dtype=torch.uint8, device=dev)
        b = torch.empty_like(a)
        sq.squeeze_init_bernoulli(h.h, a, 9, I.p_q24(0.5))
        a0 = a.clone()
        sq.squeeze_step(h.h, a, b, 2 * half)               # uninterrupted; result in a
        want = a.cpu().numpy()
        a.copy_(a0)
        sq.squeeze_step(h.h, a, b, half)                   # odd: result in b
        write(f, r, half, b.cpu().numpy(), path)
        step, state = read(f, r, path)
        assert step == half
        c = torch.from_numpy(state).to(dev)
        d = torch.empty_like(c)
        sq.squeeze_step(h.h, c, d, 2 * half - step)        # odd again: result in d
        assert np.array_equal(d.cpu().numpy(), want)
        assert sq.squeeze_device_status(h.h) == sq.SQUEEZE_OK
