"""Host-side checks of the C ABI: the library builds, loads, and exports every
entry point declared in include/squeeze.h, and a plain C99 caller builds, links
and runs against it.  No GPU is needed."""
import os
import re
import subprocess

import pytest

import paper_2201_00613_gb300 as sq
from paper_2201_00613_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    text = open(os.path.join(ROOT, "include", "squeeze.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(squeeze_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (squeeze_[a-z0-9_]+)", out))
    declared = declared_entry_points()
    assert declared, "no declarations parsed"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    # the Python binding wraps exactly the declared names
    assert sorted(sq.exported_names()) == declared


def test_library_loads_and_reports_status_strings():
    assert sq.squeeze_status_string(0) == "ok"
    assert "argument" in sq.squeeze_status_string(-1)
    assert sq.squeeze_status_string(12345) == "unknown status"


@pytest.mark.parametrize("s,k,offsets,r", [
    (1, 1, [(0, 0)], 3),                    # s < 2
    (2, 5, [(0, 0)] * 5, 3),                # k > s*s
    (2, 3, [(0, 0), (1, 0), (2, 0)], 3),    # offset outside [0, s)
    (2, 3, [(0, 0), (1, 0), (1, 0)], 3),    # repeated offset
    (2, 3, [(0, 0), (1, 0), (0, 1)], 31),   # s^r > 2^30
    (17, 3, [(0, 0), (1, 0), (0, 1)], 2),   # s > 16
])
def test_create_rejects_bad_descriptors_before_touching_the_device(s, k, offsets, r):
    with pytest.raises(sq.SqueezeError) as e:
        sq.squeeze_create(s, k, offsets, r)
    assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG


def test_null_handle_is_rejected():
    with pytest.raises(sq.SqueezeError) as e:
        sq.squeeze_info(None)
    assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
    for call in (lambda: sq.squeeze_set_wait_limit(None, 0),
                 lambda: sq.squeeze_set_fault_injection(None, 0),
                 lambda: sq.squeeze_last_step_info(None),
                 lambda: sq.squeeze_record_bytes(None),
                 lambda: sq.squeeze_write_records(None, 16, 16, 0),
                 lambda: sq.squeeze_batch_states_written(None),
                 lambda: sq.squeeze_batch_create_with_records([], [])):
        with pytest.raises(sq.SqueezeError) as e:
            call()
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG
    assert "unsafe" in sq.squeeze_status_string(sq.SQUEEZE_ERR_DEVICE_UNSAFE)


@pytest.mark.parametrize("s,k,offsets,r", [
    (1, 1, [(0, 0, 0)], 3),                           # s < 2
    (9, 1, [(0, 0, 0)], 3),                           # s > 8
    (2, 9, [(0, 0, 0)] * 9, 3),                       # k > s^3
    (2, 2, [(0, 0, 0), (0, 0, 2)], 3),                # offset outside [0, s)
    (2, 2, [(1, 0, 1), (1, 0, 1)], 3),                # repeated offset
    (2, 1, [(0, 0, 0)], 31),                          # s^r > 2^30
    (3, 20, [(x, y, z) for z in range(3) for y in range(3) for x in range(3)
             if (x == 1) + (y == 1) + (z == 1) <= 1], 10),   # k^r > 2^40
])
def test_3d_create_rejects_bad_descriptors_before_touching_the_device(s, k, offsets, r):
    with pytest.raises(sq.SqueezeError) as e:
        sq.squeeze_3d_create(s, k, offsets, r)
    assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG


def test_3d_null_handle_is_rejected():
    for call in (lambda: sq.squeeze_3d_info(None), lambda: sq.squeeze_3d_set_rule(None, 0, 0),
                 lambda: sq.squeeze_3d_set_neighbourhood(None, 1)):
        with pytest.raises(sq.SqueezeError) as e:
            call()
        assert e.value.code == sq.SQUEEZE_ERR_INVALID_ARG


C_CALLER = r"""
#include <stdio.h>
#include <string.h>
#include "squeeze.h"

int main(int argc, char **argv) {
  const uint8_t tri[6] = {0, 0, 1, 0, 0, 1};
  const uint8_t bad[6] = {0, 0, 1, 0, 1, 0};           /* repeated offset */
  uint8_t state[27], back[27];
  uint64_t step = 0;
  squeeze_handle *h = 0;
  int i;
  if (argc < 2) return 90;
  if (strcmp(squeeze_status_string(SQUEEZE_ERR_IO), "ok") == 0) return 91;
  if (squeeze_create(2, 3, bad, 3, &h) != SQUEEZE_ERR_INVALID_ARG || h) return 92;
  if (squeeze_info(0, 0, 0, 0, 0) != SQUEEZE_ERR_INVALID_ARG) return 93;
  for (i = 0; i < 27; ++i) state[i] = (uint8_t)(i % 2);
  if (squeeze_checkpoint_write(2, 3, tri, 3, 42, state, argv[1]) != SQUEEZE_OK) return 94;
  if (squeeze_checkpoint_read(2, 3, tri, 3, &step, back, argv[1]) != SQUEEZE_OK) return 95;
  if (step != 42 || memcmp(state, back, 27) != 0) return 96;
  if (squeeze_checkpoint_read(2, 3, tri, 4, &step, back, argv[1]) != SQUEEZE_ERR_INVALID_ARG)
    return 97;
  printf("c caller ok\n");
  return 0;
}
"""


def test_c_caller_compiles_links_and_runs_without_a_gpu(tmp_path):
    """The header is plain C99; a C program linked against the library calls
    entry points that need no GPU (status text, argument errors, checkpoints)."""
    path = build.build()
    src = tmp_path / "caller.c"
    src.write_text(C_CALLER)
    exe = tmp_path / "caller"
    libdir = os.path.dirname(path)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                    "-L", libdir, "-lsqueeze", "-Wl,-rpath," + libdir], check=True)
    res = subprocess.run([str(exe), str(tmp_path / "c.ckpt")], capture_output=True, text=True)
    assert res.returncode == 0, (res.returncode, res.stderr)
    assert "c caller ok" in res.stdout
