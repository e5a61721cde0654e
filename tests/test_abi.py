"""Host-side checks of the C ABI: the library builds, loads, and exports every
entry point declared in include/squeeze.h.  No GPU is needed."""
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
