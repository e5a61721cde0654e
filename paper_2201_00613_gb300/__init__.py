"""GB300-native compact-fractal cellular automaton (Squeeze, arXiv 2201.00613).

The compute path is the CUDA library ``libsqueeze.so`` (C ABI in
``include/squeeze.h``); ``paper_2201_00613_gb300._lib`` is its ctypes binding
with the same entry-point names.  ``inputs`` holds the seeded synthetic inputs.
"""
from ._lib import *  # noqa: F401,F403
from ._lib import Handle, Handle3, SqueezeError, exported_names, lib, library_path  # noqa: F401
