"""FP64 CPU oracle for SIVF spherical k-means.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg. The product path (the CUDA library and its
binding) never imports this package.

Parity of every function here is pinned by tests/test_oracle_pins.py (brute
force on tiny inputs, closed forms, the ICP invariant, monotone objective).
"""
from .sivf_oracle import Oracle, AssignStats, UpdateStats, build_library  # noqa: F401
