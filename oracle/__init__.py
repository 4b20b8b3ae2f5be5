"""CPU oracle of the discrete Cosserat-rod step (plain C, FP64), with a ctypes wrapper.

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke`` and by the
benchmark's CPU-baseline leg.  The product package never imports it.
"""
from .oracle import Oracle, build_oracle, oracle_library_path  # noqa: F401
