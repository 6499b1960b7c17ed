"""FP64 CPU oracle of the coupled LBM cathode step (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The product path never does.
"""
from .oracle import Oracle, build_oracle, lib  # noqa: F401
