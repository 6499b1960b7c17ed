"""FP64 CPU oracle of the coupled LBM cathode step (test infrastructure).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The product path never does.
"""
from .oracle import Oracle, TangentOracle, build_oracle, build_tangent, lib  # noqa: F401
