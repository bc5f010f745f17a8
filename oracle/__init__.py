"""FP64 CPU oracle for the PICsar time step (arXiv 1407.1810).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg load it.  The GPU library never imports it.
"""
from .oracle import Oracle, build_oracle, params  # noqa: F401
