"""FP64 CPU oracle for the SRTM filter/smoother (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The library under test never does.
"""
from .oracle import build, sequential, parallel, filter_op, smoother_op, lifted, loglik  # noqa: F401
