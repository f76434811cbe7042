"""FP64 CPU oracle for ACCORD-FBS.

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package smoke check and
by the benchmark's CPU-baseline leg.  The CUDA library never uses it.
"""
from . import accord_ref  # noqa: F401
