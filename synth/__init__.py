"""Seeded synthetic workloads for the ACCORD-FBS solver.

This package only draws random inputs (precision matrices and Gaussian data
with a given precision).  It holds none of the estimator's arithmetic, so both
the CUDA library's tests and the CPU oracle's tests can consume it without
sharing any of the method's code.
"""

from .generators import (  # noqa: F401
    Workload,
    ar1_precision,
    ba_tree_precision,
    hub_block_precision,
    er_precision,
    sample_gaussian,
    orthogonal_design,
    workload,
    PathWorkload,
    path_workload,
    DiffWorkload,
    diff_workload,
    ar1_random_precision,
    WORKLOADS,
)
