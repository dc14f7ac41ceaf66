"""Seeded synthetic inputs shaped like the paper's workloads.

This package draws particle sets and interaction lists only. It holds none of
the force arithmetic: both the CUDA path and the FP64 oracle read what it
produces, and neither imports the other.
"""

from .workloads import (  # noqa: F401
    plummer,
    king,
    king_profile,
    plummer_cube_mix,
    clustered_box,
    tree_groups,
    unit_vectors,
    log_pairs,
    uniform_sphere,
    morton_order,
    sample_indices,
    CONFIG_SEEDS,
)
