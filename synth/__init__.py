"""Seeded synthetic inputs shaped like the paper's workloads.

This package only draws inputs (baseline coordinates, visibility values,
weights, model images).  It holds none of the gridding method's arithmetic, so
both the FP64 oracle and the CUDA path can consume the same arrays.
"""
from .workloads import (  # noqa: F401
    Workload,
    SEED_BASE,
    small_disk,
    meerkat_like,
    point_source_model,
    wstack_layers,
    random_case,
    WORKLOADS,
)
