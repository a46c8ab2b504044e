"""Seeded synthetic snapshot matrices shaped like the paper's double-gyre data.

This package only *generates inputs*. It holds none of the rPOD arithmetic
(no sketch, no QR, no SVD, no projection): both the FP64 oracle and the CUDA
path read the matrices it makes, and nothing else is shared between them.
"""
from .snapshots import (  # noqa: F401
    ModeRecipe,
    mode_pairs,
    make_recipe,
    mode_matrix,
    time_matrix,
    snapshot_matrix,
    parametric_recipe,
    batched_recipes,
    steady_field,
)
