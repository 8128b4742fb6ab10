"""Seeded synthetic inputs for cross-scale OMP workloads.

This package generates the inputs that both the CUDA path and the CPU
oracle consume: multi-scale dictionaries, scale links, sensing codes,
ground-truth signals and their (noisy) measurements.  It holds none of the
solver's arithmetic: no OMP, no least squares, no patch extraction and no
aggregation.  The only signal processing it does is the forward simulation
of the camera (y = Phi x + e, Sec. III-C) and the construction of the
coarse dictionaries, which in the paper come from training (Sec. III-D)
and here stand in for it.
"""

from .workloads import (  # noqa: F401
    Geometry,
    Sensing,
    TrainingSet,
    Workload,
    WORKLOAD_NAMES,
    make_workload,
    make_independent_problems,
    make_training_set,
    patch_count_1d,
)
