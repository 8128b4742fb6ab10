"""FP64 CPU oracle for batched plain and cross-scale OMP.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of
``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import this
package.  The product path (the CUDA library and its binding) never calls it
and shares no code with it.

Parity status of each function is recorded beside it in the tests; every
function here is pinned by a CPU test against a fact that does not come from
the oracle itself (closed forms, exhaustive search, recovery guarantees,
library least squares, invariants).
"""

from .reference import (  # noqa: F401
    EPS_D,
    EPS_R,
    U_up,
    W_down,
    aggregate,
    bayer_channel,
    children_lists,
    cross_scale_omp,
    extract_patches,
    meas_dim,
    num_threads,
    omp_batch,
    patch_grid,
    patch_origins,
    phi_apply,
    plain_omp,
    psnr,
    sensing_matrix,
    snr,
    synthesize,
)
