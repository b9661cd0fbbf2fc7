"""FP64 CPU oracle for the Simplex-GP lattice MVM and CG (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs import this package.  It shares no code with the CUDA library.
"""

from .oracle import (  # noqa: F401
    OracleLattice,
    MATERN32_COVERAGE,
    RBF_BINOMIAL,
    RBF_COVERAGE,
    PRECOND_SEED_XOR,
    build_oracle,
    condition_estimate,
    dense_rbf,
    elevate,
    gp_posterior,
    lanczos_quadrature,
    max_threads,
    nystrom_apply,
    nystrom_factor,
    nystrom_shifted,
    nystrom_shifted_apply,
    rademacher_sketch,
    set_threads,
    splitmix64,
    simplex,
    fourier_coverage,
    spatial_coverage,
    stencil,
)
