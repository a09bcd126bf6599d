"""FP64 CPU oracle for GP-SPCA (test infrastructure, not product code).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never calls it, and it imports nothing from the CUDA library.
"""

from .gpower import (  # noqa: F401
    FORMS,
    STATUS_CONVERGED,
    STATUS_MAXIT,
    STATUS_ZERO,
    STATUS_DEGENERATE,
    OracleResult,
    column_norms,
    gamma_from_rho,
    objective_parts,
    gradient_direction,
    loadings,
    polar,
    initial_iterate,
    project_start,
    block_start,
    sketch_signs,
    splitmix64,
    POWER_STEPS,
    gpower,
)
from .deflation import gpower_deflated  # noqa: F401,E402
from .projection import project  # noqa: F401,E402
