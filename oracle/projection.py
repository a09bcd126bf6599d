"""Scores of samples on sparse loadings.

TEST INFRASTRUCTURE ONLY (parity oracle; FP64, no code shared with the CUDA
library).

Section 4.2 learns the components on training samples, then maps every sample
into the subspace they span before classification.  With loadings Z (n x m,
the Z of a solve) and samples B (q x n, rows = samples of the same n
variables), the scores are S = B Z: column j is sum_i Z[i, j] b_i over the
columns b_i of B (only the support of z_j contributes).
"""

from __future__ import annotations

import numpy as np


def project(B, Z) -> np.ndarray:
    """S = B Z in float64 (B q x n, Z n x m)."""
    B = np.asarray(B, dtype=np.float64)
    Z = np.asarray(Z, dtype=np.float64)
    if B.ndim != 2 or Z.ndim != 2 or B.shape[1] != Z.shape[0]:
        raise ValueError("B must be q x n and Z n x m")
    return B @ Z
