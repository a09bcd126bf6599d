"""Independent checks used to pin the oracle (and reused by the GPU tests).

Nothing here calls the oracle's arithmetic: these are the left column of
Table 1 ("Original form"), written from its own definition, so that the
reformulated objective, the threshold and the loadings the oracle computes
can be checked against it.
"""

import numpy as np


def original_single(form, A, x, z, gamma):
    """Original-form value of one single-unit solution (Table 1, left column).

    SL1: sqrt(z^T Sigma z) - gamma ||z||_1 with Sigma = A^T A, z in B^n.
    SL0: z^T Sigma z - gamma ||z||_0.
    Also returns the value with x held fixed (x^T A z in place of ||A z||),
    which equals the reformulated objective at that x for the optimal z.
    """
    Az = A @ z
    quad = float(Az @ Az)
    xAz = float(x @ Az)
    if form == "SL1":
        l1 = float(np.abs(z).sum())
        return np.sqrt(quad) - gamma * l1, xAz - gamma * l1
    l0 = float(np.count_nonzero(z))
    return quad - gamma * l0, xAz * xAz - gamma * l0


def original_block(form, A, X, Z, gamma, mu):
    """Original-form value of a block solution (Table 1, left column).

    BL1: Tr(X^T A Z N) - sum_j gamma_j ||z_j||_1
    BL0: Tr(Diag(X^T A Z N)^2) - sum_j gamma_j ||z_j||_0
    with N = Diag(mu), X on the Stiefel manifold, Z with unit (or zero) columns.
    """
    M = X.T @ A @ Z @ np.diag(mu)
    if form == "BL1":
        return float(np.trace(M)) - float(np.sum(gamma * np.abs(Z).sum(axis=0)))
    d = np.diag(M)
    return float(np.sum(d * d)) - float(np.sum(gamma * np.count_nonzero(Z, axis=0)))
