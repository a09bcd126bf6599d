"""Several sparse components from single-unit solves, by projection deflation.

TEST INFRASTRUCTURE ONLY (the parity oracle; same rules as ``gpower``: FP64,
slow on purpose, no code shared with the CUDA library).

The paper's efficiency experiments (Section 4.1, Fig. 3) extract several
components (m = 5) with the single-unit formulations SL1 / SL0 of Table 1 but
do not state how the components after the first are obtained.  Reading taken:
projection deflation.  With z_j the unit loading of component j (the Z column
of a single-unit solve),

    A_0 = A,    u_j = A_{j-1} z_j,    A_j = A_{j-1} - u_j z_j^T = A_{j-1} (I - z_j z_j^T),

and component j is the single-unit solve on A_{j-1} (start, stopping rule and
threshold exactly as in ``gpower``).  A_j z_j = 0, so the variance explained
by z_j is removed before the next solve; for gamma = 0 the loadings are the
right singular vectors of A in order (the deflation then removes one singular
pair at a time).  Only the columns in the support of z_j change.  A relative
gamma is taken against the largest column norm of the matrix being solved
(A_{j-1}).
"""

from __future__ import annotations

import numpy as np

from .gpower import OracleResult, _check_form, _is_block, gamma_from_rho, gpower


def gpower_deflated(A, form: str, gamma, tol: float = 1e-6, maxit: int = 1000, relative: bool = False,
                    return_deflated: bool = False):
    """Components j = 0..m-1, component j the single-unit solve with gamma[j]
    on the deflated matrix A_{j-1} (module docstring).

    Returns an ``OracleResult`` whose column j holds component j (objective[j]
    is f of component j on A_{j-1}; gamma the absolute values used; the extra
    attribute ``cnorms``, n x m, holds the column norms of each matrix solved,
    A_{j-1}), and with ``return_deflated`` also the final deflated matrix A_m.
    """
    _check_form(form)
    if _is_block(form):
        raise ValueError("deflation extracts single-unit components (SL1 or SL0)")
    Aj = np.array(A, dtype=np.float64, copy=True)
    if Aj.ndim != 2:
        raise ValueError("A must be 2-D (p x n)")
    p, n = Aj.shape
    gamma = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
    m = int(gamma.size)
    X = np.zeros((p, m))
    Z = np.zeros((n, m))
    T = np.zeros((n, m))
    objective = np.zeros(m)
    iters = np.zeros(m, dtype=np.int64)
    status = np.zeros(m, dtype=np.int64)
    gabs = np.zeros(m)
    history = []
    cnorms = np.zeros((n, m))
    for j in range(m):
        cnorms[:, j] = np.linalg.norm(Aj, axis=0)
        gj = float(gamma_from_rho(Aj, form, gamma[j])[0]) if relative else float(gamma[j])
        r = gpower(Aj, form, [gj], tol=tol, maxit=maxit)
        X[:, j] = r.X[:, 0]
        Z[:, j] = r.Z[:, 0]
        T[:, j] = r.T[:, 0]
        objective[j] = r.objective[0]
        iters[j] = r.iters[0]
        status[j] = r.status[0]
        gabs[j] = gj
        history.append(r.history[0])
        z = Z[:, j]
        u = Aj @ z  # u_j = A_{j-1} z_j
        Aj = Aj - np.outer(u, z)  # A_j = A_{j-1} (I - z_j z_j^T)
    res = OracleResult(X, Z, objective, iters, status, gabs, np.ones(m), history, T)
    res.cnorms = cnorms
    return (res, Aj) if return_deflated else res
