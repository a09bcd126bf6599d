"""Plain FP64 NumPy implementation of the generalized power method for sparse PCA.

TEST INFRASTRUCTURE ONLY.  This module is the parity oracle for the CUDA
library: it is slow on purpose, works in float64 throughout, and shares no code,
constants or helpers with the GPU path.  Only ``tests/``, the smoke check in
``__graft_entry__`` and the CPU-baseline legs of ``bench.py`` may use it.

What it computes (paper: "Large-Scale Paralleled Sparse Principal Component
Analysis", Section 2 and Table 1):

* ``A`` is p x n (p samples of n variables); ``a_i`` is its i-th column.
* Four formulations (Table 1, right column "Reformulation"):

  - SL1:  max_{x in S^p}  sum_i [ |a_i^T x| - gamma ]_+^2
  - SL0:  max_{x in S^p}  sum_i [ (a_i^T x)^2 - gamma ]_+
  - BL1:  max_{X in S^p_m} sum_j sum_i [ mu_j |a_i^T x_j| - gamma_j ]_+^2
  - BL0:  max_{X in S^p_m} sum_j sum_i [ (mu_j a_i^T x_j)^2 - gamma_j ]_+

* Each objective is convex in x (resp. X) and is maximised over the unit
  sphere (m = 1) or the Stiefel manifold (m > 1), Section 2.  The paper does
  not print the iteration; it names the generalized power method of its
  reference [9].  For a convex f the power step
  x+ = argmax_{x feasible} <grad f(x_k), x> never decreases f, and over the
  sphere that argmax is grad/||grad||, over the Stiefel manifold the polar
  factor of grad.  This module runs exactly that step.

Readings taken where the paper is silent or garbled (each is also listed in
the project's design notes):

* BL1: the Table 1 row labels the left side phi^2 but prints the summand
  unsquared; the summand is read as squared, which is the only reading that
  reduces to SL1 for m = 1, mu = 1.
* BL0: the row prints ``(mu_j a_i^T x)^2`` without the index on x; read x_j.
* Stiefel manifold printed as a subset of R^{n x m}; read R^{p x m}.
* gamma is absolute here; ``gamma_from_rho`` converts the paper's unitless
  values, read as relative to max_i ||a_i|| (L1) and its square (L0).
* Initialisation: single-unit x0 = a_{i*}/||a_{i*}|| with i* the first index of
  the largest column norm.  Block: a PCA start, X0 = the Rayleigh-Ritz
  vectors of A A^T on the subspace reached by two block power steps from a
  fixed Rademacher sketch (``block_start``); the m largest columns are a poor
  start (on planted spikes they all come from the strongest spike and the
  iteration stalls in degenerate local maxima).
* Stopping: after computing f_k, stop if f_k == 0 (status ZERO), else if k > 0
  and |f_k - f_{k-1}| < tol * f_{k-1} (CONVERGED), else if k == maxit - 1
  (MAXIT).  The returned iterate is x_k, the one that produced f_k.
* A threshold tie (|t| == gamma, t^2 == gamma) is inactive (strict >), and
  sign(0) = 0.
* Block polar step: if lambda_min(Y^T Y) <= 1e-12 * lambda_max(Y^T Y) the
  solve stops with status DEGENERATE and keeps the last valid X.
* The gamma path: single-unit forms accept m gamma values and run m
  independent solves that start from the same x0.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

FORMS = ("SL1", "SL0", "BL1", "BL0")

STATUS_CONVERGED = 0
STATUS_MAXIT = 1
STATUS_ZERO = 2
STATUS_DEGENERATE = 3

# lambda_min / lambda_max at or below this makes the polar factor degenerate.
DEGENERATE_RATIO = 1e-12


def _check_form(form: str) -> None:
    if form not in FORMS:
        raise ValueError(f"unknown formulation {form!r}; expected one of {FORMS}")


def _is_l1(form: str) -> bool:
    return form in ("SL1", "BL1")


def _is_block(form: str) -> bool:
    return form in ("BL1", "BL0")


def column_norms(A: np.ndarray) -> np.ndarray:
    """c_i = ||a_i||_2 for every column a_i of A (Section 2 notation)."""
    return np.linalg.norm(np.asarray(A, dtype=np.float64), axis=0)


def gamma_from_rho(A: np.ndarray, form: str, rho) -> np.ndarray:
    """Absolute gamma from the paper's unitless sparsity parameter.

    Section 4.1 quotes gamma in {0.01, 0.05} without units.  Read as relative:
    gamma = rho * max_i ||a_i|| for the L1 forms and (rho * max_i ||a_i||)^2
    for the L0 forms, which puts gamma on the scale of |a_i^T x| resp.
    (a_i^T x)^2 in Table 1.
    """
    _check_form(form)
    cmax = float(column_norms(A).max())
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    if _is_l1(form):
        return rho * cmax
    return (rho * cmax) ** 2


def objective_parts(form: str, T: np.ndarray, gamma: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Per-component objective f_j of Table 1 (right column), T = A^T X.

    L1 forms: f_j = sum_i [mu_j |t_ij| - gamma_j]_+^2   (SL1: mu_j = 1)
    L0 forms: f_j = sum_i [(mu_j t_ij)^2 - gamma_j]_+    (SL0: mu_j = 1)
    """
    if _is_l1(form):
        s = np.maximum(mu * np.abs(T) - gamma, 0.0)
        return np.sum(s * s, axis=0)
    s = np.maximum((mu * T) ** 2 - gamma, 0.0)
    return np.sum(s, axis=0)


def gradient_direction(form: str, T: np.ndarray, gamma: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """G such that the gradient of f at X is 2 A G: the power step's input.

    Differentiating the Table 1 summands with respect to x_j:
      L1: d/dx_j [mu_j|a_i^T x_j| - gamma_j]_+^2
            = 2 mu_j sign(t_ij) [mu_j|t_ij| - gamma_j]_+ a_i
      L0: d/dx_j [(mu_j a_i^T x_j)^2 - gamma_j]_+
            = 2 mu_j^2 t_ij 1[(mu_j t_ij)^2 > gamma_j] a_i
    The common factor 2 does not change the normalised or polar step.
    """
    if _is_l1(form):
        return mu * np.sign(T) * np.maximum(mu * np.abs(T) - gamma, 0.0)
    return (mu * mu) * T * ((mu * T) ** 2 > gamma)


def loadings(form: str, T: np.ndarray, gamma: np.ndarray, mu: np.ndarray) -> np.ndarray:
    """Sparse loadings Z (Table 1, left column "Original form") for fixed X.

    For fixed x (resp. X) the original-form problems over z in B^n (resp.
    Z in [S^n]^m) are maximised by
      L1: z_ij proportional to sign(t_ij) [mu_j |t_ij| - gamma_j]_+
      L0: z_ij proportional to mu_j t_ij 1[(mu_j t_ij)^2 > gamma_j]
    with each column scaled to unit norm; an all-zero column stays zero.
    """
    if _is_l1(form):
        Zr = np.sign(T) * np.maximum(mu * np.abs(T) - gamma, 0.0)
    else:
        Zr = mu * T * ((mu * T) ** 2 > gamma)
    norms = np.linalg.norm(Zr, axis=0)
    Z = np.zeros_like(Zr)
    nz = norms > 0
    Z[:, nz] = Zr[:, nz] / norms[nz]
    return Z


def polar(Y: np.ndarray):
    """Polar factor of Y (p x m): the maximiser of Tr(X^T Y) over X^T X = I.

    Computed as U V^T from the thin SVD Y = U S V^T, which equals
    Y (Y^T Y)^{-1/2}.  Returns (X, degenerate) where degenerate means
    lambda_min(Y^T Y) <= 1e-12 lambda_max(Y^T Y), i.e. s_min^2 <= 1e-12 s_max^2.
    """
    U, s, Vt = np.linalg.svd(Y, full_matrices=False)
    smax2 = float(s[0] ** 2) if s.size else 0.0
    smin2 = float(s[-1] ** 2) if s.size else 0.0
    degenerate = (smax2 == 0.0) or (smin2 <= DEGENERATE_RATIO * smax2)
    return U @ Vt, degenerate


# SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
# generators", OOPSLA 2014): the k-th output (k = 1, 2, ...) of the stream with
# seed s is mix(s + k * GOLDEN).
_GOLDEN = 0x9E3779B97F4A7C15
_MIX1 = 0xBF58476D1CE4E5B9
_MIX2 = 0x94D049BB133111EB
SKETCH_SEED = 0x5EED5EED5EED5EED
POWER_STEPS = 2


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """k-th SplitMix64 output of the stream seeded with ``seed`` (uint64 arrays)."""
    k = np.asarray(k, dtype=np.uint64)
    z = np.uint64(seed) + k * np.uint64(_GOLDEN)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(_MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(_MIX2)
    return z ^ (z >> np.uint64(31))


def sketch_signs(p: int, m: int) -> np.ndarray:
    """p x m Rademacher sketch: entry (r, j) is -1 if the top bit of output
    k = j * 2^32 + r + 1 of SplitMix64(SKETCH_SEED) is set, else +1."""
    r = np.arange(p, dtype=np.uint64)[:, None]
    j = np.arange(m, dtype=np.uint64)[None, :]
    z = splitmix64(SKETCH_SEED, (j << np.uint64(32)) + r + np.uint64(1))
    return np.where((z >> np.uint64(63)) == np.uint64(1), -1.0, 1.0)


def block_start(A: np.ndarray, m: int, steps: int = POWER_STEPS):
    """PCA start for the block forms (reading of an unstated detail).

    Q_0 = polar(Omega) for the Rademacher sketch Omega; Q_{s+1} = polar(A A^T Q_s)
    for s < steps; then Rayleigh-Ritz on span(Q): B = sym(Q^T A A^T Q),
    B = V diag(w) V^T with w in decreasing order and each column of V signed
    so that its largest-magnitude entry (first on ties) is positive;
    X0 = Q V.  Returns (X0, status) like ``initial_iterate``.
    """
    p = A.shape[0]
    Q, degenerate = polar(sketch_signs(p, m))
    if degenerate:
        return np.zeros((p, m)), STATUS_DEGENERATE
    for _ in range(steps):
        Q, degenerate = polar(A @ (A.T @ Q))
        if degenerate:
            return np.zeros((p, m)), STATUS_DEGENERATE
    B = Q.T @ (A @ (A.T @ Q))
    B = 0.5 * (B + B.T)
    w, V = np.linalg.eigh(B)
    V = V[:, ::-1]
    for j in range(m):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            V[:, j] = -V[:, j]
    return Q @ V, None


def initial_iterate(A: np.ndarray, form: str, m: int):
    """Starting point (reading of an unstated detail, see module docstring).

    Returns (X0 p x m, status) where status is None when X0 is usable, or
    STATUS_ZERO (A == 0) / STATUS_DEGENERATE (block, a rank-deficient step of
    ``block_start``).
    """
    c = column_norms(A)
    p = A.shape[0]
    if c.size == 0 or float(c.max()) == 0.0:
        return np.zeros((p, m)), STATUS_ZERO
    if not _is_block(form):
        i_star = int(np.argmax(c))  # first index attaining the maximum
        x0 = A[:, i_star] / c[i_star]
        return np.repeat(x0[:, None], m, axis=1), None
    return block_start(A, m)


def project_start(x0: np.ndarray, form: str):
    """A caller's starting iterate, projected on the feasible set: columns
    normalised (sphere, single-unit) or the polar factor (Stiefel, block).
    Returns (X0, status) like ``initial_iterate``."""
    p, m = x0.shape
    if _is_block(form):
        X0, degenerate = polar(x0)
        if degenerate:
            return np.zeros((p, m)), STATUS_DEGENERATE
        return X0, None
    norms = np.linalg.norm(x0, axis=0)
    if np.any(norms == 0):
        return np.zeros((p, m)), STATUS_DEGENERATE
    return x0 / norms, None


@dataclass
class OracleResult:
    """Outcome of one oracle call.

    X: p x m iterate that produced the returned objective.
    Z: n x m unit-norm (or zero) loadings; support = Z != 0.
    objective: length-m; per gamma for single-unit forms, per component f_j
      for block forms (the block objective is its sum, ``total``).
    iters: length-m number of sweeps t = A^T x performed (block: same value).
    status: length-m termination reason (STATUS_*).
    history: per solve (single-unit: per gamma; block: one list) the objective
      after each sweep, for the monotone-ascent check.
    gamma: the absolute gamma values used.
    """

    X: np.ndarray
    Z: np.ndarray
    objective: np.ndarray
    iters: np.ndarray
    status: np.ndarray
    gamma: np.ndarray
    mu: np.ndarray
    history: List[List[float]] = field(default_factory=list)
    T: Optional[np.ndarray] = None

    @property
    def support(self) -> np.ndarray:
        return self.Z != 0

    @property
    def total(self) -> float:
        return float(np.sum(self.objective))


def _stop(k: int, f: float, f_prev: Optional[float], tol: float, maxit: int):
    if f == 0.0:
        return STATUS_ZERO
    if k > 0 and abs(f - f_prev) < tol * f_prev:
        return STATUS_CONVERGED
    if k == maxit - 1:
        return STATUS_MAXIT
    return None


def _single_unit(A, form, gamma_j, x0, tol, maxit):
    """One single-unit solve (SL1 or SL0) with scalar gamma, from x0."""
    g1 = np.array([gamma_j])
    one = np.ones(1)
    x = x0.copy()
    f_prev = None
    hist: List[float] = []
    status = STATUS_MAXIT
    t = None
    k = 0
    for k in range(maxit):
        t = A.T @ x  # column sweep t_i = a_i^T x
        f = float(objective_parts(form, t[:, None], g1, one)[0])
        hist.append(f)
        st = _stop(k, f, f_prev, tol, maxit)
        if st is not None:
            status = st
            break
        g = gradient_direction(form, t[:, None], g1, one)[:, 0]
        y = A @ g  # rank update y = A g
        ny = float(np.linalg.norm(y))
        if ny == 0.0:
            status = STATUS_DEGENERATE
            break
        x = y / ny  # projection on the sphere S^p
        f_prev = f
    return x, t, hist[-1], k + 1, status, hist


def _block(A, form, gamma, mu, X0, tol, maxit):
    """One block solve (BL1 or BL0) with m components."""
    X = X0.copy()
    f_prev = None
    hist: List[float] = []
    status = STATUS_MAXIT
    T = None
    fparts = None
    k = 0
    for k in range(maxit):
        T = A.T @ X  # column sweep T = A^T X
        fparts = objective_parts(form, T, gamma, mu)
        f = float(np.sum(fparts))
        hist.append(f)
        st = _stop(k, f, f_prev, tol, maxit)
        if st is not None:
            status = st
            break
        G = gradient_direction(form, T, gamma, mu)
        Y = A @ G  # rank update Y = A G
        Xn, degenerate = polar(Y)  # projection on the Stiefel manifold
        if degenerate:
            status = STATUS_DEGENERATE
            break
        X = Xn
        f_prev = f
    return X, T, fparts, k + 1, status, hist


def gpower(A, form: str, gamma, mu=None, tol: float = 1e-6, maxit: int = 1000, x0=None) -> OracleResult:
    """Generalized power method for the four GP-SPCA formulations (Table 1).

    A: p x n array (any float dtype; converted exactly to float64).
    form: "SL1", "SL0", "BL1" or "BL0".
    gamma: m absolute sparsity parameters.  Single-unit forms: m independent
      solves (a gamma path) sharing A and x0.  Block forms: gamma_j per
      component.
    mu: block weights mu_j > 0 (default all 1); must be all 1 (or None) for
      single-unit forms.
    x0: optional p x m starting iterate, projected on the feasible set
      (``project_start``).
    """
    _check_form(form)
    A = np.asarray(A, dtype=np.float64)
    if A.ndim != 2:
        raise ValueError("A must be 2-D (p x n)")
    p, n = A.shape
    gamma = np.atleast_1d(np.asarray(gamma, dtype=np.float64))
    m = int(gamma.size)
    if m < 1:
        raise ValueError("need at least one gamma")
    if np.any(gamma < 0) or not np.all(np.isfinite(gamma)):
        raise ValueError("gamma must be finite and >= 0")
    if maxit < 1:
        raise ValueError("maxit must be >= 1")
    if mu is None:
        mu = np.ones(m)
    mu = np.atleast_1d(np.asarray(mu, dtype=np.float64))
    if mu.size != m or np.any(mu <= 0):
        raise ValueError("mu must have m entries, all > 0")
    if not _is_block(form) and np.any(mu != 1.0):
        raise ValueError("single-unit formulations take no weights (mu = 1)")
    if _is_block(form) and m > p:
        raise ValueError("block formulations need m <= p")
    if not np.all(np.isfinite(A)):
        raise ValueError("A has non-finite entries")

    X = np.zeros((p, m))
    Z = np.zeros((n, m))
    T_out = np.zeros((n, m))
    objective = np.zeros(m)
    iters = np.zeros(m, dtype=np.int64)
    status = np.zeros(m, dtype=np.int64)
    history: List[List[float]] = []

    if x0 is None:
        X0, st0 = initial_iterate(A, form, m)
    else:
        X0, st0 = project_start(np.asarray(x0, dtype=np.float64).reshape(p, m), form)
    if st0 is not None:
        status[:] = st0
        return OracleResult(X, Z, objective, iters, status, gamma, mu, history, T_out)

    if _is_block(form):
        Xb, T, fparts, k, st, hist = _block(A, form, gamma, mu, X0, tol, maxit)
        X[:] = Xb
        T_out[:] = T
        Z[:] = loadings(form, T, gamma, mu)
        objective[:] = fparts
        iters[:] = k
        status[:] = st
        history.append(hist)
    else:
        for j in range(m):
            x, t, f, k, st, hist = _single_unit(A, form, gamma[j], X0[:, j], tol, maxit)
            X[:, j] = x
            T_out[:, j] = t
            Z[:, j] = loadings(form, t[:, None], gamma[j : j + 1], np.ones(1))[:, 0]
            objective[j] = f
            iters[j] = k
            status[j] = st
            history.append(hist)
    return OracleResult(X, Z, objective, iters, status, gamma, mu, history, T_out)
