"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random matrices and nothing else: it holds none of the
GP-SPCA arithmetic, so both the CUDA path and the CPU oracle can take their
inputs from it.

Layout: every generator returns ``At`` of shape (n, p), C-contiguous, whose
row i is column a_i of the p x n data matrix A (p samples of n variables,
Section 2).  That is A stored column-major, the layout the C-ABI takes.

Workloads (Section 4.1 times random instances A_{PxN} with P = N/10 whose
distribution is not stated; the recognition datasets of Section 4.2 are not
available, so planted sparse spikes stand in for structured data):

* ``gaussian``: i.i.d. N(0, 1) entries, optionally with centred columns.
* ``planted_spike``: N(0,1) noise + sum_j theta_j u_j v_j^T with
  u_j ~ N(0, I_p) and v_j unit-norm on disjoint random supports with
  Rademacher entries.  Draw order: noise, then u, then supports, then signs.
"""

from __future__ import annotations

from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np


@dataclass
class SpikeMeta:
    """What was planted: supports[j] holds the indices of v_j's nonzeros."""

    theta: np.ndarray
    U: np.ndarray  # k x p
    supports: list
    signs: list


def gaussian(p: int, n: int, seed: int, dtype=np.float64, centre: bool = False) -> np.ndarray:
    """i.i.d. N(0,1) matrix, returned as At (n x p).  ``centre`` subtracts each
    column's mean (the mean over the p samples of variable i)."""
    rng = np.random.default_rng(seed)
    At = rng.standard_normal((n, p))
    if centre:
        At = At - At.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(At.astype(dtype, copy=False))


def planted_spike(
    p: int,
    n: int,
    k: int,
    theta: Sequence[float],
    support_frac: Optional[float] = None,
    support_size: Optional[int] = None,
    seed: int = 0,
    dtype=np.float32,
    with_meta: bool = False,
):
    """Planted sparse spikes: A = N(0,1) + sum_{j<k} theta_j u_j v_j^T.

    Each v_j has ``support_size`` (or round(support_frac * n)) nonzeros,
    +-1/sqrt(s), on supports that are disjoint across j.
    """
    if support_size is None:
        support_size = int(round(float(support_frac) * n))
    s = int(support_size)
    if k * s > n:
        raise ValueError("supports must be disjoint: k * s > n")
    theta = np.asarray(theta, dtype=np.float64)
    if theta.size != k:
        raise ValueError("theta must have k entries")
    rng = np.random.default_rng(seed)
    At = rng.standard_normal((n, p), dtype=np.float32)  # noise
    U = rng.standard_normal((k, p))  # u_j ~ N(0, I_p)
    perm = rng.permutation(n)[: k * s]
    supports = [np.sort(perm[j * s : (j + 1) * s]) for j in range(k)]
    signs = [rng.choice(np.array([-1.0, 1.0]), size=s) for _ in range(k)]
    for j in range(k):
        if s == 0:
            continue
        idx = supports[j]
        v = signs[j] / np.sqrt(s)
        rows = At[idx].astype(np.float64) + theta[j] * np.outer(v, U[j])
        At[idx] = rows.astype(np.float32)
    out = np.ascontiguousarray(At.astype(dtype, copy=False))
    if with_meta:
        return out, SpikeMeta(theta, U, supports, signs)
    return out


# Named workloads with their sizes (p samples x n variables).

def workload_fp64_200x1000(seed: int = 0) -> np.ndarray:
    """200 x 1000 i.i.d. N(0,1), columns centred, float64 (single-unit L1)."""
    return gaussian(200, 1000, seed, dtype=np.float64, centre=True)


def workload_spikes_5000x20000(seed: int = 0, p: int = 5000, n: int = 20000, with_meta: bool = False):
    """5000 x 20000 float32, 5 spikes, theta_j = 40/j, 5% disjoint supports."""
    k = 5
    return planted_spike(p, n, k, [40.0 / j for j in range(1, k + 1)], support_frac=0.05,
                         seed=seed, dtype=np.float32, with_meta=with_meta)


def workload_spikes_10000x50000(seed: int = 1, p: int = 10000, n: int = 50000, with_meta: bool = False):
    """10000 x 50000 float32, 3 spikes, theta_j = 40/j, 2% disjoint supports."""
    k = 3
    return planted_spike(p, n, k, [40.0 / j for j in range(1, k + 1)], support_frac=0.02,
                         seed=seed, dtype=np.float32, with_meta=with_meta)


def workload_spikes_20000x100000(seed: int = 2, p: int = 20000, n: int = 100000, with_meta: bool = False):
    """20000 x 100000 float32, 16 spikes, theta_j = 100/sqrt(j), 1% supports."""
    k = 16
    return planted_spike(p, n, k, [100.0 / np.sqrt(j) for j in range(1, k + 1)], support_frac=0.01,
                         seed=seed, dtype=np.float32, with_meta=with_meta)


def log_spaced_rho(count: int = 64, lo: float = 1e-3, hi: float = 0.5) -> np.ndarray:
    """``count`` relative sparsity values log-spaced over [lo, hi]."""
    return np.geomspace(lo, hi, count)
