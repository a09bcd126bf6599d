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

import os
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
    noise_streams: int = 1,
    blocks: Optional[tuple] = None,
):
    """Planted sparse spikes: A = N(0,1) + sum_{j<k} theta_j u_j v_j^T.

    Each v_j has ``support_size`` (or round(support_frac * n)) nonzeros,
    +-1/sqrt(s), on supports that are disjoint across j.

    ``noise_streams`` > 1 (the matrices of billions of entries): the noise is
    drawn in that many equal blocks of columns of A, block b from the b-th
    child of ``SeedSequence(seed).spawn(noise_streams)``, filled on parallel
    threads; u, supports and signs then come from ``default_rng(seed)`` in the
    usual order.  ``blocks = (b0, b1)`` then returns only the columns of
    noise blocks b0 .. b1-1 (bit-identical to those columns of the whole
    matrix): a sample of a matrix too large to draw in full.
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
    lo, hi = 0, n
    if noise_streams > 1:
        b0, b1 = (0, noise_streams) if blocks is None else blocks
        lo, hi = b0 * n // noise_streams, b1 * n // noise_streams
        At = _noise_blocks(n, p, seed, noise_streams, b0, b1)
    else:
        if blocks is not None:
            raise ValueError("blocks needs noise_streams > 1")
        At = rng.standard_normal((n, p), dtype=np.float32)  # noise
    U = rng.standard_normal((k, p))  # u_j ~ N(0, I_p)
    perm = rng.permutation(n)[: k * s]
    supports = [np.sort(perm[j * s : (j + 1) * s]) for j in range(k)]
    signs = [rng.choice(np.array([-1.0, 1.0]), size=s) for _ in range(k)]
    for j in range(k):
        if s == 0:
            continue
        keep = (supports[j] >= lo) & (supports[j] < hi)
        idx = supports[j][keep] - lo
        v = signs[j][keep] / np.sqrt(s)
        rows = At[idx].astype(np.float64) + theta[j] * np.outer(v, U[j])
        At[idx] = rows.astype(np.float32)
    out = np.ascontiguousarray(At.astype(dtype, copy=False))
    if with_meta:
        return out, SpikeMeta(theta, U, supports, signs)
    return out


def _noise_blocks(n: int, p: int, seed: int, streams: int, b0: int = 0, b1: Optional[int] = None) -> np.ndarray:
    """N(0,1) float32 rows [b n / streams, (b+1) n / streams) of an n x p
    array, each drawn from the b-th child seed of ``seed``, for blocks b0 ..
    b1-1 (see ``planted_spike``)."""
    import concurrent.futures

    b1 = streams if b1 is None else b1
    base = b0 * n // streams
    out = np.empty((b1 * n // streams - base, p), dtype=np.float32)
    kids = np.random.SeedSequence(seed).spawn(streams)

    def fill(b):
        lo, hi = b * n // streams - base, (b + 1) * n // streams - base
        np.random.default_rng(kids[b]).standard_normal(out=out[lo:hi], dtype=np.float32)

    with concurrent.futures.ThreadPoolExecutor(min(b1 - b0, os.cpu_count() or 1)) as ex:
        list(ex.map(fill, range(b0, b1)))
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
    """10000 x 50000 float32, 3 spikes, theta_j = 40/j, 2% disjoint supports
    (noise in 16 parallel streams)."""
    k = 3
    return planted_spike(p, n, k, [40.0 / j for j in range(1, k + 1)], support_frac=0.02,
                         seed=seed, dtype=np.float32, with_meta=with_meta, noise_streams=16)


def workload_spikes_20000x100000(seed: int = 2, p: int = 20000, n: int = 100000, with_meta: bool = False,
                                 blocks: Optional[tuple] = None):
    """20000 x 100000 float32, 16 spikes, theta_j = 100/sqrt(j), 1% supports
    (noise in 16 parallel streams of 6250 columns; ``blocks`` selects some)."""
    k = 16
    return planted_spike(p, n, k, [100.0 / np.sqrt(j) for j in range(1, k + 1)], support_frac=0.01,
                         seed=seed, dtype=np.float32, with_meta=with_meta, noise_streams=16, blocks=blocks)


def log_spaced_rho(count: int = 64, lo: float = 1e-3, hi: float = 0.5) -> np.ndarray:
    """``count`` relative sparsity values log-spaced over [lo, hi]."""
    return np.geomspace(lo, hi, count)


# ---------------------------------------------------------------- counter-based generator
#
# Per-request matrices of the serving workload are drawn on the device by a
# counter-based generator so that no host-side RNG or copy sits in the
# request path; this is its NumPy twin (same counters, same float32
# arithmetic), used to regenerate any request's A on the host.
#
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
# easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and a 2 x 32-bit key; ten
# rounds, each multiplying words 0 and 2 by fixed constants (high and low
# halves of the 64-bit products) and mixing in the key, which is bumped by
# two Weyl constants between rounds.

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
TWO_PI_F32 = np.float32(6.2831855)


def philox4x32_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x32-10 of the counters (c0, c1, c2, c3) (uint32 arrays or
    scalars, broadcast) under key (k0, k1); returns four uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint32) for x in (c0, c1, c2, c3)]
    c = list(np.broadcast_arrays(*c))
    k0 &= 0xFFFFFFFF
    k1 &= 0xFFFFFFFF
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    lo_mask, sh = np.uint64(0xFFFFFFFF), np.uint64(32)
    for _ in range(10):
        p0 = m0 * c[0].astype(np.uint64)
        p1 = m1 * c[2].astype(np.uint64)
        hi0, lo0 = (p0 >> sh).astype(np.uint32), (p0 & lo_mask).astype(np.uint32)
        hi1, lo1 = (p1 >> sh).astype(np.uint32), (p1 & lo_mask).astype(np.uint32)
        c = [hi1 ^ c[1] ^ np.uint32(k0), lo1, hi0 ^ c[3] ^ np.uint32(k1), lo0]
        k0 = (k0 + PHILOX_W0) & 0xFFFFFFFF
        k1 = (k1 + PHILOX_W1) & 0xFFFFFFFF
    return c


def _uniform23(w):
    """uint32 -> float32 in (0, 1): the top 23 bits plus one half, times 2^-23
    (exact in float32, so 0 and 1 are never returned)."""
    return ((w >> np.uint32(9)).astype(np.float32) + np.float32(0.5)) * np.float32(2.0 ** -23)


def _box_muller(w0, w1, w2, w3):
    """Four N(0,1) float32 values from four words (Box-Muller on two pairs)."""
    out = []
    for a, b in ((w0, w1), (w2, w3)):
        u1, u2 = _uniform23(a), _uniform23(b)
        rad = np.sqrt(np.float32(-2.0) * np.log(u1)).astype(np.float32)
        ang = (TWO_PI_F32 * u2).astype(np.float32)
        out += [(rad * np.cos(ang)).astype(np.float32), (rad * np.sin(ang)).astype(np.float32)]
    return out


def spike_coefficients(k: int, theta, support_frac: float, n: int) -> np.ndarray:
    """theta_j / sqrt(s) in float32, s = max(1, round(support_frac * n)) the
    expected support size (the scale both generators use)."""
    s = max(1, int(round(support_frac * n)))
    return (np.asarray(theta, dtype=np.float64)[:k] / np.sqrt(s)).astype(np.float32)


def counter_spikes(p: int, n: int, k: int, theta, support_frac: float, seed: int, dtype=np.float32):
    """The device generator's matrix, on the host: At (n x p).

    Entry (r, i) = noise + [i in support of spike j] sign_i theta_j/sqrt(s) u_j[r]:
    * noise: rows 4b..4b+3 of column i from counter (b, i_lo, i_hi, 0);
    * u_j: rows 4b..4b+3 from counter (b, j, 0, 1);
    * column i's spike: counter (i_lo, i_hi, 0, 2), word 0 as a uniform v,
      j = floor(v / support_frac) if below k (disjoint supports of expected
      size support_frac n), sign from the top bit of word 1;
    key = (seed_lo, seed_hi).  float32 arithmetic, products and sums
    rounded separately; bfloat16 output rounds to nearest even."""
    P4 = (p + 3) // 4
    k0, k1 = seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF
    i = np.arange(n, dtype=np.uint64)
    ilo, ihi = (i & np.uint64(0xFFFFFFFF)).astype(np.uint32), (i >> np.uint64(32)).astype(np.uint32)
    b = np.arange(P4, dtype=np.uint32)
    w = philox4x32_10(b[None, :], ilo[:, None], ihi[:, None], np.uint32(0), k0, k1)
    z = _box_muller(*w)  # each n x P4
    At = np.stack(z, axis=2).reshape(n, 4 * P4)[:, :p].astype(np.float32)
    sw = philox4x32_10(ilo, ihi, np.uint32(0), np.uint32(2), k0, k1)
    v = _uniform23(sw[0])
    j = np.floor(v / np.float32(support_frac)).astype(np.int64) if support_frac > 0 else np.full(n, k)
    sign = np.where(sw[1] >> np.uint32(31), np.float32(-1.0), np.float32(1.0)).astype(np.float32)
    coef = spike_coefficients(k, theta, support_frac, n)
    for jj in range(k):
        cols = np.nonzero(j == jj)[0]
        if cols.size == 0:
            continue
        uw = philox4x32_10(b, np.uint32(jj), np.uint32(0), np.uint32(1), k0, k1)
        u = np.stack(_box_muller(*uw), axis=1).reshape(4 * P4)[:p].astype(np.float32)
        c = (coef[jj] * sign[cols]).astype(np.float32)
        At[cols] = (At[cols] + (c[:, None] * u[None, :]).astype(np.float32)).astype(np.float32)
    if dtype == "bf16":
        bits = At.view(np.uint32)
        rnd = (bits + np.uint32(0x7FFF) + ((bits >> np.uint32(16)) & np.uint32(1))) & np.uint32(0xFFFF0000)
        return rnd.view(np.float32)  # bfloat16 values, held in float32
    return np.ascontiguousarray(At)


@dataclass
class Request:
    """One request of the serving mix."""

    id: int
    arrival_s: float
    p: int
    n: int
    dtype: str  # "f32" or "bf16"
    form: str
    m: int
    rho: float
    seed: int

    def gammas(self):
        """Relative gammas: one per component (block), or for single-unit
        forms a path of m values linearly spaced over [rho/2, rho]."""
        if self.form.startswith("B") or self.m == 1:
            return [self.rho] * self.m
        return [self.rho * (0.5 + 0.5 * j / (self.m - 1)) for j in range(self.m)]

    def theta(self):
        k = max(self.m, 1)
        return [40.0 / (j + 1) for j in range(k)]


def serving_requests(count: int = 2000, rate: float = 200.0, seed: int = 3):
    """The serving mix: Poisson arrivals at `rate`, p and n log-uniform over
    [256, 8192] and [1024, 65536], FP32 or BF16, the four forms, m in 1..16,
    rho ~ U(0.02, 0.2); request i's matrix has seed 1000 + i."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    arr = np.cumsum(gaps) - gaps[0]
    ps = np.round(np.exp(rng.uniform(np.log(256), np.log(8192), size=count))).astype(int)
    ns = np.round(np.exp(rng.uniform(np.log(1024), np.log(65536), size=count))).astype(int)
    dts = rng.integers(0, 2, size=count)
    forms = rng.integers(0, 4, size=count)
    ms = rng.integers(1, 17, size=count)
    rhos = rng.uniform(0.02, 0.2, size=count)
    names = ["SL1", "SL0", "BL1", "BL0"]
    return [Request(i, float(arr[i]), int(ps[i]), int(ns[i]), "bf16" if dts[i] else "f32", names[forms[i]],
                    int(ms[i]), float(rhos[i]), 1000 + i) for i in range(count)]
