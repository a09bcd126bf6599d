"""Pins for the oracle's multi-component extraction by projection deflation.

The paper extracts several single-unit components (Section 4.1, Fig. 3,
m = 5) without stating the deflation; the oracle reads it as projection
deflation A_j = A_{j-1} (I - z_j z_j^T).  These checks tie that oracle to
mathematics it does not compute directly: the singular value decomposition
(gamma = 0), a closed form on orthogonal sparse spikes, and the null vector
and rank the projection leaves.  A slip such as deflating with x instead of
A z, skipping the deflation, or deflating the wrong side fails one of them.
"""

import numpy as np
import pytest

import oracle


def _spikes(p, n, thetas, s, seed):
    """A = sum_j theta_j u_j v_j^T: orthonormal u_j, v_j with disjoint supports
    of s entries, all of magnitude 1/sqrt(s) (so the SL1 loading is v_j exactly)."""
    rng = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rng.standard_normal((p, len(thetas))))
    perm = rng.permutation(n)
    V = np.zeros((n, len(thetas)))
    for j in range(len(thetas)):
        idx = perm[j * s:(j + 1) * s]
        V[idx, j] = rng.choice([-1.0, 1.0], size=s) / np.sqrt(s)
    return U @ np.diag(thetas) @ V.T, U, V


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_gamma_zero_gives_singular_vectors_in_order(form):
    # gamma = 0: each single-unit solve is the leading singular pair of A_{j-1};
    # deflating by z_j = v_j removes sigma_j, so component j is the j-th pair
    rng = np.random.default_rng(3)
    p, n, sig = 30, 50, np.array([9.0, 7.0, 5.0, 3.5])
    U, _ = np.linalg.qr(rng.standard_normal((p, 4)))
    V, _ = np.linalg.qr(rng.standard_normal((n, 4)))
    A = U @ np.diag(sig) @ V.T + 0.05 * rng.standard_normal((p, n))
    Us, S, Vt = np.linalg.svd(A)
    r = oracle.gpower_deflated(A, form, [0.0] * 4, tol=1e-15, maxit=5000)
    for j in range(4):
        assert abs(abs(r.Z[:, j] @ Vt[j]) - 1.0) < 1e-9
        assert abs(abs(r.X[:, j] @ Us[:, j]) - 1.0) < 1e-9
        assert r.objective[j] == pytest.approx(S[j] ** 2, rel=1e-10)  # f = ||A^T x||^2 at gamma = 0


def test_orthogonal_sparse_spikes_closed_form():
    # noiseless spikes with disjoint supports: at x = u_j, t = theta_j v_j, so
    # the SL1 loading is v_j, f_j = s (theta_j / sqrt(s) - gamma)^2; deflation
    # removes spike j exactly and the next solve finds spike j + 1
    thetas, s = np.array([12.0, 8.0, 5.0]), 10
    A, U, V = _spikes(40, 200, thetas, s, seed=5)
    gam = 0.5
    r = oracle.gpower_deflated(A, "SL1", [gam] * 3, tol=1e-14, maxit=200)
    for j in range(3):
        assert abs(abs(r.Z[:, j] @ V[:, j]) - 1.0) < 1e-12
        assert abs(abs(r.X[:, j] @ U[:, j]) - 1.0) < 1e-12
        assert r.objective[j] == pytest.approx(s * (thetas[j] / np.sqrt(s) - gam) ** 2, rel=1e-12)
    # SL0 on the same matrix: f_j = s (theta_j^2 / s - gamma)
    r0 = oracle.gpower_deflated(A, "SL0", [0.25] * 3, tol=1e-14, maxit=200)
    for j in range(3):
        assert abs(abs(r0.Z[:, j] @ V[:, j]) - 1.0) < 1e-12
        assert r0.objective[j] == pytest.approx(s * (thetas[j] ** 2 / s - 0.25), rel=1e-12)


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_deflation_leaves_last_loading_in_the_null_space(form):
    # A_m z_m = 0, and with full column rank (p > n, so every loading lies in
    # the row space) each nonzero component lowers the rank by one
    rng = np.random.default_rng(11)
    A = rng.standard_normal((60, 25))
    g = oracle.gamma_from_rho(A, form, 0.3)[0]
    r, Am = oracle.gpower_deflated(A, form, [g] * 3, tol=1e-12, maxit=500, return_deflated=True)
    assert np.all(r.status != oracle.STATUS_ZERO)
    assert np.linalg.norm(Am @ r.Z[:, 2]) < 1e-12 * np.linalg.norm(A)
    assert np.linalg.matrix_rank(Am) == np.linalg.matrix_rank(A) - 3
    # columns outside every support are untouched
    outside = ~np.any(r.Z != 0, axis=1)
    assert outside.sum() > 0
    assert np.array_equal(Am[:, outside], A[:, outside])


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_first_component_is_the_plain_solve(form):
    rng = np.random.default_rng(2)
    A = rng.standard_normal((20, 45))
    g = oracle.gamma_from_rho(A, form, 0.2)[0]
    r = oracle.gpower_deflated(A, form, [g, g], tol=1e-10, maxit=300)
    r1 = oracle.gpower(A, form, [g], tol=1e-10, maxit=300)
    assert np.array_equal(r.Z[:, 0], r1.Z[:, 0])
    assert r.objective[0] == r1.objective[0]


def test_relative_gamma_follows_the_deflated_matrix():
    # the relative gamma of component j scales with max column norm of A_{j-1}
    thetas, s = np.array([12.0, 8.0]), 10
    A, _, _ = _spikes(40, 200, thetas, s, seed=7)
    r = oracle.gpower_deflated(A, "SL1", [0.1, 0.1], tol=1e-14, maxit=200, relative=True)
    # column norms: theta_j / sqrt(s) on spike j's support; after removing spike 1
    # only spike 2's columns are nonzero
    assert r.gamma[0] == pytest.approx(0.1 * thetas[0] / np.sqrt(s), rel=1e-12)
    assert r.gamma[1] == pytest.approx(0.1 * thetas[1] / np.sqrt(s), rel=1e-12)


def test_rejects_block_forms():
    with pytest.raises(ValueError):
        oracle.gpower_deflated(np.eye(3), "BL1", [0.1])


def test_null_space_holds_before_convergence():
    # the projection removes z_j whatever iterate produced it: stopped after
    # two sweeps (far from the fixed point, where A z_j is not parallel to x_j)
    # A_1 z_1 = 0 still holds
    rng = np.random.default_rng(4)
    A = rng.standard_normal((40, 30))
    g = oracle.gamma_from_rho(A, "SL1", 0.2)[0]
    r, A1 = oracle.gpower_deflated(A, "SL1", [g], tol=0.0, maxit=2, return_deflated=True)
    assert r.status[0] == oracle.STATUS_MAXIT
    Az = A @ r.Z[:, 0]
    assert abs(abs(Az @ r.X[:, 0]) / np.linalg.norm(Az) - 1.0) > 1e-6  # not yet parallel
    assert np.linalg.norm(A1 @ r.Z[:, 0]) < 1e-13 * np.linalg.norm(A)
