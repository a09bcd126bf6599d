"""Pins for the FP64 oracle against what the paper and the mathematics fix.

Each test names the property it checks and the passage it follows.  Together
they are chosen so that a plausible slip in the oracle (a dropped square or
weight, a flipped sign, a transposed operand, a wrong stopping index, a
non-strict threshold) fails at least one of them.
"""

import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1312_6182_gb300 import synth
from tests.pins import original_block, original_single

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand(p, n, seed):
    return np.random.default_rng(seed).standard_normal((p, n))


def _low_rank_plus_noise(p, n, sigmas, seed, noise=0.0):
    """A = U diag(sigmas) V^T (+ noise) with known singular vectors."""
    rng = np.random.default_rng(seed)
    r = len(sigmas)
    U, _ = np.linalg.qr(rng.standard_normal((p, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return U @ np.diag(sigmas) @ V.T + noise * rng.standard_normal((p, n)), U, V


# ---------------------------------------------------------------- Table 1 scalars

def _golden_rows():
    rows = []
    with open(os.path.join(GOLDEN, "table1_scalars.tsv")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            rows.append((f[0],) + tuple(float(v) for v in f[1:]))
    return rows


@pytest.mark.parametrize("row", _golden_rows())
def test_table1_scalar_truth_table(row):
    """Table 1 summands on hand-evaluated scalars, ties included."""
    form, t, g, mu, term, grad, load = row
    T = np.array([[t]])
    gam = np.array([g])
    m = np.array([mu])
    assert oracle.objective_parts(form, T, gam, m)[0] == pytest.approx(term, abs=1e-15)
    assert oracle.gradient_direction(form, T, gam, m)[0, 0] == pytest.approx(grad, abs=1e-15)
    # loadings normalise; a two-entry column with one known entry checks the ratio
    T2 = np.array([[t], [10.0 * np.sign(t) if t != 0 else 10.0]])
    Z = oracle.loadings(form, T2, gam, m)[:, 0]
    if form in ("SL1", "BL1"):
        other = np.sign(T2[1, 0]) * max(mu * abs(T2[1, 0]) - g, 0.0)
    else:
        other = mu * T2[1, 0] * ((mu * T2[1, 0]) ** 2 > g)
    ref = np.array([load, other])
    ref = ref / np.linalg.norm(ref)
    np.testing.assert_allclose(Z, ref, atol=1e-15)


# ---------------------------------------------------------------- original form

@pytest.mark.parametrize("form", ["SL1", "SL0"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_unit_matches_original_form(form, seed):
    """Table 1: for the recovered z the original-form value at fixed x equals the
    reformulated objective (sqrt(f) for SL1, f for SL0), at every x; at the
    converged x, also with the free maximisation over x (||A z||)."""
    A = _rand(30, 80, seed)
    rho = 0.35 if form == "SL1" else 0.35
    gamma = oracle.gamma_from_rho(A, form, rho)
    r = oracle.gpower(A, form, gamma, tol=1e-13, maxit=5000)
    assert r.status[0] == oracle.STATUS_CONVERGED
    x, z, f = r.X[:, 0], r.Z[:, 0], r.objective[0]
    free, fixed = original_single(form, A, x, z, gamma[0])
    target = np.sqrt(f) if form == "SL1" else f
    assert fixed == pytest.approx(target, rel=1e-12)
    assert free == pytest.approx(target, rel=1e-6)
    # at an arbitrary unit x the fixed-x identity still holds
    rng = np.random.default_rng(seed + 100)
    xr = rng.standard_normal(30)
    xr /= np.linalg.norm(xr)
    t = A.T @ xr
    fr = oracle.objective_parts(form, t[:, None], gamma, np.ones(1))[0]
    zr = oracle.loadings(form, t[:, None], gamma, np.ones(1))[:, 0]
    if fr > 0:
        _, fixed_r = original_single(form, A, xr, zr, gamma[0])
        assert fixed_r == pytest.approx(np.sqrt(fr) if form == "SL1" else fr, rel=1e-12)


@pytest.mark.parametrize("form", ["BL1", "BL0"])
@pytest.mark.parametrize("mu", [[1, 1, 1], [1.0, 0.7, 0.4]])
def test_block_matches_original_form(form, mu):
    """Table 1 block rows: for any orthonormal X and the recovered Z,
    BL1: Tr(X^T A Z N) - sum gamma_j ||z_j||_1 = sum_j sqrt(f_j);
    BL0: Tr(Diag(X^T A Z N)^2) - sum gamma_j ||z_j||_0 = sum_j f_j."""
    mu = np.array(mu, dtype=np.float64)
    A = _rand(25, 60, 3)
    c = oracle.column_norms(A).max()
    gamma = (0.2 * c * mu) if form == "BL1" else (0.2 * c * mu) ** 2
    rng = np.random.default_rng(7)
    for trial in range(3):
        X, _ = np.linalg.qr(rng.standard_normal((25, 3)))
        T = A.T @ X
        fj = oracle.objective_parts(form, T, gamma, mu)
        Z = oracle.loadings(form, T, gamma, mu)
        val = original_block(form, A, X, Z, gamma, mu)
        target = np.sum(np.sqrt(fj)) if form == "BL1" else np.sum(fj)
        assert val == pytest.approx(target, rel=1e-12)
    r = oracle.gpower(A, form, gamma, mu=mu, tol=1e-12, maxit=3000)
    assert r.status[0] == oracle.STATUS_CONVERGED
    val = original_block(form, A, r.X, r.Z, gamma, mu)
    target = np.sum(np.sqrt(r.objective)) if form == "BL1" else r.total
    assert val == pytest.approx(target, rel=1e-12)


# ---------------------------------------------------------------- ascent + invariants

@pytest.mark.parametrize("form", oracle.FORMS)
@pytest.mark.parametrize("seed", [0, 5])
def test_monotone_ascent_and_feasibility(form, seed):
    """Section 2: a convex objective over the sphere / Stiefel manifold; each
    power step cannot decrease it.  Iterates stay feasible (unit x,
    orthonormal X) and the loadings are unit-norm or zero."""
    A = _rand(40, 150, seed)
    if form in ("SL1", "SL0"):
        gamma = oracle.gamma_from_rho(A, form, [0.05, 0.2, 0.4])
        mu = None
    else:
        mu = np.array([1.0, 0.9, 0.8, 0.7])
        c = oracle.column_norms(A).max()
        gamma = 0.15 * c * mu if form == "BL1" else (0.15 * c * mu) ** 2
    r = oracle.gpower(A, form, gamma, mu=mu, tol=0.0, maxit=60)
    for hist in r.history:
        h = np.array(hist)
        assert np.all(np.diff(h) >= -1e-12 * np.abs(h[:-1]))
    if form in ("SL1", "SL0"):
        np.testing.assert_allclose(np.linalg.norm(r.X, axis=0), 1.0, atol=1e-13)
    else:
        np.testing.assert_allclose(r.X.T @ r.X, np.eye(r.X.shape[1]), atol=1e-12)
    zn = np.linalg.norm(r.Z, axis=0)
    assert np.all((np.abs(zn - 1) < 1e-13) | (zn == 0))


def test_tol_zero_runs_exactly_maxit_sweeps():
    """Stopping reading: with tol = 0 only f = 0 or maxit stops the solve, and
    the sweep count returned equals maxit."""
    A = _rand(20, 50, 1)
    r = oracle.gpower(A, "SL1", oracle.gamma_from_rho(A, "SL1", 0.1), tol=0.0, maxit=17)
    assert r.iters[0] == 17 and r.status[0] == oracle.STATUS_MAXIT
    assert len(r.history[0]) == 17


def test_maxit_one_returns_x0():
    """With maxit = 1 the returned iterate is x0 = a_{i*}/||a_{i*}||, and the
    returned objective is the one x0 produces."""
    A = _rand(20, 50, 2)
    i = int(np.argmax(np.linalg.norm(A, axis=0)))
    r = oracle.gpower(A, "SL0", oracle.gamma_from_rho(A, "SL0", 0.1), maxit=1)
    np.testing.assert_allclose(r.X[:, 0], A[:, i] / np.linalg.norm(A[:, i]), atol=1e-15)
    t = A.T @ r.X[:, 0]
    g = r.gamma[0]
    assert r.objective[0] == pytest.approx(np.sum(np.maximum(t * t - g, 0)), rel=1e-14)


def test_start_at_fixed_point_stops_after_second_sweep():
    """Stopping reading: the first comparison is between f_1 and f_0.  If x0 is
    already a fixed point (the largest column is orthogonal to all others),
    f_1 == f_0 and the solve stops with 2 sweeps, returning x0."""
    A = np.zeros((4, 5))
    A[0, 2] = 3.0  # largest column, orthogonal to the rest
    A[1, 0] = 1.0
    A[2, 1] = 0.5
    A[3, 3] = 0.25
    A[3, 4] = 0.25
    e0 = np.zeros((4, 1))
    e0[0, 0] = 1.0  # the largest column's direction; block forms take it as x0
    for form in oracle.FORMS:
        block = form[0] == "B"
        r = oracle.gpower(A, form, [0.1], mu=[1.0] if block else None, tol=1e-6, x0=e0 if block else None)
        assert r.status[0] == oracle.STATUS_CONVERGED and r.iters[0] == 2
        assert abs(r.X[0, 0]) == 1.0
        np.testing.assert_array_equal(np.flatnonzero(r.Z[:, 0]), [2])


def test_fixed_point_at_convergence():
    """At convergence x is (to the stopping tolerance) a fixed point of the power
    step: x = A g(x) / ||A g(x)||, and X = polar(A G(X))."""
    A = _rand(30, 100, 4)
    for form in ("SL1", "SL0"):
        g = oracle.gamma_from_rho(A, form, 0.2)
        r = oracle.gpower(A, form, g, tol=1e-14, maxit=10000)
        x = r.X[:, 0]
        G = oracle.gradient_direction(form, (A.T @ x)[:, None], g, np.ones(1))[:, 0]
        y = A @ G
        np.testing.assert_allclose(y / np.linalg.norm(y), x, atol=1e-6)
    mu = np.array([1.0, 0.8, 0.6])
    c = oracle.column_norms(A).max()
    for form, gam in (("BL1", 0.2 * c * mu), ("BL0", (0.2 * c * mu) ** 2)):
        r = oracle.gpower(A, form, gam, mu=mu, tol=1e-14, maxit=10000)
        Y = A @ oracle.gradient_direction(form, A.T @ r.X, gam, mu)
        U, _, Vt = np.linalg.svd(Y, full_matrices=False)
        np.testing.assert_allclose(U @ Vt, r.X, atol=1e-6)


# ---------------------------------------------------------------- special cases

@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_gamma_zero_is_leading_singular_pair(form):
    """gamma = 0: both single-unit objectives become ||A^T x||^2 and the power
    step is the power method on A A^T: x -> leading left singular vector u_1,
    z -> leading right singular vector v_1, f -> sigma_1^2 (checked against an
    SVD computed independently)."""
    A = _rand(8, 20, 11)
    U, s, Vt = np.linalg.svd(A)
    r = oracle.gpower(A, form, [0.0], tol=1e-15, maxit=20000)
    assert abs(r.X[:, 0] @ U[:, 0]) == pytest.approx(1.0, abs=1e-10)
    assert abs(r.Z[:, 0] @ Vt[0]) == pytest.approx(1.0, abs=1e-10)
    if form == "SL0":
        assert r.objective[0] == pytest.approx(s[0] ** 2, rel=1e-10)
    else:
        assert r.objective[0] == pytest.approx(s[0] ** 2, rel=1e-10)
    assert np.count_nonzero(r.Z[:, 0]) == 20


@pytest.mark.parametrize("form", ["BL1", "BL0"])
def test_block_gamma_zero_distinct_mu_gives_ordered_singular_vectors(form):
    """gamma = 0, distinct mu: f = Tr(N^2 X^T A A^T X), maximised over the
    Stiefel manifold by the top-m left singular vectors, the largest mu paired
    with the largest singular value; f* = sum mu_j^2 sigma_j^2."""
    A, U, V = _low_rank_plus_noise(12, 30, [9.0, 6.0, 4.0, 2.0, 1.0], seed=2, noise=0.05)
    Us, s, Vts = np.linalg.svd(A)
    mu = np.array([1.0, 0.8, 0.6])
    r = oracle.gpower(A, form, np.zeros(3), mu=mu, tol=1e-15, maxit=20000)
    for j in range(3):
        assert abs(r.X[:, j] @ Us[:, j]) == pytest.approx(1.0, abs=1e-8)
        assert abs(r.Z[:, j] @ Vts[j]) == pytest.approx(1.0, abs=1e-8)
    assert r.total == pytest.approx(np.sum(mu**2 * s[:3] ** 2), rel=1e-10)


@pytest.mark.parametrize("form", oracle.FORMS)
def test_gamma_above_column_norm_bound_gives_zero(form):
    """Cauchy-Schwarz: |a_i^T x| <= ||a_i||, so gamma >= max||a_i|| (L1) or
    max||a_i||^2 (L0) zeroes every summand: f = 0, Z = 0 after one sweep.
    For single-unit forms x0 attains the bound, so just below it f > 0."""
    A = _rand(15, 40, 6)
    c = oracle.column_norms(A).max()
    m = 1 if form in ("SL1", "SL0") else 2
    mu = None if m == 1 else np.ones(m)
    big = np.full(m, c if form in ("SL1", "BL1") else c * c)
    r = oracle.gpower(A, form, big, mu=mu)
    assert np.all(r.status == oracle.STATUS_ZERO)
    assert np.all(r.iters == 1) and np.all(r.Z == 0) and np.all(r.objective == 0)
    if m == 1:
        # x0 = a_{i*}/||a_{i*}|| attains |t_{i*}| = max||a_i||, so the bound is tight
        below = big * (0.999 if form == "SL1" else 0.998)
        r2 = oracle.gpower(A, form, below, mu=mu, maxit=1)
        assert r2.total > 0


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_block_with_one_component_equals_single_unit(form):
    """m = 1, mu = 1: the block rows of Table 1 reduce to the single-unit rows."""
    A = _rand(25, 70, 8)
    g = oracle.gamma_from_rho(A, form, 0.25)
    s = oracle.gpower(A, form, g, tol=1e-10)
    x0 = oracle.initial_iterate(A, form, 1)[0]
    b = oracle.gpower(A, "B" + form[1:], g, mu=[1.0], tol=1e-10, x0=x0)
    assert s.iters[0] == b.iters[0]
    sgn = np.sign(s.X[:, 0] @ b.X[:, 0])
    np.testing.assert_allclose(b.X[:, 0], sgn * s.X[:, 0], atol=1e-12)
    np.testing.assert_allclose(b.Z[:, 0], sgn * s.Z[:, 0], atol=1e-12)
    assert b.objective[0] == pytest.approx(s.objective[0], rel=1e-12)


@pytest.mark.parametrize("form", ["BL1", "BL0"])
def test_block_mu_scaling_invariance(form):
    """Scaling mu by c and gamma by c (L1) or c^2 (L0) multiplies every
    summand by c^2 (Table 1 block rows), so the iterates are unchanged."""
    A = _rand(20, 60, 9)
    cmax = oracle.column_norms(A).max()
    mu = np.array([1.0, 0.6])
    gam = 0.2 * cmax * mu if form == "BL1" else (0.2 * cmax * mu) ** 2
    r1 = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=30)
    cs = 3.0
    gam2 = gam * cs if form == "BL1" else gam * cs * cs
    r2 = oracle.gpower(A, form, gam2, mu=mu * cs, tol=0.0, maxit=30)
    np.testing.assert_allclose(r2.X, r1.X, atol=1e-11)
    np.testing.assert_allclose(r2.Z, r1.Z, atol=1e-11)
    np.testing.assert_allclose(r2.objective, cs * cs * r1.objective, rtol=1e-11)


@pytest.mark.parametrize("form", oracle.FORMS)
def test_rotation_of_samples_is_equivariant(form):
    """Replacing A by Q A (Q orthogonal p x p) and x0 by Q x0 maps X to Q X and
    leaves t = A^T x, the objective and Z unchanged; a transposed operand
    anywhere breaks this.  (Single-unit forms pick x0 from A itself.)"""
    A = _rand(18, 45, 12)
    Q, _ = np.linalg.qr(np.random.default_rng(13).standard_normal((18, 18)))
    m = 2 if form in ("SL1", "SL0") else 3
    mu = None if form in ("SL1", "SL0") else np.array([1.0, 0.8, 0.5])
    c = oracle.column_norms(A).max()
    rho = np.array([0.1, 0.3, 0.2][:m])
    gam = rho * c if form in ("SL1", "BL1") else (rho * c) ** 2
    if mu is not None:
        gam = gam * (mu if form == "BL1" else mu * mu)
    x0 = np.linalg.qr(np.random.default_rng(14).standard_normal((18, m)))[0] if mu is not None else None
    r1 = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=25, x0=x0)
    r2 = oracle.gpower(Q @ A, form, gam, mu=mu, tol=0.0, maxit=25, x0=None if x0 is None else Q @ x0)
    np.testing.assert_allclose(r2.X, Q @ r1.X, atol=1e-10)
    np.testing.assert_allclose(r2.Z, r1.Z, atol=1e-10)
    np.testing.assert_allclose(r2.objective, r1.objective, rtol=1e-10)


def test_variable_permutation_permutes_loadings():
    """Permuting the variables (columns a_i) permutes the rows of Z and leaves
    X and f unchanged (no ties among the column norms)."""
    A = _rand(16, 40, 14)
    perm = np.random.default_rng(15).permutation(40)
    for form in oracle.FORMS:
        m = 2
        mu = None if form in ("SL1", "SL0") else np.array([1.0, 0.7])
        c = oracle.column_norms(A).max()
        gam = np.array([0.15, 0.25]) * c
        if form in ("SL0", "BL0"):
            gam = gam ** 2
        r1 = oracle.gpower(A, form, gam, mu=mu, tol=0.0, maxit=20)
        r2 = oracle.gpower(A[:, perm], form, gam, mu=mu, tol=0.0, maxit=20)
        np.testing.assert_allclose(r2.X, r1.X, atol=1e-11)
        np.testing.assert_allclose(r2.Z, r1.Z[perm], atol=1e-11)


# ---------------------------------------------------------------- brute force

def _brute_force_sl0(A, gamma):
    """max over supports S of lambda_max(A_S^T A_S) - gamma |S| (and 0 for S empty):
    the global optimum of the SL0 original form max_{z in B^n} z^T Sigma z - gamma ||z||_0."""
    n = A.shape[1]
    best = 0.0
    for r in range(1, n + 1):
        for S in itertools.combinations(range(n), r):
            As = A[:, S]
            lam = np.linalg.eigvalsh(As.T @ As)[-1]
            best = max(best, lam - gamma * r)
    return best


@pytest.mark.parametrize("seed", range(4))
def test_sl0_against_support_enumeration(seed):
    """Brute force over all 2^n supports on tiny A (n = 10): the power method's
    value never exceeds the global optimum, equals lambda_max(A_S A_S^T) - gamma|S|
    for its own support S, and the best of 64 random starts reaches the optimum."""
    A = _rand(6, 10, 40 + seed)
    gamma = float(oracle.gamma_from_rho(A, "SL0", 0.55)[0])
    best = _brute_force_sl0(A, gamma)
    r = oracle.gpower(A, "SL0", [gamma], tol=1e-14, maxit=10000)
    f = r.objective[0]
    assert f <= best + 1e-9 * max(1.0, best)
    S = np.flatnonzero(r.Z[:, 0])
    lam = np.linalg.eigvalsh(A[:, S].T @ A[:, S])[-1]
    assert f == pytest.approx(lam - gamma * len(S), rel=1e-9)
    rng = np.random.default_rng(seed)
    vals = []
    for _ in range(64):
        x0 = rng.standard_normal(6)
        x0 /= np.linalg.norm(x0)
        vals.append(oracle.gpower(A, "SL0", [gamma], tol=1e-14, maxit=10000, x0=x0).objective[0])
    assert max(vals) == pytest.approx(best, rel=1e-9)


# ---------------------------------------------------------------- status rules

def test_degenerate_polar_keeps_last_valid_iterate():
    """Reading of an unstated case: if one component's gamma zeroes its whole
    column of G, Y = A G is rank deficient and the solve stops with status
    DEGENERATE, returning the iterate of that sweep."""
    A = _rand(12, 30, 20)
    c = oracle.column_norms(A).max()
    gam = np.array([0.1 * c, 2.0 * c])
    r = oracle.gpower(A, "BL1", gam, mu=[1.0, 1.0])
    assert np.all(r.status == oracle.STATUS_DEGENERATE)
    assert np.all(r.iters == 1)
    X0, _ = oracle.block_start(A, 2)
    np.testing.assert_allclose(r.X, X0, atol=1e-14)
    assert np.all(r.Z[:, 1] == 0)


def test_zero_matrix_and_tiny_shapes():
    """A = 0 stops before the first sweep with status ZERO; p = 1 and n = 1 run."""
    r = oracle.gpower(np.zeros((5, 7)), "SL1", [0.1])
    assert r.status[0] == oracle.STATUS_ZERO and r.iters[0] == 0
    r = oracle.gpower(np.zeros((5, 7)), "BL0", [0.1, 0.1], mu=[1, 1])
    assert np.all(r.status == oracle.STATUS_ZERO)
    A = _rand(1, 9, 3)
    r = oracle.gpower(A, "SL0", oracle.gamma_from_rho(A, "SL0", 0.3))
    assert abs(abs(r.X[0, 0]) - 1) < 1e-15
    A = _rand(9, 1, 3)
    r = oracle.gpower(A, "SL1", [0.0])
    assert r.Z[0, 0] == pytest.approx(1.0) or r.Z[0, 0] == pytest.approx(-1.0)
    np.testing.assert_allclose(np.abs(r.X[:, 0]), np.abs(A[:, 0]) / np.linalg.norm(A), atol=1e-15)


def test_input_validation():
    A = _rand(4, 6, 0)
    with pytest.raises(ValueError):
        oracle.gpower(A, "XX", [0.1])
    with pytest.raises(ValueError):
        oracle.gpower(A, "SL1", [-0.1])
    with pytest.raises(ValueError):
        oracle.gpower(A, "BL1", [0.1] * 5, mu=[1] * 5)  # m > p
    with pytest.raises(ValueError):
        oracle.gpower(A, "BL1", [0.1, 0.1], mu=[1, 0])
    with pytest.raises(ValueError):
        oracle.gpower(A, "SL1", [0.1], mu=[2.0])
    B = A.copy()
    B[0, 0] = np.nan
    with pytest.raises(ValueError):
        oracle.gpower(B, "SL1", [0.1])


# ---------------------------------------------------------------- gamma path

def test_gamma_path_equals_independent_solves():
    """Single-unit forms with m gammas are m independent solves from one x0."""
    A = _rand(20, 60, 21)
    g = oracle.gamma_from_rho(A, "SL1", [0.05, 0.2, 0.35])
    path = oracle.gpower(A, "SL1", g, tol=1e-8)
    for j in range(3):
        one = oracle.gpower(A, "SL1", g[j : j + 1], tol=1e-8)
        np.testing.assert_array_equal(path.X[:, j], one.X[:, 0])
        np.testing.assert_array_equal(path.Z[:, j], one.Z[:, 0])
        assert path.iters[j] == one.iters[0]


# ---------------------------------------------------------------- planted recovery

def test_planted_spike_support_recovery():
    """Statistical sanity (not parity): on strong planted sparse spikes the
    single-unit solutions recover the first spike's support exactly and the
    block solutions (PCA start) recover all three supports, one per component."""
    At, meta = synth.planted_spike(400, 3000, 3, [40.0, 20.0, 13.3], support_frac=0.05,
                                   seed=0, dtype=np.float64, with_meta=True)
    A = At.T
    for form in ("SL1", "SL0"):
        g = oracle.gamma_from_rho(A, form, 0.1)
        r = oracle.gpower(A, form, g)
        assert r.status[0] == oracle.STATUS_CONVERGED
        assert set(np.flatnonzero(r.Z[:, 0])) == set(meta.supports[0].tolist())
    c = oracle.column_norms(A).max()
    for form in ("BL1", "BL0"):
        for mu in (np.ones(3), np.array([1.0, 0.8, 0.6])):
            g = np.full(3, 0.1 * c) if form == "BL1" else np.full(3, (0.1 * c) ** 2)
            r = oracle.gpower(A, form, g, mu=mu)
            assert r.status[0] == oracle.STATUS_CONVERGED
            found = [set(np.flatnonzero(r.Z[:, j]).tolist()) for j in range(3)]
            assert found == [set(sp.tolist()) for sp in meta.supports]


# ---------------------------------------------------------------- block start

def test_splitmix64_published_outputs():
    """SplitMix64 seeded with 0: the published first outputs of the generator."""
    out = oracle.splitmix64(0, np.arange(1, 4, dtype=np.uint64))
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sketch_is_balanced_rademacher():
    S = oracle.sketch_signs(4000, 8)
    assert set(np.unique(S)) == {-1.0, 1.0}
    assert abs(S.mean()) < 0.03
    np.testing.assert_array_equal(S, oracle.sketch_signs(4000, 8))
    np.testing.assert_array_equal(S[:100, :3], oracle.sketch_signs(100, 3))  # entries depend on (r, j) only


def test_block_start_rayleigh_ritz_and_svd_limit():
    """The start X0 = Q V is orthonormal and diagonalises A A^T on its span
    with non-increasing Ritz values; with many power steps it is the top-m
    left singular vectors of A (independent SVD), signed by the rule."""
    A, U, V = _low_rank_plus_noise(30, 80, [12.0, 8.0, 5.0, 3.0], seed=5, noise=0.1)
    X0, st = oracle.block_start(A, 3)
    assert st is None
    np.testing.assert_allclose(X0.T @ X0, np.eye(3), atol=1e-13)
    R = X0.T @ A @ A.T @ X0
    np.testing.assert_allclose(R - np.diag(np.diag(R)), 0.0, atol=1e-9 * np.abs(R).max())
    assert np.all(np.diff(np.diag(R)) <= 1e-9 * np.abs(R).max())
    Xl, _ = oracle.block_start(A, 3, steps=300)
    Us = np.linalg.svd(A)[0][:, :3]
    for j in range(3):
        assert abs(Xl[:, j] @ Us[:, j]) == pytest.approx(1.0, abs=1e-10)


def test_block_start_rank_deficient_is_degenerate():
    A = np.outer(np.arange(1.0, 7.0), np.ones(10))  # rank one, m = 2
    X0, st = oracle.block_start(A, 2)
    assert st == oracle.STATUS_DEGENERATE
    r = oracle.gpower(A, "BL1", [0.1, 0.1], mu=[1, 1])
    assert np.all(r.status == oracle.STATUS_DEGENERATE) and np.all(r.iters == 0)


def test_gamma_from_rho_hand_values():
    """Relative gamma (reading of Section 4.1's unitless values): rho times the
    largest column norm for L1, its square for L0.  On A = [[3, 0], [4, 1]]
    the columns have norms 5 and 1 (the rows 3 and sqrt 17, the whole matrix
    sqrt 26), so a row norm, a Frobenius norm, or rho * max||a_i||^2 for L0
    all give other numbers than the hand values below."""
    A = np.array([[3.0, 0.0], [4.0, 1.0]])
    np.testing.assert_array_equal(oracle.gamma_from_rho(A, "SL1", 0.1), [0.5])
    np.testing.assert_array_equal(oracle.gamma_from_rho(A, "BL1", [0.1, 0.2]), [0.5, 1.0])
    np.testing.assert_allclose(oracle.gamma_from_rho(A, "SL0", 0.1), [0.25], rtol=1e-15)
    np.testing.assert_allclose(oracle.gamma_from_rho(A, "BL0", [0.1, 0.4]), [0.25, 4.0], rtol=1e-15)
    # the largest column may come last
    B = np.array([[0.0, 3.0], [1.0, 4.0]])
    np.testing.assert_array_equal(oracle.gamma_from_rho(B, "SL1", 1.0), [5.0])
    np.testing.assert_allclose(oracle.gamma_from_rho(B, "SL0", 1.0), [25.0], rtol=1e-15)
