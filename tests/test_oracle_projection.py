"""Pins for the oracle's projection S = B Z (samples onto sparse loadings,
Section 4.2), tied to the power iteration's fixed points rather than to the
product itself: a wrong operand, a transposed Z or a dropped column fails one
of them."""

import numpy as np
import pytest

import oracle
from paper_1312_6182_gb300 import synth


@pytest.mark.parametrize("form", ["SL1", "SL0"])
def test_single_unit_fixed_point_scores_are_the_iterate(form):
    # at the fixed point x = A g / ||A g|| with z = g / ||g||: A z = c x, c > 0
    At = synth.planted_spike(120, 400, 2, [25.0, 12.0], support_frac=0.05, seed=3, dtype=np.float64)
    A = At.T
    g = oracle.gamma_from_rho(A, form, 0.1)
    r = oracle.gpower(A, form, g, tol=1e-14, maxit=5000)
    S = oracle.project(A, r.Z)
    s = S[:, 0]
    c = s @ r.X[:, 0]
    assert c > 0
    assert np.linalg.norm(s - c * r.X[:, 0]) < 1e-9 * np.linalg.norm(s)


def test_gamma_zero_scores_are_the_singular_pair():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((30, 80))
    U, sig, Vt = np.linalg.svd(A, full_matrices=False)
    S = oracle.project(A, Vt[:2].T)
    np.testing.assert_allclose(S, U[:, :2] * sig[:2], rtol=0, atol=1e-12 * sig[0])


def test_block_scores_span_the_iterate():
    # block fixed point: X = polar(A G) and each G column is a positive multiple
    # of the Z column, so span(A Z) = span(X)
    At = synth.planted_spike(150, 500, 3, [30.0, 20.0, 12.0], support_frac=0.04, seed=6, dtype=np.float64)
    A = At.T
    g = oracle.gamma_from_rho(A, "BL1", [0.1] * 3)
    r = oracle.gpower(A, "BL1", g, mu=[1.0, 0.9, 0.8], tol=1e-14, maxit=5000)
    Q, _ = np.linalg.qr(oracle.project(A, r.Z))
    cosines = np.linalg.svd(Q.T @ r.X, compute_uv=False)
    assert np.all(cosines > 1 - 1e-9)


def test_new_samples_and_zero_loading():
    # a zero loading column scores zero; scores of new samples are linear in B
    rng = np.random.default_rng(7)
    Z = np.zeros((40, 2))
    Z[[3, 9, 17], 0] = [0.6, -0.48, 0.64]
    B1, B2 = rng.standard_normal((5, 40)), rng.standard_normal((5, 40))
    S = oracle.project(B1 + 2 * B2, Z)
    assert np.all(S[:, 1] == 0)
    np.testing.assert_allclose(S, oracle.project(B1, Z) + 2 * oracle.project(B2, Z), atol=1e-13)
    np.testing.assert_allclose(S[:, 0], (B1 + 2 * B2)[:, [3, 9, 17]] @ np.array([0.6, -0.48, 0.64]), atol=1e-13)
