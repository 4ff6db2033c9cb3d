"""Pins of the oracle's per-row conditional and linear algebra.

The per-row update (Alg. 1 inner loops; Sec. 3.1) is the exact Gaussian
conditional of the BPMF model.  These tests check it against routines the
oracle does not use (numpy/LAPACK Cholesky, solve and inverse), against the
prior for degree-0 rows, against brute-force quadrature for K = 1, and
against Monte-Carlo moments of many draws.
"""
import math

import numpy as np
import pytest

import oracle


def _spd(rng, K, cond=10.0):
    Q, _ = np.linalg.qr(rng.standard_normal((K, K)))
    ev = np.exp(np.linspace(0, math.log(cond), K))
    return (Q * ev) @ Q.T


@pytest.mark.parametrize("K", [1, 2, 5, 16, 64])
def test_cholesky_matches_lapack(K):
    rng = np.random.default_rng(K)
    A = _spd(rng, K, 1e3)
    L = oracle.cholesky(A)
    np.testing.assert_allclose(L, np.linalg.cholesky(A), rtol=1e-10, atol=1e-12)
    assert np.all(np.triu(L, 1) == 0.0)


def test_cholesky_rejects_indefinite():
    with pytest.raises(RuntimeError):
        oracle.cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))


@pytest.mark.parametrize("K", [1, 3, 10])
def test_spd_inverse_matches_numpy(K):
    rng = np.random.default_rng(100 + K)
    A = _spd(rng, K, 50.0)
    np.testing.assert_allclose(oracle.spd_inverse(A), np.linalg.inv(A), rtol=1e-10, atol=1e-12)


def test_row_stats_match_numpy():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((257, 6)) * 3 + 1
    xbar, S = oracle.row_stats(X)
    np.testing.assert_allclose(xbar, X.mean(0), rtol=1e-12)
    np.testing.assert_allclose(S, np.cov(X.T, bias=True), rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("K", [2, 3, 4])
@pytest.mark.parametrize("d", [0, 1, 2, 5])
def test_row_conditional_closed_form(K, d):
    rng = np.random.default_rng(10 * K + d)
    LamX = _spd(rng, K, 5.0)
    muX = rng.standard_normal(K)
    alpha = 1.7
    Y = rng.standard_normal((9, K))
    idx = rng.choice(9, size=d, replace=False).astype(np.int32)
    val = rng.standard_normal(d)
    z = rng.standard_normal(K)
    mean, x = oracle.row_conditional(LamX, LamX @ muX, alpha, idx, val, Y, z)
    Yc = Y[idx]
    Lam = LamX + alpha * Yc.T @ Yc
    b = alpha * Yc.T @ val + LamX @ muX
    mu_ref = np.linalg.solve(Lam, b)
    np.testing.assert_allclose(mean, mu_ref, rtol=1e-10, atol=1e-12)
    # sample - mean = L^{-T} z with L = chol(Lambda): covariance L^{-T} L^{-1} = Lambda^{-1}
    L = np.linalg.cholesky(Lam)
    np.testing.assert_allclose(x - mean, np.linalg.solve(L.T, z), rtol=1e-10, atol=1e-12)
    if d == 0:
        np.testing.assert_allclose(mean, muX, rtol=1e-10, atol=1e-12)


def test_row_conditional_k1_quadrature():
    # K = 1: p(u) ~ exp(-alpha/2 sum (r_c - u y_c)^2 - lam/2 (u - mu)^2); integrate numerically.
    alpha, lam, mu = 3.0, 0.7, 0.4
    y = np.array([0.9, -1.3, 0.2])
    r = np.array([1.1, -0.4, 0.8])
    grid = np.linspace(-20, 20, 400_001)
    logp = -0.5 * alpha * ((r[None, :] - grid[:, None] * y[None, :]) ** 2).sum(1) \
        - 0.5 * lam * (grid - mu) ** 2
    p = np.exp(logp - logp.max())
    m_quad = np.trapezoid(grid * p, grid) / np.trapezoid(p, grid)
    v_quad = np.trapezoid((grid - m_quad) ** 2 * p, grid) / np.trapezoid(p, grid)
    z = np.array([1.0])
    mean, x = oracle.row_conditional(np.array([[lam]]), np.array([lam * mu]), alpha,
                                     np.arange(3, dtype=np.int32), r, y[:, None], z)
    assert mean[0] == pytest.approx(m_quad, rel=1e-8)
    # one unit of noise moves the sample by one standard deviation
    assert (x[0] - mean[0]) == pytest.approx(math.sqrt(v_quad), rel=1e-6)


def test_row_conditional_monte_carlo():
    # Many draws with different noise: mean -> mu_i, covariance -> Lambda_i^{-1}.
    rng = np.random.default_rng(5)
    K, n = 3, 40_000
    LamX = _spd(rng, K, 4.0)
    muX = rng.standard_normal(K)
    Y = rng.standard_normal((6, K))
    idx = np.arange(6, dtype=np.int32)
    val = rng.standard_normal(6)
    alpha = 2.0
    Z = oracle.normal_stream(77, 0, 0, 0, 0, n * K).reshape(n, K)
    xs = np.array([oracle.row_conditional(LamX, LamX @ muX, alpha, idx, val, Y, z)[1] for z in Z])
    Lam = LamX + alpha * Y.T @ Y
    mu = np.linalg.solve(Lam, alpha * Y.T @ val + LamX @ muX)
    cov = np.linalg.inv(Lam)
    se = np.sqrt(np.diag(cov) / n)
    assert np.all(np.abs(xs.mean(0) - mu) < 5 * se)
    emp = np.cov(xs.T)
    tol = 5 * np.sqrt((np.outer(np.diag(cov), np.diag(cov)) + cov**2) / n)
    assert np.all(np.abs(emp - cov) < tol)
