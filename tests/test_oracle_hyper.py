"""Pins of the oracle's Normal-Wishart hyper-parameter draw.

The hyper step (Alg. 1, "sample hyper-parameters ... based on U/V") draws
Lambda ~ Wishart(W*, nu*) and mu ~ N(mu*, (beta* Lambda)^{-1}) with the
posterior parameters of the BPMF Normal-Wishart hyperprior.  The checks use
closed-form Wishart moments, E = nu W and Var(L_ij) = nu (W_ij^2 + W_ii W_jj),
with W* computed here by numpy from its definition, and the whitened mean draw.
"""
import numpy as np

import oracle


def _setup(K=3, n=40, seed=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, K)) @ rng.standard_normal((K, K)) * 0.5 + 0.3
    xbar = X.mean(0)
    S = np.cov(X.T, bias=True)
    beta0, nu0 = 2.0, float(K)
    mu0 = np.array([0.1, -0.2, 0.05])[:K]
    W0 = np.eye(K) + 0.2 * np.ones((K, K))
    return n, xbar, S, beta0, nu0, mu0, W0


def _posterior(n, xbar, S, beta0, nu0, mu0, W0):
    beta_s, nu_s = beta0 + n, nu0 + n
    mu_s = (beta0 * mu0 + n * xbar) / beta_s
    d = (mu0 - xbar)[:, None]
    Wsinv = np.linalg.inv(W0) + n * S + beta0 * n / beta_s * (d @ d.T)
    return beta_s, nu_s, mu_s, np.linalg.inv(Wsinv)


def test_wishart_moments_and_mean_draw():
    n, xbar, S, beta0, nu0, mu0, W0 = _setup()
    K = len(xbar)
    beta_s, nu_s, mu_s, Ws = _posterior(n, xbar, S, beta0, nu0, mu0, W0)
    W0inv = np.linalg.inv(W0)
    draws = 20_000
    Lams = np.empty((draws, K, K))
    white = np.empty((draws, K))
    for s in range(draws):
        Lam, mu = oracle.nw_draw(n, xbar, S, beta0, nu0, mu0, W0inv, seed=4, sweep=s,
                                 c3_normals=4, c3_gamma=6)
        Lams[s] = Lam
        # whitening: chol(beta* Lambda)^T (mu - mu*) ~ N(0, I)
        white[s] = np.linalg.cholesky(beta_s * Lam).T @ (mu - mu_s)
    np.testing.assert_allclose(Lams, np.transpose(Lams, (0, 2, 1)), rtol=0, atol=1e-12)
    mean = nu_s * Ws
    var = nu_s * (Ws**2 + np.outer(np.diag(Ws), np.diag(Ws)))
    se = np.sqrt(var / draws)
    assert np.all(np.abs(Lams.mean(0) - mean) < 5 * se)
    emp_var = Lams.var(0)
    # relative error of a sample variance ~ sqrt(2/n) for near-Gaussian entries (nu* = 43)
    assert np.all(np.abs(emp_var / var - 1.0) < 6 * np.sqrt(2.0 / draws) * 1.5)
    assert np.all(np.abs(white.mean(0)) < 5 / np.sqrt(draws))
    np.testing.assert_allclose(np.cov(white.T), np.eye(K), atol=5 * np.sqrt(2.0 / draws))


def test_wishart_reduces_to_chi_square_for_k1():
    # K = 1: Lambda = W* chi^2(nu*), mu | Lambda ~ N(mu*, 1/(beta* Lambda))
    n, xbar, S = 10, np.array([0.5]), np.array([[2.0]])
    beta0, nu0, mu0, W0 = 1.0, 1.0, np.array([0.0]), np.array([[1.0]])
    beta_s, nu_s, mu_s, Ws = _posterior(n, xbar, S, beta0, nu0, mu0, W0)
    lam = np.array([oracle.nw_draw(n, xbar, S, beta0, nu0, mu0, np.linalg.inv(W0), 8, s, 5, 7)[0][0, 0]
                    for s in range(20_000)])
    from scipy import stats
    assert stats.kstest(lam / Ws[0, 0], "chi2", args=(nu_s,)).pvalue > 1e-4


def test_nw_draw_is_deterministic_in_counters():
    n, xbar, S, beta0, nu0, mu0, W0 = _setup()
    W0inv = np.linalg.inv(W0)
    a = oracle.nw_draw(n, xbar, S, beta0, nu0, mu0, W0inv, 4, 9, 4, 6)
    b = oracle.nw_draw(n, xbar, S, beta0, nu0, mu0, W0inv, 4, 9, 4, 6)
    c = oracle.nw_draw(n, xbar, S, beta0, nu0, mu0, W0inv, 4, 10, 4, 6)
    np.testing.assert_array_equal(a[0], b[0])
    assert not np.allclose(a[0], c[0])
