"""Pins for classic EM (Sec. II-B) and its Woodbury/IRLS form (Sec. II-C)."""
import numpy as np
import pytest

from oracle.em import em, estep_explicit, estep_woodbury, log_marginal_likelihood, mstep
from synth import dense_gaussian


def test_explicit_and_woodbury_agree():
    """EM and IRLS always yield the same result (Sec. V-B); the two E-steps
    use different factorisations (D x D Cholesky vs N x N Woodbury)."""
    p = dense_gaussian(40, 120, 8, 20.0, seed=5)
    rng = np.random.default_rng(1)
    alpha = rng.uniform(0.2, 50.0, 120)
    mu1, S = estep_explicit(p.phi, p.y, p.beta, alpha)
    mu2, d2 = estep_woodbury(p.phi, p.y, p.beta, alpha)
    np.testing.assert_allclose(mu1, mu2, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(np.diag(S), d2, rtol=1e-9)
    r1 = em(p.phi, p.y, p.beta, 12, estep="explicit")
    r2 = em(p.phi, p.y, p.beta, 12, estep="woodbury")
    for k in ("alpha", "mu", "diag_sigma"):
        np.testing.assert_allclose(r1[k], r2[k], rtol=1e-7)


def test_estep_matches_definition_by_inverse():
    p = dense_gaussian(20, 30, 4, 20.0, seed=2)
    alpha = np.linspace(0.5, 3.0, 30)
    Phi = p.phi.astype(np.float64)
    Sigma_inv = np.linalg.inv(p.beta * Phi.T @ Phi + np.diag(alpha))
    mu, S = estep_explicit(p.phi, p.y, p.beta, alpha)
    np.testing.assert_allclose(S, Sigma_inv, rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(mu, p.beta * Sigma_inv @ Phi.T @ p.y.astype(np.float64), rtol=1e-8)


def test_em_loglik_monotone():
    """EM never decreases log p(y | alpha) (Sec. II-B)."""
    p = dense_gaussian(64, 256, 12, 20.0, seed=9)
    r = em(p.phi, p.y, p.beta, 30, track_loglik=True)
    ll = r["loglik"]
    assert np.all(np.diff(ll) >= -1e-8 * np.abs(ll[:-1]))
    assert ll[-1] > ll[0]


def test_loglik_matches_gaussian_density():
    from scipy.stats import multivariate_normal
    p = dense_gaussian(15, 25, 3, 20.0, seed=4)
    alpha = np.linspace(0.3, 4.0, 25)
    Phi = p.phi.astype(np.float64)
    C = np.eye(15) / p.beta + Phi @ np.diag(1.0 / alpha) @ Phi.T
    want = multivariate_normal(mean=np.zeros(15), cov=C).logpdf(p.y.astype(np.float64))
    assert abs(log_marginal_likelihood(p.phi, p.y, p.beta, alpha) - want) < 1e-8 * abs(want)


def test_orthonormal_dictionary_closed_form():
    """Phi = I: A = diag(beta + alpha), mu_j = beta y_j / (beta + alpha_j),
    Sigma_jj = 1 / (beta + alpha_j); EM is a scalar recurrence per coordinate."""
    D = 32
    rng = np.random.default_rng(0)
    y = rng.standard_normal(D)
    beta = 7.0
    T = 15
    r = em(np.eye(D), y, beta, T)
    a = np.ones(D)
    for _ in range(T - 1):
        m = beta * y / (beta + a)
        a = 1.0 / (m * m + 1.0 / (beta + a))
    np.testing.assert_allclose(r["alpha"], a, rtol=1e-12)
    np.testing.assert_allclose(r["mu"], beta * y / (beta + a), rtol=1e-12)
    np.testing.assert_allclose(r["diag_sigma"], 1.0 / (beta + a), rtol=1e-12)


def test_zero_dictionary():
    """Phi = 0: mu = 0 and Sigma = diag(alpha)^-1."""
    alpha = np.linspace(0.5, 5.0, 10)
    mu, S = estep_explicit(np.zeros((4, 10)), np.ones(4), 3.0, alpha)
    assert np.all(mu == 0.0)
    np.testing.assert_allclose(np.diag(S), 1.0 / alpha, rtol=1e-14)


def test_mstep_formula_and_clamp():
    mu = np.array([1.0, 0.0, 2.0])
    d = np.array([1.0, 1e-20, 0.25])
    np.testing.assert_allclose(mstep(mu, d, alpha_max=1e12), [0.5, 1e12, 1.0 / 4.25])


def test_theorem1_estimator_spread_on_inactive_and_active_sets():
    """Thm. 1 with Lemma 1's exact spread nu_j = sqrt((1/K) sum_{j' != j}
    Sigma_jj'^2) along exact EM: on the inactive coordinates it goes to zero
    (halving, roughly, with each doubling of t), and on the coordinates EM
    keeps (alpha_j finite) it stays below the theorem's bound
    (1/sqrt(K)) ||Theta^-1 Phi_S^T Phi_S - I||_2 / (beta sigma_min^2(Phi_S))
    with Theta = diag(Phi_S^T Phi_S)."""
    p = dense_gaussian(64, 128, 6, 40.0, seed=1)
    Phi = p.phi.astype(np.float64)
    K = 8
    inactive = np.ones(p.D, bool)
    inactive[p.support] = False
    med = []
    for T in (50, 100, 200, 400):
        a = em(Phi, p.y, p.beta, T, alpha_max=1e12)["alpha"]
        Sig = np.linalg.inv(p.beta * Phi.T @ Phi + np.diag(a))
        off = Sig - np.diag(np.diag(Sig))
        nu = np.sqrt(np.sum(off ** 2, axis=1) / K)
        med.append(np.median(nu[inactive]))
    assert all(m1 < 0.7 * m0 for m0, m1 in zip(med, med[1:])), med
    assert med[-1] < 1e-2 * np.median(nu[~inactive])
    S = a < 1e6
    PS = Phi[:, S]
    G = PS.T @ PS
    bound = (np.linalg.norm(np.diag(1.0 / np.diag(G)) @ G - np.eye(S.sum()), 2)
             / (p.beta * np.linalg.svd(PS, compute_uv=False).min() ** 2) / np.sqrt(K))
    assert np.all(nu[S] <= bound), (nu[S].max(), bound)


def test_theorem2_jacobi_preconditioned_condition_number_stays_bounded():
    """Thm. 2's mechanism along exact EM: kappa(A^(t)) grows without bound
    (alpha_j -> infinity off the support), while the Jacobi-preconditioned
    A' = M^-1/2 A M^-1/2, M = diag(beta theta + alpha), stays below
    (1 + delta) / (1 - delta), delta = ||Theta^-1 Phi_S^T Phi_S - I||_2 over
    the coordinates EM keeps (alpha_j finite)."""
    p = dense_gaussian(200, 400, 5, 40.0, seed=1)
    Phi = p.phi.astype(np.float64)
    theta = np.sum(Phi ** 2, axis=0)
    kap = {}
    for T in (100, 400):
        a = em(Phi, p.y, p.beta, T, alpha_max=1e12)["alpha"]
        A = p.beta * Phi.T @ Phi + np.diag(a)
        m = p.beta * theta + a
        ev = np.linalg.eigvalsh(A)
        evp = np.linalg.eigvalsh(A / np.sqrt(np.outer(m, m)))
        S = a < 1e6
        G = Phi[:, S].T @ Phi[:, S]
        delta = np.linalg.norm(G / np.diag(G)[:, None] - np.eye(S.sum()), 2)
        assert delta < 1.0
        kap[T] = (ev[-1] / ev[0], evp[-1] / evp[0])
        assert kap[T][1] <= (1 + delta) / (1 - delta), (T, kap[T], delta)
    assert kap[400][0] > 4.0 * kap[100][0] and kap[400][0] > 100.0 * kap[400][1]
