"""Classic EM for sparse Bayesian learning with an explicit covariance
(oracle side; test infrastructure, FP64, CPU).

Model (Sec. II-A, Eq. model): z ~ N(0, diag(alpha)^-1), y | z ~ N(Phi z, beta^-1 I).
E-step (Sec. II-B, Eq. estep-params):
    Sigma = (beta Phi^T Phi + diag(alpha))^-1,   mu = beta Sigma Phi^T y.
M-step (Eq. mstep): alpha_j <- 1 / (mu_j^2 + Sigma_jj); under the rectified
    Gaussian prior of the non-negativity subsection, 1 / E[z_j^2] of N(mu_j,
    Sigma_jj) restricted to z_j >= 0 (second_moment).
Objective (Eq. mle2): log p(y | alpha) = log N(y; 0, C_y),
    C_y = beta^-1 I + Phi diag(alpha)^-1 Phi^T  (standard Gaussian marginal).

Two independent E-step routes:
* explicit : Cholesky of the D x D matrix A = Sigma^-1.
* woodbury : the IRLS form of Sec. II-C (Eq. woodbury) with an N x N inverse.
  The printed form omits beta; with C = diag(alpha)^-1 the identity reads
      Sigma = C - C Phi^T (beta^-1 I + Phi C Phi^T)^-1 Phi C.
"""
from __future__ import annotations

import numpy as np
from scipy import special
import scipy.linalg as sla


def estep_explicit(Phi, y, beta, alpha):
    """(mu, Sigma) by a D x D Cholesky factorisation of A = beta Phi^T Phi + diag(alpha)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    A = beta * (Phi.T @ Phi) + np.diag(np.asarray(alpha, dtype=np.float64))
    c = sla.cho_factor(A, lower=True)
    Sigma = sla.cho_solve(c, np.eye(A.shape[0]))
    mu = beta * (Sigma @ (Phi.T @ np.asarray(y, dtype=np.float64)))
    return mu, Sigma


def estep_woodbury(Phi, y, beta, alpha):
    """(mu, diag Sigma) through the N x N Woodbury form (beta restored)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    c = 1.0 / np.asarray(alpha, dtype=np.float64)           # C = diag(c)
    PhiC = Phi * c[None, :]                                   # Phi C
    S = np.eye(Phi.shape[0]) / beta + PhiC @ Phi.T           # beta^-1 I + Phi C Phi^T
    cf = sla.cho_factor(S, lower=True)
    G = sla.cho_solve(cf, PhiC)                               # S^-1 Phi C
    diag = c - np.einsum("ij,ij->j", PhiC, G)                 # diag(C - C Phi^T S^-1 Phi C)
    Phity = Phi.T @ np.asarray(y, dtype=np.float64)
    # Sigma Phi^T y = C Phi^T y - C Phi^T S^-1 Phi C Phi^T y
    mu = beta * (c * Phity - PhiC.T @ sla.cho_solve(cf, PhiC @ Phity))
    return mu, diag


def log_marginal_likelihood(Phi, y, beta, alpha):
    """log p(y | alpha) of Eq. mle2 for the Gaussian model (closed form)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    N = Phi.shape[0]
    Cy = np.eye(N) / beta + (Phi / np.asarray(alpha, dtype=np.float64)[None, :]) @ Phi.T
    cf = sla.cho_factor(Cy, lower=True)
    logdet = 2.0 * np.sum(np.log(np.diag(cf[0])))
    quad = float(y @ sla.cho_solve(cf, y))
    return -0.5 * (N * np.log(2.0 * np.pi) + logdet + quad)


def second_moment(mu, s, prior="gaussian"):
    """E[z_j^2] of the M-step: mu_j^2 + Sigma_jj under the Gaussian prior (Eq.
    mstep); under the rectified Gaussian prior (non-negativity subsection) the
    second moment of N(mu_j, Sigma_jj) restricted to z_j >= 0,
    mu^2 + Sigma + mu sqrt(2 Sigma / pi) exp(-xi^2) / erfc(-xi),
    xi = mu / sqrt(2 Sigma) (the printed third term's factor 2 restored; no
    term where Sigma <= 0; exp(-xi^2) / erfc(-xi) evaluated as 1 / erfcx(-xi)).
    `s` is Sigma_jj or its estimate."""
    mu = np.asarray(mu, dtype=np.float64)
    s = np.asarray(s, dtype=np.float64)
    m2 = mu ** 2 + s
    if prior == "gaussian":
        return m2
    if prior != "rectified":
        raise ValueError(prior)
    pos = s > 0
    sp = np.where(pos, s, 1.0)
    xi = mu / np.sqrt(2.0 * sp)
    corr = mu * np.sqrt(2.0 * sp / np.pi) / special.erfcx(-xi)
    return m2 + np.where(pos, corr, 0.0)


def mstep(mu, diag_sigma, alpha_max=np.inf, prior="gaussian"):
    """alpha_j <- 1 / E[z_j^2] (Eq. mstep), with the second moment floored at
    1/alpha_max (a no-op for exact EM, where it is >= Sigma_jj > 0)."""
    m2 = second_moment(mu, diag_sigma, prior)
    return 1.0 / np.maximum(m2, 1.0 / alpha_max)


def em(Phi, y, beta, T, alpha0=None, estep="explicit", alpha_max=np.inf, track_loglik=False,
       prior="gaussian"):
    """T iterations of classic EM, laid out like Alg. 1 (T E-steps, T-1
    M-steps; returns alpha^(T) with the mu, diag Sigma of the last E-step)."""
    Phi = np.asarray(Phi, dtype=np.float64)
    D = Phi.shape[1]
    alpha = np.ones(D) if alpha0 is None else np.asarray(alpha0, dtype=np.float64).copy()
    loglik = []
    mu = dsig = None
    for t in range(1, T + 1):
        if estep == "explicit":
            mu, Sigma = estep_explicit(Phi, y, beta, alpha)
            dsig = np.diag(Sigma).copy()
        elif estep == "woodbury":
            mu, dsig = estep_woodbury(Phi, y, beta, alpha)
        else:
            raise ValueError(estep)
        if track_loglik:
            loglik.append(log_marginal_likelihood(Phi, y, beta, alpha))
        if t < T:
            alpha = mstep(mu, dsig, alpha_max, prior)
    return dict(alpha=alpha, mu=mu, diag_sigma=dsig, loglik=np.array(loglik))


def em_multitask(Phis, ys, beta, T, alpha0=None, alpha_max=np.inf):
    """Multi-task EM (multi-task subsection of Sec. III): L tasks with their own
    (y_l, Phi_l) and a shared alpha; an explicit E-step per task, then
    alpha_j <- L / sum_l (mu_lj^2 + Sigma_l,jj) (floored at 1/alpha_max).
    Returns alpha^(T) and the last E-step's mu (L x D) and diag Sigma (L x D)."""
    L = len(Phis)
    D = np.asarray(Phis[0]).shape[1]
    alpha = np.ones(D) if alpha0 is None else np.asarray(alpha0, dtype=np.float64).copy()
    mu = dsig = None
    for t in range(1, T + 1):
        mu = np.empty((L, D))
        dsig = np.empty((L, D))
        for l in range(L):
            m, S = estep_explicit(np.asarray(Phis[l], dtype=np.float64), ys[l], beta, alpha)
            mu[l], dsig[l] = m, np.diag(S)
        if t < T:
            m2 = np.sum(mu ** 2 + dsig, axis=0) / L
            alpha = 1.0 / np.maximum(m2, 1.0 / alpha_max)
    return dict(alpha=alpha, mu=mu, diag_sigma=dsig)
