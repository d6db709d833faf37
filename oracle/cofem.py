"""Covariance-free EM (CoFEM) in FP64 on the CPU (oracle side; test infrastructure).

Follows the paper's two algorithms step by step:

Alg. 1 (CovarianceFreeEM)   for t = 1..T:
    A <- beta Phi^T Phi + diag(alpha^(t))
    draw p_1..p_K Rademacher (fresh each t)
    B <- [beta Phi^T y | p_1 .. p_K]         (mu in column 0: see "readings")
    X <- LinearSolver(A, B)
    s_j <- (1/K) sum_k p_kj x_kj            (Eq. diag-estimate)
    if t < T: alpha_j^(t+1) <- 1 / (mu_j^2 + s_j)
    return alpha^(T), mu, s

Alg. 2 (ParallelConjGradient) with the diagonal preconditioner
M = diag(beta theta + alpha) of Sec. III-C.

Readings of the paper taken here (each a choice where the text is silent,
garbled or at odds with itself):
 1. Alg. 2 initialises P <- B and updates P <- R + P H.  With M != I that is not
    preconditioned CG, while the text defines W = M^-1 R and rho = R^T W.  We use
    P_0 = W_0 = M^-1 B and P <- W + P H (standard PCG, Hestenes-Stiefel /
    Shewchuk, both cited for CG).  For M = I both readings agree.
 2. The pi_q sum is printed with index d; it is the row index j.
 3. Stopping: default is per column, delta_q = ||r_q|| / ||b_q|| <= tol with
    that column then frozen ("masked"); conv="frobenius" reproduces the
    printed global test ||R||_F / ||B||_F <= tol.  A column with ||b_q|| = 0 has
    x_q = 0 and starts converged.
 4. The test uses the unpreconditioned residual after the X, R update and
    before W.  cg_iters[t] = number of operator applications in EM iteration t
    (the largest over columns), residual-replacement applications excluded.
 5. X starts at 0 in every EM iteration (cold start, as printed).
 6. b = beta Phi^T y is computed once per fit (it does not depend on t).
 7. Probes: Philox4x64-10 rule of oracle.philox, fresh for every t.
 8. T E-steps and T-1 M-steps; the returned alpha is alpha^(T).
 9. theta: Jacobi (theta_j = ||phi_j||^2) by default, or theta = 1 ("one");
    precond="none" runs Alg. 2 unpreconditioned (M = I), the comparison of the
    paper's preconditioner study (Sec. V, empirical insights, Fig. 3b).
10. The second moment mu_j^2 + s_j can be <= 0 for finite K (s is unbiased,
    not positive); alpha_j = 1 / max(mu_j^2 + s_j, 1/alpha_max), alpha_max = 1e12.
11. Residual replacement (precision form, rr_period > 0): when the iteration
    count u is a multiple of rr_period, right after the X, R update the still
    active columns take R <- B - A X before the stopping test, then W, rho and
    P continue from that R (P is kept, as in van der Vorst and Ye's reliable
    updates).  With replacement (or check_residual) the CG loop's end is
    verified: every column's true residual B - A X meets the stopping test, or
    the column restarts from it (R <- B - A X, P <- M^-1 R) and the loop goes
    on within the same budget of maxit steps; the true residuals of the
    returned X are reported.  (In FP64 the recursive residual stays close to
    the true one, so the check rarely restarts anything here.)
12. Non-negativity (prior="rectified", the rectified Gaussian prior of the
    non-negativity subsection): the M-step takes alpha_j = 1 / E[z_j^2] with
    E[z_j^2] the second moment of N(mu_j, Sigma_jj) truncated to z_j >= 0,
    mu_j^2 + Sigma_jj + mu_j sqrt(2 Sigma_jj / pi) exp(-xi_j^2) / erfc(-xi_j),
    xi_j = mu_j / sqrt(2 Sigma_jj).  The printed third term has sqrt(Sigma_jj /
    pi); with the printed xi that is not the truncated moment the text
    describes, so the factor 2 is restored.  Sigma_jj is replaced by s_j (as
    the paper says); where s_j <= 0 the term is undefined and dropped, and the
    floor 1/alpha_max applies as in reading 10.  exp(-xi^2) / erfc(-xi) is
    evaluated as 1 / erfcx(-xi), the same function without overflow.
14. Warm start with probe reuse (beyond the paper, which starts each E-step
    at X = 0 with fresh probes): every E-step draws the probes of t = 1 and
    E-step t >= 2 starts Alg. 2 from the previous E-step's X with R = B - A X.
13. Multi-task CoFEM (cofem_multitask; multi-task subsection of Sec. III):
    the L tasks share alpha and beta; each task l draws its own probes
    (Philox counter word 3 = l; task 0 is the single-task rule), its own
    preconditioner M_l = beta theta_l + alpha, and its K+1 columns join one
    batched PCG (per-column stopping, so each task's columns stop on their
    own); cg_iters[t] is the batched loop's count, the largest over tasks.
    M-step: alpha_j = L / sum_l (mu_lj^2 + s_lj), floored at 1/alpha_max.
"""
from __future__ import annotations

import numpy as np

from .em import second_moment  # noqa: F401  (the M-step's E[z_j^2], reading 12)
from .operators import apply_A
from .philox import rademacher_probes

FLAG_CG_NOT_CONVERGED = 1
FLAG_ALPHA_CLAMPED = 2
FLAG_BREAKDOWN = 4


def diag_estimate(P, X):
    """s_j = (1/K) sum_k p_kj x_kj for Rademacher probes (Eq. diag-estimate).
    P, X: (D, K) arrays whose column k is p_k and x_k = Sigma p_k."""
    K = P.shape[1]
    return np.sum(P * X, axis=1) / K


def diag_estimate_general(P, X):
    """The general rule of Prop. 1 (Eq. single-diag-estimator):
    s_j = sum_k p_kj x_kj / sum_k p_kj^2."""
    return np.sum(P * X, axis=1) / np.sum(P * P, axis=1)


def _meets_tol(rnorm, bnorm, tol, conv):
    """Alg. 2 stopping test on residual norms: per column, or the printed
    Frobenius test applied to all columns at once."""
    if conv == "per_column":
        return rnorm <= tol * bnorm
    if conv == "frobenius":
        ok = np.linalg.norm(rnorm) <= tol * np.linalg.norm(bnorm)
        return np.full(rnorm.shape, ok)
    raise ValueError(conv)


def pcg(apply_a, B, minv, tol, maxit, conv="per_column", rr_period=0, history=None, check=False, info=None,
        x0=None):
    """Alg. 2 (ParallelConjGradient) on the D x Q block B with M^-1 = diag(minv).

    Returns (X, iters, flags).  `history`, if a list, receives a copy of X after
    every iteration (for convergence-bound tests).  check (reading 11): when
    the loop ends, every column's true residual B - A X is tested against tol;
    a column that misses it (not broken down, budget left) restarts from it
    with P = M^-1 R and the loop goes on.  `info`, if a dict, receives
    "true_res", the relative true residuals ||b_q - A x_q|| / ||b_q|| of the
    returned X (when check is set).  x0: initial X (warm start, reading 14 of
    the oracle); R starts as B - A x0."""
    B = np.asarray(B, dtype=np.float64)
    D, Q = B.shape
    minv = np.asarray(minv, dtype=np.float64)[:, None]
    if x0 is None:
        X = np.zeros((D, Q))
        R = B.copy()
    else:
        X = np.array(x0, dtype=np.float64)
        R = B - apply_a(X)
    W = minv * R
    P = W.copy()
    rho = np.sum(R * W, axis=0)
    bnorm = np.linalg.norm(B, axis=0)
    active = bnorm > 0.0
    broken = np.zeros(Q, dtype=bool)
    flags = 0
    u = 0
    true_res = None
    while True:
        while u < maxit and active.any():
            Psi = apply_a(P)                                   # Apply matrix
            pi = np.sum(P * Psi, axis=0)
            a = active
            # a CG step needs a positive, finite p^T A p (A symmetric positive
            # definite); any other value freezes the column (breakdown)
            bad = a & ~((pi > 0.0) & np.isfinite(pi))
            if np.any(bad):
                flags |= FLAG_BREAKDOWN
                broken |= bad
                active = active & ~bad
                a = active
            gamma = np.zeros(Q)
            gamma[a] = rho[a] / pi[a]
            X[:, a] += P[:, a] * gamma[a]
            R[:, a] -= Psi[:, a] * gamma[a]
            u += 1
            if rr_period > 0 and u % rr_period == 0:
                R[:, a] = (B - apply_a(X))[:, a]               # residual replacement
            rn = np.full(Q, np.inf)
            rn[a] = np.linalg.norm(R[:, a], axis=0)
            if conv == "frobenius":   # the printed test: all columns' residuals together
                rn = np.linalg.norm(R, axis=0)
            active = active & ~_meets_tol(rn, bnorm, tol, conv)
            a = active
            W = minv * R                                       # Apply preconditioner
            rho_new = np.sum(R * W, axis=0)
            eta = np.zeros(Q)
            eta[a] = rho_new[a] / rho[a]
            P[:, a] = W[:, a] + P[:, a] * eta[a]
            rho[a] = rho_new[a]
            if history is not None:
                history.append(X.copy())
        if not check:
            break
        Rt = B - apply_a(X)                                    # true residual of X
        tn = np.linalg.norm(Rt, axis=0)
        true_res = np.where(bnorm > 0.0, tn / np.where(bnorm > 0.0, bnorm, 1.0), 0.0)
        miss = (bnorm > 0.0) & ~_meets_tol(tn, bnorm, tol, conv) & ~broken
        if not miss.any() or u >= maxit:
            if miss.any():
                active = miss                                  # budget spent: not converged
            break
        R[:, miss] = Rt[:, miss]                               # restart from the true residual
        W = minv * R
        P[:, miss] = W[:, miss]
        rho[miss] = np.sum(R * W, axis=0)[miss]
        active = miss
    if active.any():
        flags |= FLAG_CG_NOT_CONVERGED
    if info is not None:
        info["true_res"] = true_res
    return X, u, flags


def cofem(op, y, beta, K, T, cg_tol, cg_maxit, seed, alpha0=None, precond="jacobi",
          alpha_max=1e12, conv="per_column", rr_period=0, probe_fn=None,
          solver="pcg", return_x=False, prior="gaussian", check_residual=False, warm_start=False):
    """Alg. 1 (CovarianceFreeEM) with Alg. 2 as the linear solver.

    op        oracle.operators.DenseOperator / ToeplitzOperator
    probe_fn  optional callable (t, K, D) -> (K, D) probe block; default is the
              Philox Rademacher rule with `seed`.
    solver    "pcg" (Alg. 2) or "direct" (exact dense solve, small D only).
    prior     "gaussian" (Eq. mstep) or "rectified" (non-negativity, reading 12).
    check_residual  true-residual check at the end of each E-step (reading 11;
              always on with rr_period > 0).
    warm_start  probe reuse and warm start (reading 14): every E-step draws the
              probes of t = 1 and E-step t >= 2 starts from the previous X.
    Returns dict(alpha, mu, s, cg_iters, flags, true_res (T x (K+1), NaN where
    not checked)[, X]).
    """
    D = op.D
    yv = np.asarray(y, dtype=np.float64)
    b = beta * op.apply_t(yv)                              # computed once per fit
    theta = op.column_sq_norms() if precond == "jacobi" else np.ones(D)
    alpha = np.ones(D) if alpha0 is None else np.asarray(alpha0, dtype=np.float64).copy()
    cg_iters = np.zeros(T, dtype=np.int64)
    true_res = np.full((T, K + 1), np.nan)
    flags = 0
    mu = s = X = None
    for t in range(1, T + 1):
        tp = 1 if warm_start else t
        probes = (rademacher_probes(seed, tp, K, D) if probe_fn is None
                  else np.asarray(probe_fn(tp, K, D), dtype=np.float64))
        B = np.empty((D, K + 1))
        B[:, 0] = b
        B[:, 1:] = probes.T
        minv = np.ones(D) if precond == "none" else 1.0 / (beta * theta + alpha)

        def apply_a(V, alpha=alpha):
            return apply_A(op, V, alpha, beta)

        if solver == "pcg":
            info = {}
            X, u, f = pcg(apply_a, B, minv, cg_tol, cg_maxit, conv=conv, rr_period=rr_period,
                          check=rr_period > 0 or check_residual, info=info,
                          x0=X if warm_start and t > 1 else None)
            cg_iters[t - 1] = u
            flags |= f
            if info["true_res"] is not None:
                true_res[t - 1] = info["true_res"]
        elif solver == "direct":
            Phi = op.dense()
            A = beta * (Phi.T @ Phi) + np.diag(alpha)
            X = np.linalg.solve(A, B)
        else:
            raise ValueError(solver)
        mu = X[:, 0].copy()
        s = diag_estimate(B[:, 1:], X[:, 1:])
        if t < T:
            m2 = second_moment(mu, s, prior)
            if np.any(m2 < 1.0 / alpha_max):
                flags |= FLAG_ALPHA_CLAMPED
            alpha = 1.0 / np.maximum(m2, 1.0 / alpha_max)
    out = dict(alpha=alpha, mu=mu, s=s, cg_iters=cg_iters, flags=flags, true_res=true_res)
    if return_x:
        out["X"] = X
    return out


def cofem_multitask(ops, ys, beta, K, T, cg_tol, cg_maxit, seed, alpha0=None, precond="jacobi",
                    alpha_max=1e12, conv="per_column", probe_fn=None, solver="pcg"):
    """Multi-task CoFEM (reading 13): Alg. 1 with L E-steps per iteration (one
    batched Alg. 2 over the L (K+1) columns; the tasks' columns are independent,
    so the batch is the L per-task solves) and the shared-alpha M-step.

    ops, ys   per-task operators (oracle.operators) and observations (one D)
    probe_fn  optional callable (t, K, D, l) -> (K, D) probe block of task l
    Returns dict(alpha, mu (L x D), s (L x D), cg_iters (T,), flags)."""
    L = len(ops)
    D = ops[0].D
    bs = [beta * op.apply_t(np.asarray(y, dtype=np.float64)) for op, y in zip(ops, ys)]
    thetas = [op.column_sq_norms() if precond == "jacobi" else np.ones(D) for op in ops]
    alpha = np.ones(D) if alpha0 is None else np.asarray(alpha0, dtype=np.float64).copy()
    cg_iters = np.zeros(T, dtype=np.int64)
    flags = 0
    mu = s = None
    for t in range(1, T + 1):
        mu = np.empty((L, D))
        s = np.empty((L, D))
        for l in range(L):
            probes = (rademacher_probes(seed, t, K, D, task=l) if probe_fn is None
                      else np.asarray(probe_fn(t, K, D, l), dtype=np.float64))
            B = np.empty((D, K + 1))
            B[:, 0] = bs[l]
            B[:, 1:] = probes.T
            if solver == "pcg":
                minv = 1.0 / (beta * thetas[l] + alpha)
                X, u, f = pcg(lambda V, op=ops[l]: apply_A(op, V, alpha, beta), B, minv, cg_tol, cg_maxit,
                              conv=conv)
                cg_iters[t - 1] = max(cg_iters[t - 1], u)
                flags |= f
            elif solver == "direct":
                Phi = ops[l].dense()
                X = np.linalg.solve(beta * (Phi.T @ Phi) + np.diag(alpha), B)
            else:
                raise ValueError(solver)
            mu[l] = X[:, 0]
            s[l] = diag_estimate(B[:, 1:], X[:, 1:])
        if t < T:
            m2 = np.sum(mu ** 2 + s, axis=0) / L
            if np.any(m2 < 1.0 / alpha_max):
                flags |= FLAG_ALPHA_CLAMPED
            alpha = 1.0 / np.maximum(m2, 1.0 / alpha_max)
    return dict(alpha=alpha, mu=mu, s=s, cg_iters=cg_iters, flags=flags)
