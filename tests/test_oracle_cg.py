"""Pins for Alg. 2 (ParallelConjGradient) with the diagonal preconditioner."""
import numpy as np
import pytest

from oracle.cofem import pcg


def _system(N, D, beta, seed, alpha_spread=(0.1, 1e4)):
    rng = np.random.default_rng(seed)
    Phi = rng.standard_normal((N, D)) / np.sqrt(N)
    alpha = np.exp(rng.uniform(np.log(alpha_spread[0]), np.log(alpha_spread[1]), D))
    A = beta * Phi.T @ Phi + np.diag(alpha)
    theta = (Phi ** 2).sum(axis=0)
    minv = 1.0 / (beta * theta + alpha)
    return A, minv


def test_pcg_matches_direct_solve_within_condition_bound():
    A, minv = _system(30, 80, 50.0, 1)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((80, 5))
    tol = 1e-8
    X, iters, flags = pcg(lambda V: A @ V, B, minv, tol, 500)
    assert flags == 0
    Xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    rel = np.linalg.norm(X - Xs, axis=0) / np.linalg.norm(Xs, axis=0)
    # ||x - x*|| / ||x*|| <= kappa(A) ||r|| / ||b||
    assert np.all(rel <= kappa * tol)
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= tol * (1 + 1e-6))


def test_pcg_error_bound_every_iteration():
    """Lemma (CG convergence) for the preconditioned system:
    ||e_u||_A <= 2 ((sqrt k' - 1)/(sqrt k' + 1))^u ||e_0||_A, k' = kappa(M^-1/2 A M^-1/2).
    A wrong direction update (e.g. P <- R + eta P with M != I) breaks it."""
    A, minv = _system(40, 60, 200.0, 3)
    rng = np.random.default_rng(4)
    b = rng.standard_normal((60, 1))
    xs = np.linalg.solve(A, b)
    Ms = np.sqrt(minv)
    Ap = Ms[:, None] * A * Ms[None, :]
    ev = np.linalg.eigvalsh(Ap)
    kp = ev[-1] / ev[0]
    q = (np.sqrt(kp) - 1.0) / (np.sqrt(kp) + 1.0)
    hist = []
    pcg(lambda V: A @ V, b, minv, 1e-13, 200, history=hist)
    e0 = float(np.sqrt(xs[:, 0] @ A @ xs[:, 0]))
    assert len(hist) > 3
    for u, X in enumerate(hist, start=1):
        e = xs[:, 0] - X[:, 0]
        eA = float(np.sqrt(max(e @ A @ e, 0.0)))
        assert eA <= 2.0 * q ** u * e0 * (1 + 1e-6) + 1e-12 * e0


def test_cg_identity_preconditioner_finite_termination():
    """With M = I, Alg. 2 is textbook CG: exact in at most D steps."""
    rng = np.random.default_rng(5)
    D = 12
    G = rng.standard_normal((D, D))
    A = G @ G.T + D * np.eye(D)
    b = rng.standard_normal((D, 2))
    X, iters, _ = pcg(lambda V: A @ V, b, np.ones(D), 1e-13, D)
    np.testing.assert_allclose(X, np.linalg.solve(A, b), rtol=1e-9)


def test_jacobi_on_diagonal_system_converges_in_one_step():
    d = np.linspace(1.0, 1e6, 50)
    B = np.random.default_rng(6).standard_normal((50, 3))
    X, iters, _ = pcg(lambda V: d[:, None] * V, B, 1.0 / d, 1e-12, 50)
    assert iters == 1
    np.testing.assert_allclose(X, B / d[:, None], rtol=1e-14)


def test_zero_rhs_column_starts_converged():
    A, minv = _system(10, 20, 5.0, 7)
    B = np.zeros((20, 2))
    B[:, 1] = 1.0
    X, iters, flags = pcg(lambda V: A @ V, B, minv, 1e-10, 100)
    assert np.all(X[:, 0] == 0.0)
    np.testing.assert_allclose(X[:, 1], np.linalg.solve(A, B[:, 1]), rtol=1e-8)


def test_per_column_masking_and_frobenius():
    A, minv = _system(30, 70, 1e4, 8)
    rng = np.random.default_rng(9)
    B = rng.standard_normal((70, 4))
    B[:, 0] *= 1e4            # a large-norm column (like beta Phi^T y)
    tol = 1e-6
    X, it_pc, _ = pcg(lambda V: A @ V, B, minv, tol, 1000, conv="per_column")
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(res <= tol * (1 + 1e-6))
    Xf, it_f, _ = pcg(lambda V: A @ V, B, minv, tol, 1000, conv="frobenius")
    assert np.linalg.norm(B - A @ Xf) / np.linalg.norm(B) <= tol * (1 + 1e-6)


def test_residual_replacement_keeps_solution():
    A, minv = _system(30, 70, 1e3, 10)
    B = np.random.default_rng(11).standard_normal((70, 3))
    X1, it1, _ = pcg(lambda V: A @ V, B, minv, 1e-9, 500)
    X2, it2, _ = pcg(lambda V: A @ V, B, minv, 1e-9, 500, rr_period=5)
    Xs = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    for X in (X1, X2):
        assert np.all(np.linalg.norm(X - Xs, axis=0) / np.linalg.norm(Xs, axis=0) <= kappa * 1e-9)
    assert it2 <= 1.2 * it1 + 5          # replacement must not stall the iteration


def test_maxit_sets_flag():
    A, minv = _system(30, 70, 1e3, 12)
    B = np.random.default_rng(13).standard_normal((70, 2))
    _, iters, flags = pcg(lambda V: A @ V, B, minv, 1e-14, 3)
    assert iters == 3 and flags & 1


def test_breakdown_flagged_and_column_frozen():
    """Alg. 2 divides by pi_q = p_q^T A p_q, which a symmetric positive
    definite A keeps positive.  On an indefinite A a column whose first
    direction has p^T A p < 0 cannot take a CG step: it is flagged and frozen
    at X = 0, while a column that only sees the positive part still solves."""
    from oracle.cofem import FLAG_BREAKDOWN
    d = np.array([1.0, 2.0, -1.0])
    B = np.zeros((3, 2))
    B[0, 0] = 1.0          # column 0: e_1, in the positive part (one step, exact)
    B[2, 1] = 1.0          # column 1: e_3, p^T A p = -1
    X, iters, flags = pcg(lambda V: d[:, None] * V, B, np.ones(3), 1e-12, 10)
    assert flags & FLAG_BREAKDOWN
    np.testing.assert_allclose(X[:, 0], [1.0, 0.0, 0.0], rtol=1e-15)
    assert np.all(X[:, 1] == 0.0)
    assert iters == 1


def test_breakdown_on_non_finite_pi():
    """A non-finite pi_q is a breakdown too.  An infinite entry of M^-1 (a zero
    diagonal of the preconditioner) makes W = M^-1 R infinite where R is not
    zero and NaN (inf * 0) where it is, so every column's pi is +inf or NaN:
    all are flagged and frozen at X = 0, and no NaN reaches X."""
    from oracle.cofem import FLAG_BREAKDOWN
    D = 6
    d = np.linspace(1.0, 3.0, D)
    minv = 1.0 / d
    minv[2] = np.inf
    B = np.zeros((D, 2))
    B[:, 0] = 1.0          # R[2] != 0: W[2] = inf, pi = +inf
    B[0, 1] = 1.0          # R[2] == 0: W[2] = NaN, pi = NaN
    with np.errstate(invalid="ignore", over="ignore"):
        X, iters, flags = pcg(lambda V: d[:, None] * V, B, minv, 1e-12, 10)
    assert flags & FLAG_BREAKDOWN
    assert np.all(X == 0.0)
    assert iters == 1


def test_true_residual_check_restarts_a_column_that_misses_tol():
    """Reading 11's check: a column whose recursive residual met tol while its
    true residual did not (here forced by an operator that is off by a
    perturbation inside the CG loop only) restarts from the true residual and
    ends within tol of the exact solve; the reported true residuals are those
    of the returned X."""
    A, minv = _system(30, 70, 1e3, 14)
    B = np.random.default_rng(15).standard_normal((70, 3))
    rng = np.random.default_rng(16)
    E = 1e-4 * rng.standard_normal((70, 70))
    calls = {"n": 0}

    def perturbed(V):          # wrong operator for the first 60 applications
        calls["n"] += 1
        return (A + E) @ V if calls["n"] <= 60 else A @ V

    info = {}
    X, iters, flags = pcg(perturbed, B, minv, 1e-9, 500, check=True, info=info)
    res = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert flags == 0
    assert np.all(res <= 1e-9 * (1 + 1e-6))
    np.testing.assert_allclose(info["true_res"], res, rtol=1e-6)
    # without the check the same run returns an X whose true residual misses tol
    calls["n"] = 0
    X0, _, _ = pcg(perturbed, B, minv, 1e-9, 500)
    assert np.max(np.linalg.norm(B - A @ X0, axis=0) / np.linalg.norm(B, axis=0)) > 1e-8


def test_true_residual_check_reports_without_restart_in_fp64():
    """With an exact operator the FP64 recursive residual tracks the true
    one: the check restarts nothing and reports residuals below tol."""
    A, minv = _system(30, 70, 1e3, 17)
    B = np.random.default_rng(18).standard_normal((70, 4))
    info = {}
    X1, it1, f1 = pcg(lambda V: A @ V, B, minv, 1e-8, 500, check=True, info=info)
    X2, it2, f2 = pcg(lambda V: A @ V, B, minv, 1e-8, 500)
    assert it1 == it2 and f1 == f2 == 0
    np.testing.assert_array_equal(X1, X2)
    assert np.all(info["true_res"] <= 1e-8 * (1 + 1e-6))


def test_warm_start_from_the_solution_takes_one_step():
    """x0 = A^-1 B: the initial residual is rounding level, the first update
    keeps X there and the column stops after one step."""
    A, minv = _system(30, 70, 1e3, 19)
    B = np.random.default_rng(20).standard_normal((70, 3))
    Xs = np.linalg.solve(A, B)
    X, iters, flags = pcg(lambda V: A @ V, B, minv, 1e-9, 100, x0=Xs)
    assert iters == 1 and flags == 0
    np.testing.assert_allclose(X, Xs, rtol=1e-9)


def test_warm_start_converges_to_the_same_solution():
    A, minv = _system(30, 70, 1e3, 21)
    rng = np.random.default_rng(22)
    B = rng.standard_normal((70, 3))
    Xs = np.linalg.solve(A, B)
    X, iters, flags = pcg(lambda V: A @ V, B, minv, 1e-10, 500, x0=rng.standard_normal((70, 3)))
    assert flags == 0
    kappa = np.linalg.cond(A)
    assert np.all(np.linalg.norm(X - Xs, axis=0) / np.linalg.norm(Xs, axis=0) <= kappa * 1e-10)
