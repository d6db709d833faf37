"""Pins for the oracle's dictionary operators (Sec. V-A "Dictionary", Sec. VI-A)."""
import numpy as np
import pytest

from oracle.operators import DenseOperator, ToeplitzOperator, apply_A
from synth import double_exponential_filter


def _explicit_toeplitz(h, N):
    """Column j holds h delayed by j samples, truncated at N (loop form)."""
    L = len(h)
    Phi = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            tau = i - j
            if 0 <= tau < L:
                Phi[i, j] = h[tau]
    return Phi


@pytest.mark.parametrize("N,L", [(50, 7), (300, 256), (257, 256), (10, 16)])
def test_toeplitz_fft_matches_convolve_and_matrix(N, L):
    rng = np.random.default_rng(N + L)
    h = rng.standard_normal(L)
    op = ToeplitzOperator(h, N)
    Phi = _explicit_toeplitz(h, N)
    V = rng.standard_normal((N, 3))
    np.testing.assert_allclose(op.apply(V), Phi @ V, atol=1e-12)
    np.testing.assert_allclose(op.apply_t(V), Phi.T @ V, atol=1e-12)
    # np.convolve route (linear convolution truncated to N samples)
    np.testing.assert_allclose(op.apply(V[:, 0]), np.convolve(V[:, 0], h)[:N], atol=1e-12)
    np.testing.assert_allclose(op.column_sq_norms(), (Phi ** 2).sum(axis=0), atol=1e-12)
    np.testing.assert_allclose(op.dense(), Phi)


def test_calcium_filter_shape():
    h = double_exponential_filter(256)
    assert h[0] == 0.0
    assert int(np.argmax(h)) == 10
    assert abs(float(h.max()) - 0.697) < 1e-3
    # the last column of the D x D convolution is h[0] alone -> zero
    op = ToeplitzOperator(h, 600)
    assert op.column_sq_norms()[-1] == 0.0


def test_dense_apply_matches_loops():
    rng = np.random.default_rng(3)
    Phi = rng.standard_normal((5, 7))
    op = DenseOperator(Phi)
    v = rng.standard_normal(7)
    u = rng.standard_normal(5)
    want = [sum(Phi[i, j] * v[j] for j in range(7)) for i in range(5)]
    np.testing.assert_allclose(op.apply(v), want, atol=1e-12)
    want_t = [sum(Phi[i, j] * u[i] for i in range(5)) for j in range(7)]
    np.testing.assert_allclose(op.apply_t(u), want_t, atol=1e-12)
    np.testing.assert_allclose(op.column_sq_norms(), [sum(Phi[i, j] ** 2 for i in range(5)) for j in range(7)])


def test_apply_A_matches_explicit_matrix():
    rng = np.random.default_rng(4)
    Phi = rng.standard_normal((6, 9))
    alpha = rng.uniform(0.1, 3.0, 9)
    beta = 2.5
    A = beta * Phi.T @ Phi + np.diag(alpha)
    V = rng.standard_normal((9, 4))
    np.testing.assert_allclose(apply_A(DenseOperator(Phi), V, alpha, beta), A @ V, atol=1e-12)


def test_dct_operator_matches_its_definition_and_is_orthonormal():
    """Sec. V-A "DCT": Phi = M Omega^-1.  The fast transforms agree with the
    matrix written from the DCT-II definition, Phi^T is the adjoint, the kept
    rows are orthonormal (Phi Phi^T = I_N), and with all rows kept
    Phi^T Phi = I_D."""
    from oracle import DCTOperator
    rng = np.random.default_rng(0)
    D = 96
    rows = np.sort(rng.choice(D, size=D // 3, replace=False))
    op = DCTOperator(D, rows)
    Phi = op.dense()
    V = rng.standard_normal((D, 3))
    U = rng.standard_normal((D // 3, 3))
    np.testing.assert_allclose(op.apply(V), Phi @ V, atol=1e-12)
    np.testing.assert_allclose(op.apply_t(U), Phi.T @ U, atol=1e-12)
    np.testing.assert_allclose(Phi @ Phi.T, np.eye(D // 3), atol=1e-12)
    np.testing.assert_allclose(op.column_sq_norms(), np.sum(Phi ** 2, axis=0), atol=1e-12)
    full = DCTOperator(D, np.arange(D)).dense()
    np.testing.assert_allclose(full.T @ full, np.eye(D), atol=1e-12)


def test_dct_dictionary_with_all_rows_gives_the_orthonormal_closed_form():
    """Phi^T Phi = I: A = diag(beta + alpha), so Jacobi-preconditioned CG
    converges in one step, mu_j = beta (Phi^T y)_j / (beta + alpha_j) and
    s_j = 1 / (beta + alpha_j) for any probes (the orthonormal case of
    Sec. III-C's preconditioner)."""
    from oracle import DCTOperator, cofem
    rng = np.random.default_rng(1)
    D = 128
    op = DCTOperator(D, np.arange(D))
    y = rng.standard_normal(D)
    beta = 50.0
    alpha0 = np.exp(rng.uniform(-1, 2, D))
    r = cofem(op, y, beta, 6, 1, 1e-12, 50, seed=2, alpha0=alpha0)
    assert np.all(r["cg_iters"] == 1)
    np.testing.assert_allclose(r["mu"], beta * op.apply_t(y) / (beta + alpha0), rtol=1e-10)
    np.testing.assert_allclose(r["s"], 1.0 / (beta + alpha0), rtol=1e-10)
