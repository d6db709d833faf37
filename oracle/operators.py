"""Dictionary operators Phi, Phi^T in FP64 (oracle side; test infrastructure).

CoFEM only needs Phi and Phi^T applied to blocks of vectors (Sec. III-B: CG needs
A v = beta Phi^T (Phi v) + diag(alpha) v, never A itself).

* DenseOperator   : Phi is an explicit N x D matrix (Sec. V-A "Dense Gaussian").
* ToeplitzOperator: Phi is the causal convolution with a length-L filter h,
  N = D; column j of Phi is h delayed by j samples and truncated at N
  (Sec. V-A "Convolutional", Sec. VI-A).  Applied by FFT in FP64, as the paper
  does for calcium deconvolution (Sec. VI-A "Spike Inference").
* DCTOperator     : Phi = M Omega^-1 with Omega the orthonormal 1-D DCT of
  size D and M the selection of N of its D outputs (Sec. V-A "DCT").
  Applied with scipy's fast DCT; the explicit matrix (dense()) is written
  from the DCT-II definition.
"""
from __future__ import annotations

import numpy as np


class DenseOperator:
    def __init__(self, phi):
        self.phi = np.asarray(phi, dtype=np.float64)
        self.N, self.D = self.phi.shape

    def apply(self, V):
        """Phi @ V for V of shape (D,) or (D, Q)."""
        return self.phi @ V

    def apply_t(self, U):
        """Phi^T @ U for U of shape (N,) or (N, Q)."""
        return self.phi.T @ U

    def column_sq_norms(self):
        """theta_j = sum_i Phi_ij^2 (Jacobi choice of theta, Sec. III-C)."""
        return np.einsum("ij,ij->j", self.phi, self.phi)

    def dense(self):
        return self.phi


class ToeplitzOperator:
    """(Phi v)_i = sum_{tau=0}^{L-1} h[tau] v[i - tau]  (zero for i - tau < 0),
    (Phi^T u)_j = sum_{tau=0}^{L-1} h[tau] u[j + tau]  (zero for j + tau >= N)."""

    def __init__(self, h, N):
        self.h = np.asarray(h, dtype=np.float64)
        self.L = self.h.shape[0]
        self.N = self.D = int(N)
        n = 1
        while n < self.N + self.L - 1:
            n *= 2
        self._n = n
        self._H = np.fft.rfft(self.h, n)

    def _fft_apply(self, V, spectrum):
        V = np.asarray(V, dtype=np.float64)
        out = np.fft.irfft(np.fft.rfft(V, self._n, axis=0) * (spectrum[:, None] if V.ndim == 2 else spectrum),
                           self._n, axis=0)
        return out[: self.N]

    def apply(self, V):
        return self._fft_apply(V, self._H)

    def apply_t(self, U):
        # circular correlation with zero padding n >= N + L - 1 equals the
        # truncated linear correlation on [0, N)
        return self._fft_apply(U, np.conj(self._H))

    def column_sq_norms(self):
        """theta_j = sum of h[tau]^2 over the taps of column j that fall inside
        the N rows: tau < min(L, N - j)."""
        c = np.concatenate([[0.0], np.cumsum(self.h ** 2)])
        j = np.arange(self.D)
        return c[np.minimum(self.L, self.N - j)]

    def dense(self):
        """Explicit N x D matrix (small N only; for tests)."""
        Phi = np.zeros((self.N, self.D))
        for j in range(self.D):
            m = min(self.L, self.N - j)
            Phi[j:j + m, j] = self.h[:m]
        return Phi


class DCTOperator:
    """Phi = M Omega^-1: Omega is the orthonormal DCT-II of size D,
    Omega_kn = c_k cos(pi k (2n + 1) / (2D)), c_0 = sqrt(1/D), c_k = sqrt(2/D);
    Omega^-1 = Omega^T; M keeps the rows `rows` (N distinct indices < D) of
    Omega^-1 v."""

    def __init__(self, D, rows):
        self.D = int(D)
        self.rows = np.asarray(rows, dtype=np.int64)
        self.N = self.rows.shape[0]

    def apply(self, V):
        from scipy import fft
        return fft.idct(np.asarray(V, dtype=np.float64), type=2, norm="ortho", axis=0)[self.rows]

    def apply_t(self, U):
        from scipy import fft
        U = np.asarray(U, dtype=np.float64)
        full = np.zeros((self.D,) + U.shape[1:])
        full[self.rows] = U
        return fft.dct(full, type=2, norm="ortho", axis=0)

    def dense(self):
        """Explicit N x D matrix: row i of Omega^-1 is column i of Omega."""
        n = self.rows[:, None].astype(np.float64)
        k = np.arange(self.D, dtype=np.float64)[None, :]
        c = np.where(k == 0, np.sqrt(1.0 / self.D), np.sqrt(2.0 / self.D))
        return c * np.cos(np.pi * k * (2.0 * n + 1.0) / (2.0 * self.D))

    def column_sq_norms(self):
        return np.sum(self.dense() ** 2, axis=0)


def make_operator(kind: str, phi, N: int):
    if kind == "dense":
        return DenseOperator(phi)
    if kind == "toeplitz":
        return ToeplitzOperator(phi, N)
    raise ValueError(kind)


def apply_A(op, V, alpha, beta):
    """A V = beta Phi^T (Phi V) + diag(alpha) V  (Sec. III, Eq. mat-eq; Alg. 2
    "Apply matrix")."""
    V = np.asarray(V, dtype=np.float64)
    a = np.asarray(alpha, dtype=np.float64)
    return beta * op.apply_t(op.apply(V)) + (a[:, None] * V if V.ndim == 2 else a * V)
