"""Seeded synthetic workloads for covariance-free EM (CoFEM) sparse Bayesian learning.

This module only *generates inputs*: a dictionary Phi (dense Gaussian or the
causal double-exponential convolution filter), a sparse ground truth z*, noisy
measurements y = Phi z* + eps and the noise precision beta.  It holds none of the
method's arithmetic (no E-step, no CG, no probes, no M-step), so both the FP64
CPU oracle and the CUDA path may be fed from it.

Recipes follow the paper's simulation setup (Sec. V-A "General Structure" and
"Dictionary"): spikes at uniformly random positions, y = Phi z* + eps with
eps ~ N(0, sigma^2 I), and, for the dense dictionary, Phi_ij ~ N(0, 1/N).
The noise level is set from a target SNR in dB:
    sigma^2 = ||Phi z*||^2 / (N * 10^(SNR/10)),   beta = 1/sigma^2
(beta taken from sigma, not from the realised eps).

Everything is produced with numpy's PCG64 from an explicit integer seed, so a
workload is a pure function of its parameters.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "Problem",
    "MultiTaskProblem",
    "dense_gaussian",
    "dense_gaussian_multitask",
    "DCTProblem",
    "dct_sparse",
    "double_exponential_filter",
    "toeplitz_calcium",
    "WORKLOADS",
    "workload",
    "serving_requests",
]


@dataclasses.dataclass
class Problem:
    """One sparse-coding problem y = Phi z* + eps.

    kind      "dense" (phi is an N x D float32 row-major matrix) or
              "toeplitz" (phi is the length-L float32 causal filter h; N = D).
    beta      noise precision 1/sigma^2 (float).
    z         ground-truth sparse code (float64, length D).
    """

    kind: str
    N: int
    D: int
    phi: np.ndarray
    y: np.ndarray
    z: np.ndarray
    beta: float
    sigma2: float
    support: np.ndarray

    @property
    def L(self) -> int:
        return int(self.phi.shape[0]) if self.kind == "toeplitz" else 0


def _noise(rng: np.random.Generator, clean: np.ndarray, snr_db: float, sigma: Optional[float] = None):
    N = clean.shape[0]
    if sigma is not None:   # a fixed noise level instead of a target SNR
        sigma2 = float(sigma) ** 2
    else:
        sigma2 = float(np.dot(clean, clean)) / (N * 10.0 ** (snr_db / 10.0))
    if sigma2 <= 0.0:  # all-zero signal: fall back to unit precision
        sigma2 = 1.0
    eps = rng.standard_normal(N) * math.sqrt(sigma2)
    return clean + eps, sigma2


def dense_gaussian(N: int, D: int, d: int, snr_db: float, seed: int,
                   spike: str = "normal", sigma: Optional[float] = None) -> Problem:
    """Dense Gaussian dictionary Phi_ij ~ N(0, 1/N) (float32), d spikes at
    uniformly random positions with N(0,1) (or Uniform(-2,2)) amplitudes.
    The noise is set by snr_db, or by a fixed standard deviation `sigma` when
    given (snr_db is then ignored)."""
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((N, D), dtype=np.float32)
    phi *= np.float32(1.0 / math.sqrt(N))
    support = np.sort(rng.choice(D, size=d, replace=False)) if d > 0 else np.zeros(0, np.int64)
    z = np.zeros(D, dtype=np.float64)
    if spike == "normal":
        z[support] = rng.standard_normal(d)
    elif spike == "uniform2":
        z[support] = rng.uniform(-2.0, 2.0, size=d)
    else:
        raise ValueError(spike)
    clean = phi[:, support].astype(np.float64) @ z[support] if d > 0 else np.zeros(N)
    y, sigma2 = _noise(rng, clean, snr_db, sigma)
    return Problem("dense", N, D, phi, y.astype(np.float32), z, 1.0 / sigma2, sigma2, support)


@dataclasses.dataclass
class MultiTaskProblem:
    """L problems y_l = Phi z*_l + eps_l sharing one dense dictionary (multiple
    measurement vectors) and one noise precision beta; Y is L x N, Z is L x D."""

    N: int
    D: int
    L: int
    phi: np.ndarray
    Y: np.ndarray
    Z: np.ndarray
    beta: float
    support: np.ndarray


def dense_gaussian_multitask(N: int, D: int, d: int, snr_db: float, L: int, seed: int) -> MultiTaskProblem:
    """Shared dense Gaussian dictionary Phi_ij ~ N(0, 1/N) (float32); the L
    codes z*_l share d uniformly random support positions (the joint sparsity
    a shared alpha models) with independent N(0,1) amplitudes; one noise level
    sigma^2 = mean_l ||Phi z*_l||^2 / (N 10^(SNR/10)), beta = 1/sigma^2."""
    rng = np.random.default_rng(seed)
    phi = rng.standard_normal((N, D), dtype=np.float32)
    phi *= np.float32(1.0 / math.sqrt(N))
    support = np.sort(rng.choice(D, size=d, replace=False))
    Z = np.zeros((L, D), dtype=np.float64)
    Z[:, support] = rng.standard_normal((L, d))
    clean = Z[:, support] @ phi[:, support].astype(np.float64).T          # L x N
    sigma2 = float(np.mean(np.sum(clean * clean, axis=1))) / (N * 10.0 ** (snr_db / 10.0))
    Y = clean + rng.standard_normal((L, N)) * math.sqrt(sigma2)
    return MultiTaskProblem(N, D, L, phi, Y.astype(np.float32), Z, 1.0 / sigma2, support)


@dataclasses.dataclass
class DCTProblem:
    """y = Phi z* + eps with the DCT dictionary Phi = M Omega^-1 (the rows
    `rows` of the inverse orthonormal DCT-II of size D)."""

    N: int
    D: int
    rows: np.ndarray      # int32, sorted, distinct, < D
    y: np.ndarray         # float32, N
    z: np.ndarray         # float64, D
    beta: float
    support: np.ndarray


def dct_sparse(D: int, N: int, d: int, sigma: float, seed: int, spike_sd: float = 5.0) -> DCTProblem:
    """The DCT dictionary of Sec. V-A: N of the D rows of Omega^-1 kept at
    random, d spikes N(0, spike_sd^2) at uniform positions, noise sigma
    (beta = 1/sigma^2).  y is formed with scipy's orthonormal inverse DCT."""
    from scipy import fft
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(D, size=N, replace=False)).astype(np.int32)
    support = np.sort(rng.choice(D, size=d, replace=False))
    z = np.zeros(D, dtype=np.float64)
    z[support] = rng.standard_normal(d) * spike_sd
    clean = fft.idct(z, type=2, norm="ortho")[rows]
    y = clean + rng.standard_normal(N) * sigma
    return DCTProblem(N, D, rows, y.astype(np.float32), z, 1.0 / sigma ** 2, support)


def double_exponential_filter(L: int = 256, tau_decay: float = 40.0,
                              tau_rise: float = 4.0) -> np.ndarray:
    """Calcium-style response h[t] = exp(-t/40) - exp(-t/4), t = 0..L-1 (float32).
    h[0] = 0 and the peak (about 0.697) is at t = 10."""
    t = np.arange(L, dtype=np.float64)
    return (np.exp(-t / tau_decay) - np.exp(-t / tau_rise)).astype(np.float32)


def toeplitz_calcium(D: int, L: int, rate: float, snr_db: float, seed: int) -> Problem:
    """Convolutional dictionary (N = D): column j of Phi holds h delayed by j
    samples and truncated at N (paper Sec. V-A, "Convolutional").  z* is
    Bernoulli(rate) spikes with Exp(1) amplitudes."""
    rng = np.random.default_rng(seed)
    h = double_exponential_filter(L)
    mask = rng.random(D) < rate
    support = np.nonzero(mask)[0]
    z = np.zeros(D, dtype=np.float64)
    z[support] = rng.exponential(1.0, size=support.size)
    # y_i = sum_tau h[tau] z[i - tau]  (causal, truncated to N = D samples)
    clean = np.convolve(z, h.astype(np.float64))[:D]
    y, sigma2 = _noise(rng, clean, snr_db)
    return Problem("toeplitz", D, D, h, y.astype(np.float32), z, 1.0 / sigma2, sigma2, support)


# Named workloads (the shapes of the paper's simulations, scaled per the
# deployment configurations).  Each entry gives the problem recipe and the
# CoFEM run parameters.  Seeds: data seed 1, probe seed 2.
WORKLOADS = {
    "dense_n256_d1024_k20": dict(
        kind="dense", N=256, D=1024, d=51, snr_db=20.0, K=20, T=50,
        cg_tol=1e-5, cg_maxit=400, precision="f32", rr_period=0),
    # FP32 dictionary with the skinny products on the tensor cores (3xTF32)
    "dense_n2500_d10000_k32": dict(
        kind="dense", N=2500, D=10000, d=200, snr_db=25.0, K=32, T=50,
        cg_tol=1e-5, cg_maxit=400, precision="tf32x3", rr_period=0),
    "toeplitz_d1e6_l256_k16": dict(
        kind="toeplitz", N=1_000_000, D=1_000_000, L=256, rate=0.01, snr_db=15.0,
        K=16, T=30, cg_tol=1e-5, cg_maxit=400, precision="f32", rr_period=0),
    # The precision form: residual replacement every 20 CG iterations (with X
    # held as an FP32 pair and B - A X formed accurately) and the end-of-E-step
    # true-residual check.
    "dense_n8192_d32768_k32_bf16": dict(
        kind="dense", N=8192, D=32768, d=327, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="bf16", rr_period=20),
    # the precision form at a quarter of the size (Phi~ 128 MiB, its slice
    # images 384 MiB each: larger than L2, a few GB on the device in all), for
    # profiler captures of the same kernels
    "dense_n4096_d16384_k32_bf16": dict(
        kind="dense", N=4096, D=16384, d=164, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="bf16", rr_period=20),
    # profiling sizes of the FP8 and 3xTF32 operators (each product's image
    # larger than L2: 128 MiB of codes, 256 MiB of FP32)
    "dense_n8192_d16384_k32_fp8": dict(
        kind="dense", N=8192, D=16384, d=164, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="fp8", rr_period=0),
    "dense_n4096_d16384_k32_tf32x3": dict(
        kind="dense", N=4096, D=16384, d=164, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="tf32x3", rr_period=0),
    "dense_n8192_d32768_k32_f32": dict(
        kind="dense", N=8192, D=32768, d=327, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="f32", rr_period=0),
    "dense_n8192_d32768_k32_fp8": dict(
        kind="dense", N=8192, D=32768, d=327, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="fp8", rr_period=0),
    "dense_n8192_d32768_k32_tf32x3": dict(
        kind="dense", N=8192, D=32768, d=327, snr_db=30.0, K=32, T=30,
        cg_tol=1e-5, cg_maxit=400, precision="tf32x3", rr_period=0),
}

DATA_SEED = 1
PROBE_SEED = 2


def workload(name: str, seed: Optional[int] = None, **overrides) -> tuple[Problem, dict]:
    """Build the named workload's problem; returns (problem, run parameters)."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    seed = DATA_SEED if seed is None else seed
    if spec["kind"] == "dense":
        prob = dense_gaussian(spec["N"], spec["D"], spec["d"], spec["snr_db"], seed)
    else:
        prob = toeplitz_calcium(spec["D"], spec["L"], spec["rate"], spec["snr_db"], seed)
    run = {k: spec[k] for k in ("K", "T", "cg_tol", "cg_maxit", "precision", "rr_period")}
    run["seed"] = PROBE_SEED
    return prob, run


def serving_requests(n: int, base_seed: int = 1000, rate_hz: float = 100.0,
                     d_min: int = 1024, d_max: int = 16384, frac: float = 0.03,
                     snr_lo: float = 15.0, snr_hi: float = 30.0, Ks=(8, 16, 32),
                     T: int = 30, arrival_seed: int = 7):
    """Request stream for the serving loop: Poisson arrivals at `rate_hz`;
    request i has D ~ U[d_min, d_max], N = D/4, 3 % spikes, SNR ~ U[15,30] dB,
    K drawn from Ks, T EM iterations and data seed base_seed + i.  Returns a
    list of dicts (no arrays: the problem is generated from its seed)."""
    rng = np.random.default_rng(arrival_seed)
    gaps = rng.exponential(1.0 / rate_hz, size=n)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(n):
        D = int(rng.integers(d_min, d_max + 1))
        out.append(dict(index=i, arrival_s=float(t[i]), D=D, N=max(1, D // 4),
                        d=max(1, int(frac * D)), snr_db=float(rng.uniform(snr_lo, snr_hi)),
                        K=int(rng.choice(Ks)), T=T, seed=base_seed + i))
    return out
