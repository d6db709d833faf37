"""Pins for the whole CoFEM oracle (Alg. 1 + Alg. 2)."""
import numpy as np
import pytest

from oracle import cofem as cofem_mod
from oracle.cofem import cofem, second_moment, FLAG_ALPHA_CLAMPED
from oracle.em import em, estep_explicit
from oracle.operators import DenseOperator, ToeplitzOperator
from oracle.philox import rademacher_probes
from synth import dense_gaussian, toeplitz_calcium


def _hadamard(n):
    H = np.array([[1.0]])
    while H.shape[0] < n:
        H = np.block([[H, H], [H, -H]])
    return H


@pytest.mark.parametrize("solver,tol", [("direct", None), ("pcg", 1e-13)])
def test_hadamard_probes_reproduce_em(solver, tol):
    """With the D Hadamard columns as probes, s = diag(Sigma) exactly, so
    CoFEM with an exact (or tight) solve is EM (Prop. 1 expansion, K = D)."""
    p = dense_gaussian(24, 64, 5, 25.0, seed=3)
    H = _hadamard(64)
    T = 10
    r = cofem(DenseOperator(p.phi), p.y, p.beta, 64, T, tol or 1e-10, 2000, seed=0,
              probe_fn=lambda t, K, D: H, solver=solver)
    e = em(p.phi, p.y, p.beta, T)
    np.testing.assert_allclose(r["mu"], e["mu"], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(r["s"], e["diag_sigma"], rtol=1e-7)
    np.testing.assert_allclose(r["alpha"], e["alpha"], rtol=1e-7)


def test_rademacher_error_matches_lemma1():
    """One E-step: the error s_j - Sigma_jj, normalised by Lemma 1's
    nu_j = sqrt((1/K) sum_{j' != j} Sigma_jj'^2), has mean square about 1;
    and it shrinks as 1/sqrt(K)."""
    p = dense_gaussian(64, 256, 10, 20.0, seed=8)
    op = DenseOperator(p.phi)
    alpha = np.exp(np.random.default_rng(1).uniform(-1, 3, 256))
    _, Sigma = estep_explicit(p.phi, p.y, p.beta, alpha)
    off2 = (Sigma ** 2).sum(axis=1) - np.diag(Sigma) ** 2
    rms = []
    for K in (20, 200, 2000):
        r = cofem(op, p.y, p.beta, K, 1, 1e-12, 2000, seed=2, alpha0=alpha)
        z2 = (r["s"] - np.diag(Sigma)) ** 2 / (off2 / K)
        assert 0.75 < z2.mean() < 1.3, (K, z2.mean())
        rms.append(np.sqrt(np.mean((r["s"] - np.diag(Sigma)) ** 2)))
    assert 2.3 < rms[0] / rms[1] < 4.5 and 2.3 < rms[1] / rms[2] < 4.5


def test_identity_dictionary_closed_form():
    """Phi = I, Jacobi theta = 1: M = A exactly, PCG takes one step, and
    mu_j = beta y_j/(beta+alpha_j), s_j = 1/(beta+alpha_j) for any probes."""
    D = 128
    rng = np.random.default_rng(2)
    y = rng.standard_normal(D)
    beta = 9.0
    T = 12
    r = cofem(DenseOperator(np.eye(D)), y, beta, 8, T, 1e-10, 50, seed=5)
    assert np.all(r["cg_iters"] == 1)
    a = np.ones(D)
    for _ in range(T - 1):
        m = beta * y / (beta + a)
        a = 1.0 / (m * m + 1.0 / (beta + a))
    np.testing.assert_allclose(r["alpha"], a, rtol=1e-12)
    np.testing.assert_allclose(r["mu"], beta * y / (beta + a), rtol=1e-12)
    np.testing.assert_allclose(r["s"], 1.0 / (beta + a), rtol=1e-12)


def test_zero_dictionary_gives_inverse_alpha():
    """Phi = 0: b = 0 (mu column starts converged), A = M = diag(alpha),
    s_j = (1/K) sum_k p_kj^2 / alpha_j = 1/alpha_j exactly."""
    D = 100
    alpha0 = np.linspace(0.5, 9.0, D)
    r = cofem(DenseOperator(np.zeros((10, D))), np.ones(10), 4.0, 6, 1, 1e-12, 20, seed=1,
              alpha0=alpha0)
    assert np.all(r["mu"] == 0.0)
    np.testing.assert_allclose(r["s"], 1.0 / alpha0, rtol=1e-14)


def test_column_zero_is_mu_and_probes_are_philox():
    p = dense_gaussian(16, 40, 3, 20.0, seed=1)
    r = cofem(DenseOperator(p.phi), p.y, p.beta, 4, 1, 1e-13, 500, seed=9, return_x=True)
    Phi = p.phi.astype(np.float64)
    A = p.beta * Phi.T @ Phi + np.eye(40)
    P = rademacher_probes(9, 1, 4, 40).T
    np.testing.assert_allclose(r["X"][:, 0], np.linalg.solve(A, p.beta * Phi.T @ p.y.astype(np.float64)), rtol=1e-8)
    np.testing.assert_allclose(r["X"][:, 1:], np.linalg.solve(A, P), rtol=1e-7, atol=1e-12)


def _sec5_fixture():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sec5_accuracy_settings.json")))


def _sec5_problem(g, seed=11):
    """The printed accuracy setting: dense Gaussian Phi, N = D/4, d = 0.06 D
    spikes Uniform(-2, 2), noise sigma = 0.01 (beta = 1/sigma^2 = 1e4)."""
    D = g["D"]
    p = dense_gaussian(D // 4, D, int(0.06 * D), 0.0, seed=seed, spike="uniform2", sigma=g["sigma"])
    assert p.beta == g["beta"]
    return p


def _nrmse(mu, z):
    return np.linalg.norm(mu - z) / np.linalg.norm(z)


def test_support_recovery_gaussian():
    """Sec. V settings and outcome (tests/golden/sec5_accuracy_settings.json:
    sigma = 0.01, beta = 1e4, K = 20, U = 400, theta = 1, T = 30).  CoFEM with
    eps = 1e-5 (per column or Frobenius) gives the fit of an exact E-step
    solve with the same probes (mu within 2e-3, NRMSE within 2 %), recovers
    every spike clearly above the noise and nothing else.  (At this noise
    level the exact-solve fit itself has NRMSE 1.6-3.2 % over seeds 1-8,
    2.26 % here, so the printed "< 2 %" is checked at 40 dB below.)"""
    g = _sec5_fixture()
    p = _sec5_problem(g)
    op = DenseOperator(p.phi)
    ex = cofem(op, p.y, p.beta, g["K"], g["T"], 1e-5, g["U"], seed=3, precond="one", solver="direct")
    off = np.ones(p.D, bool)
    off[p.support] = False
    big = np.abs(p.z) > 0.1
    for conv in ("per_column", "frobenius"):
        r = cofem(op, p.y, p.beta, g["K"], g["T"], 1e-5, g["U"], seed=3, precond="one", conv=conv)
        assert np.linalg.norm(r["mu"] - ex["mu"]) / np.linalg.norm(ex["mu"]) < 2e-3, conv
        assert _nrmse(r["mu"], p.z) < 1.02 * _nrmse(ex["mu"], p.z), conv
        assert np.all(np.abs(r["mu"][big]) > 0.05)
        assert np.max(np.abs(r["mu"][off])) < 0.05


def test_printed_cg_tolerance_leaves_mu_inexact():
    """Reading of Sec. V-C's eps: with the per-column stopping test, the
    printed eps = 1e-4 stops the mu column early enough that the fit departs
    from the exact-solve fit (mu more than 1e-2 away, NRMSE over 1.5 times the
    exact one), while eps = 1e-5 stays within 2e-3 of it; the workloads
    therefore use 1e-5."""
    g = _sec5_fixture()
    p = _sec5_problem(g)
    op = DenseOperator(p.phi)
    ex = cofem(op, p.y, p.beta, g["K"], g["T"], 1e-5, g["U"], seed=3, precond="one", solver="direct")
    d = {}
    for eps in (1e-4, 1e-5):
        r = cofem(op, p.y, p.beta, g["K"], g["T"], eps, g["U"], seed=3, precond="one")
        d[eps] = (np.linalg.norm(r["mu"] - ex["mu"]) / np.linalg.norm(ex["mu"]),
                  _nrmse(r["mu"], p.z) / _nrmse(ex["mu"], p.z))
    assert d[1e-4][0] > 1e-2 and d[1e-4][1] > 1.5, d
    assert d[1e-5][0] < 2e-3 and d[1e-5][1] < 1.02, d


def test_support_recovery_gaussian_40db():
    """The printed outcome, NRMSE < 2 % after T = 30 (same settings as above,
    noise at 40 dB SNR instead of sigma = 0.01), at eps = 1e-5."""
    g = _sec5_fixture()
    D = g["D"]
    p = dense_gaussian(D // 4, D, int(0.06 * D), 40.0, seed=11, spike="uniform2")
    for conv in ("per_column", "frobenius"):
        r = cofem(DenseOperator(p.phi), p.y, p.beta, g["K"], g["T"], 1e-5, g["U"], seed=3, precond="one",
                  conv=conv)
        assert _nrmse(r["mu"], p.z) < g["nrmse_below"], conv


@pytest.mark.parametrize("N,D,d,snr,seed,K,T,far", [
    (77, 301, 9, 20.0, 1, 1, 6, True), (120, 500, 15, 25.0, 11, 6, 8, True), (200, 800, 16, 25.0, 12, 8, 8, True),
    (250, 500, 10, 15.0, 11, 16, 10, False), (200, 501, 10, 15.0, 5, 5, 8, False)])
def test_fit_sensitivity_to_cg_tolerance(N, D, d, snr, seed, K, T, far):
    """Why whole-fit parity at tol 1e-5 is checked on the better-conditioned
    problems: on the ill-conditioned ones (far=True) the FP64 fit at
    tol 1e-5 is itself more than the parity tolerance (1e-4 on mu, 1e-3 on
    1/alpha) away from the same fit at tol 1e-7, so the result at 1e-5 is
    not determined to that tolerance by the method; on the others it is."""
    p = dense_gaussian(N, D, d, snr, seed=seed)
    op = DenseOperator(p.phi)
    a = cofem(op, p.y, p.beta, K, T, 1e-5, 400, seed=2)
    b = cofem(op, p.y, p.beta, K, T, 1e-7, 2000, seed=2)
    e_mu = np.linalg.norm(a["mu"] - b["mu"]) / np.linalg.norm(b["mu"])
    e_a = np.linalg.norm(1 / a["alpha"] - 1 / b["alpha"]) / np.linalg.norm(1 / b["alpha"])
    if far:
        assert e_mu > 1e-3 and e_a > 1e-3, (e_mu, e_a)
    else:
        assert e_mu < 1e-4 and e_a < 1e-3, (e_mu, e_a)


def test_toeplitz_cofem_matches_dense_route():
    """The convolution operator (FFT) and its explicit matrix give the same fit."""
    p = toeplitz_calcium(300, 32, 0.05, 20.0, seed=4)
    opT = ToeplitzOperator(p.phi, 300)
    opD = DenseOperator(opT.dense())
    r1 = cofem(opT, p.y, p.beta, 6, 5, 1e-10, 500, seed=2)
    r2 = cofem(opD, p.y, p.beta, 6, 5, 1e-10, 500, seed=2)
    for k in ("mu", "s"):
        np.testing.assert_allclose(r1[k], r2[k], rtol=1e-5, atol=1e-9)
    # alpha_j near the clamp is 1/(mu_j^2 + s_j) of a tiny difference: compare
    # the second moment 1/alpha, the quantity the M-step actually forms
    np.testing.assert_allclose(1.0 / r1["alpha"], 1.0 / r2["alpha"], rtol=1e-5, atol=1e-12)


def test_alpha_clamp_flag():
    """An M-step with mu^2 + s <= 1/alpha_max clamps alpha at alpha_max and flags it."""
    D = 8
    r = cofem(DenseOperator(np.zeros((4, D))), np.zeros(4), 1.0, 1, 2, 1e-12, 10, seed=1,
              alpha0=np.full(D, 1e13), alpha_max=1e12)
    assert r["flags"] & FLAG_ALPHA_CLAMPED
    assert np.all(r["alpha"] == 1e12)


def test_last_iteration_skips_mstep():
    """Alg. 1 returns alpha^(T): with T = 1 alpha stays at alpha0."""
    p = dense_gaussian(16, 40, 3, 20.0, seed=1)
    a0 = np.linspace(1, 2, 40)
    r = cofem(DenseOperator(p.phi), p.y, p.beta, 4, 1, 1e-8, 100, seed=1, alpha0=a0)
    np.testing.assert_array_equal(r["alpha"], a0)


@pytest.mark.parametrize("mu", [-4.0, -1.0, -0.2, 0.0, 0.5, 2.0, 6.0])
@pytest.mark.parametrize("s", [0.01, 0.3, 1.0, 4.0])
def test_rectified_second_moment_is_the_truncated_normal_moment(mu, s):
    """Non-negativity subsection: the M-step's E[z_j^2] is the second moment
    of N(mu, Sigma) restricted to z >= 0 (reading 12), checked against
    quadrature of that density (no error function involved)."""
    from scipy import integrate
    sd = np.sqrt(s)
    if mu >= 0.0:   # unnormalised density, peak 1 at z = mu
        pdf = lambda z: np.exp(-0.5 * ((z - mu) / sd) ** 2)   # noqa: E731
        hi = mu + 40.0 * sd
    else:           # the same times exp(mu^2 / 2s): peak 1 at z = 0
        pdf = lambda z: np.exp(-z * z / (2.0 * s) + z * mu / s)   # noqa: E731
        hi = 40.0 * min(sd, s / -mu)
    lo = 0.0
    mass = integrate.quad(pdf, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0]
    m2 = integrate.quad(lambda z: z * z * pdf(z), lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)[0] / mass
    got = second_moment(mu, s, "rectified")
    np.testing.assert_allclose(got, m2, rtol=1e-8)


def test_rectified_second_moment_special_cases():
    """mu = 0: the half-normal moment, Sigma; s <= 0: no truncation term
    (reading 12); the sign of mu orders it against the Gaussian prior's
    mu^2 + s (the inverse Mills ratio is positive)."""
    s = np.array([0.5, 2.0, 1e-3])
    np.testing.assert_array_equal(second_moment(np.zeros(3), s, "rectified"), s)
    mu = np.array([1.5, -2.0, 0.3])
    neg = np.array([-0.1, 0.0, -1e-9])
    np.testing.assert_array_equal(second_moment(mu, neg, "rectified"), mu ** 2 + neg)
    g = second_moment(mu, np.full(3, 0.7), "gaussian")
    r = second_moment(mu, np.full(3, 0.7), "rectified")
    assert np.all((r > g) == (mu > 0)) and np.all(r > 0)


def test_rectified_prior_enters_the_m_step():
    """With T = 2 the returned alpha is the M-step of E-step 1, whose mu and s
    do not depend on the prior: under the rectified prior the components with
    a negative posterior mean (and s > 0) get a larger alpha than under the
    Gaussian prior, those with a positive mean a smaller one, and alpha is the
    reciprocal of the truncated moment of E-step 1's (mu, s)."""
    p = toeplitz_calcium(1024, 32, 0.02, 20.0, seed=4)
    op = ToeplitzOperator(p.phi, p.N)
    e1 = cofem(op, p.y, p.beta, 16, 1, 1e-9, 2000, seed=2)
    g = cofem(op, p.y, p.beta, 16, 2, 1e-9, 2000, seed=2)
    r = cofem(op, p.y, p.beta, 16, 2, 1e-9, 2000, seed=2, prior="rectified")
    mu, sv = e1["mu"], e1["s"]
    m2 = second_moment(mu, sv, "rectified")
    np.testing.assert_allclose(r["alpha"], 1.0 / np.maximum(m2, 1e-12), rtol=1e-12)
    sel = (sv > 0) & (np.abs(mu) > 1e-6)
    assert np.all((r["alpha"][sel] > g["alpha"][sel]) == (mu[sel] < 0))


def test_hadamard_probes_reproduce_em_with_rectified_prior():
    """The Hadamard-probe equivalence (s = diag Sigma exactly) holds under the
    rectified prior too: CoFEM with an exact solve is EM with the truncated
    second moment in its M-step."""
    p = toeplitz_calcium(64, 16, 0.1, 25.0, seed=5)
    H = _hadamard(64)
    T = 8
    op = ToeplitzOperator(p.phi, p.N)
    r = cofem(op, p.y, p.beta, 64, T, 1e-10, 2000, seed=0, probe_fn=lambda t, K, D: H,
              solver="direct", prior="rectified")
    e = em(op.dense(), p.y, p.beta, T, alpha_max=1e12, prior="rectified")
    np.testing.assert_allclose(r["mu"], e["mu"], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(r["s"], e["diag_sigma"], rtol=1e-7)
    np.testing.assert_allclose(r["alpha"], e["alpha"], rtol=1e-7)
    g = em(op.dense(), p.y, p.beta, T, alpha_max=1e12)
    assert not np.allclose(g["alpha"], e["alpha"])


def test_multitask_probes_are_per_task_and_task0_is_the_single_task_rule():
    a = rademacher_probes(2, 3, 4, 700)
    np.testing.assert_array_equal(rademacher_probes(2, 3, 4, 700, task=0), a)
    b = rademacher_probes(2, 3, 4, 700, task=1)
    assert not np.array_equal(a, b) and abs(np.mean(a * b)) < 0.05   # independent signs


def test_multitask_with_one_task_is_single_task_cofem():
    from oracle import cofem_multitask
    p = dense_gaussian(60, 200, 6, 20.0, seed=9)
    op = DenseOperator(p.phi)
    m = cofem_multitask([op], [p.y], p.beta, 8, 4, 1e-8, 500, seed=2)
    r = cofem(op, p.y, p.beta, 8, 4, 1e-8, 500, seed=2)
    np.testing.assert_array_equal(m["alpha"], r["alpha"])
    np.testing.assert_array_equal(m["mu"][0], r["mu"])
    np.testing.assert_array_equal(m["cg_iters"], r["cg_iters"])


def test_multitask_hadamard_probes_reproduce_multitask_em():
    """Multi-task subsection: with the D Hadamard columns as every task's
    probes and exact solves, multi-task CoFEM is multi-task EM (explicit
    covariances, shared alpha = L / sum_l (mu_l^2 + Sigma_l,jj))."""
    from oracle import cofem_multitask, em_multitask
    D, L, T = 64, 3, 6
    H = _hadamard(D)
    probs = [dense_gaussian(24, D, 5, 25.0, seed=20 + l) for l in range(L)]
    beta = probs[0].beta
    ops = [DenseOperator(p.phi) for p in probs]
    r = cofem_multitask(ops, [p.y for p in probs], beta, D, T, 1e-10, 2000, seed=0,
                        probe_fn=lambda t, K, D_, l: H, solver="direct")
    e = em_multitask([p.phi for p in probs], [p.y for p in probs], beta, T, alpha_max=1e12)
    np.testing.assert_allclose(r["mu"], e["mu"], rtol=1e-7, atol=1e-10)
    np.testing.assert_allclose(r["s"], e["diag_sigma"], rtol=1e-7)
    np.testing.assert_allclose(r["alpha"], e["alpha"], rtol=1e-7)


def test_multitask_em_with_identical_tasks_is_single_task_em():
    """L copies of one task: alpha = L / (L (mu^2 + Sigma)) is the single-task
    update, so multi-task EM follows single-task EM (up to the rounding of
    (3 x) / 3, amplified by the E-steps' conditioning)."""
    from oracle import em_multitask
    p = dense_gaussian(30, 80, 5, 20.0, seed=4)
    m = em_multitask([p.phi] * 3, [p.y] * 3, p.beta, 5)
    e = em(p.phi, p.y, p.beta, 5)
    np.testing.assert_allclose(m["alpha"], e["alpha"], rtol=1e-9)
    for l in range(3):
        np.testing.assert_allclose(m["mu"][l], e["mu"], rtol=1e-9, atol=1e-14)


def test_unpreconditioned_cg_solves_the_same_systems():
    """precond="none" (M = I, the comparison of the paper's preconditioner
    study) reaches the same E-step solution as the Jacobi preconditioner, in
    more CG steps."""
    p = dense_gaussian(80, 300, 8, 25.0, seed=12)
    op = DenseOperator(p.phi)
    # one E-step (alpha = 1, kappa(A) ~ 4e4): both stop at ||r|| <= 1e-12 ||b||
    a = cofem(op, p.y, p.beta, 6, 1, 1e-12, 3000, seed=2)
    n = cofem(op, p.y, p.beta, 6, 1, 1e-12, 3000, seed=2, precond="none")
    assert a["flags"] == 0 and n["flags"] == 0
    # |x error| <= kappa(A) tol |x| ~ 4e-8 |x|
    np.testing.assert_allclose(n["mu"], a["mu"], rtol=0, atol=1e-7 * np.max(np.abs(a["mu"])))
    np.testing.assert_allclose(n["s"], a["s"], rtol=0, atol=1e-7 * np.max(np.abs(a["s"])))
    # later E-steps (alpha spread over orders of magnitude): Jacobi needs fewer steps
    a3 = cofem(op, p.y, p.beta, 6, 3, 1e-8, 3000, seed=2)
    n3 = cofem(op, p.y, p.beta, 6, 3, 1e-8, 3000, seed=2, precond="none")
    assert n3["cg_iters"][-1] > a3["cg_iters"][-1]


def test_breakdown_fit_goes_on():
    """Phi = 0 and alpha0 = 0: the Jacobi preconditioner M = beta theta + alpha
    is zero, so the probe columns of the first E-step break down (pi not
    finite) and are frozen at x = 0; mu = 0 (b = 0), s = 0, the M-step clamps
    alpha at alpha_max, and the next E-step is regular (M = alpha_max):
    s = 1/alpha_max exactly (Phi = 0 closed form)."""
    from oracle.cofem import FLAG_BREAKDOWN
    D = 40
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        r1 = cofem(DenseOperator(np.zeros((10, D))), np.ones(10), 3.0, 4, 1, 1e-10, 50, seed=1,
                   alpha0=np.zeros(D))
        r3 = cofem(DenseOperator(np.zeros((10, D))), np.ones(10), 3.0, 4, 3, 1e-10, 50, seed=1,
                   alpha0=np.zeros(D))
    assert r1["flags"] & FLAG_BREAKDOWN
    assert np.all(r1["mu"] == 0.0) and np.all(r1["s"] == 0.0)
    assert r3["flags"] & FLAG_BREAKDOWN and r3["flags"] & FLAG_ALPHA_CLAMPED
    for k in ("mu", "s", "alpha"):
        assert np.all(np.isfinite(r3[k])), k
    np.testing.assert_array_equal(r3["alpha"], 1e12)
    np.testing.assert_allclose(r3["s"], 1e-12, rtol=1e-14)


def test_warm_start_with_probe_reuse_is_cofem_with_fixed_probes():
    """Probe reuse draws the t = 1 probes at every E-step; with tight CG
    tolerances the warm-started fit is the cold-started fit whose probe_fn
    returns those probes at every t (the same systems, solved from another
    start), and with exact solves the warm start changes nothing."""
    p = dense_gaussian(60, 200, 6, 20.0, seed=12)
    op = DenseOperator(p.phi)
    fixed = lambda t, K, D: rademacher_probes(4, 1, K, D)   # noqa: E731
    w = cofem(op, p.y, p.beta, 8, 6, 1e-12, 2000, seed=4, warm_start=True)
    c = cofem(op, p.y, p.beta, 8, 6, 1e-12, 2000, seed=4, probe_fn=fixed)
    for k in ("mu", "s"):
        np.testing.assert_allclose(w[k], c[k], rtol=1e-6, atol=1e-9)
    np.testing.assert_allclose(1 / w["alpha"], 1 / c["alpha"], rtol=1e-7)
