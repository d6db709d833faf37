"""GPU parity: libcofem (through its C ABI) against the FP64 CPU oracle on the
same seeded inputs and the same Philox probes.

Tolerances: probes are bit-exact (integer work); operator applications are
compared per column in relative l2 (FP32 accumulation over up to N*D terms,
bound 2e-5); whole fits use relative l2 <= 1e-4 on mu and <= 1e-3 on s, on
the second moment 1/alpha = max(mu^2 + s, 1/alpha_max) (the quantity the M-step
forms) and on alpha itself where it is well determined (alpha < 1e6, its
second moment mu^2 + s within 1e-2 of the largest and not a cancelling
difference; elsewhere alpha is the reciprocal of a small difference)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import DenseOperator, ToeplitzOperator, apply_A, cofem as oracle_cofem  # noqa: E402
from oracle.philox import rademacher_probes  # noqa: E402
from synth import dense_gaussian, toeplitz_calcium, double_exponential_filter  # noqa: E402


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


DEV = "cuda:0"


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    n = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (n if n > 0 else 1.0))


def bf16_round(x):
    """Round float32 to the nearest bfloat16 (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def _e4m3_grid():
    """Non-negative E4M3 values in code order (codes 0x00 .. 0x7E): subnormals
    m/8 * 2^-6, normals (1 + m/8) * 2^(e-7); 0x7F is NaN and never produced."""
    v = [m / 8 * 2.0 ** -6 for m in range(8)]
    v += [(1 + m / 8) * 2.0 ** (e - 7) for e in range(1, 16) for m in range(8)]
    return np.array(v[:127])


def e4m3_quantise(phi):
    """Per-row scales s_i = max|Phi_i| / 448 (FP32) and E4M3 codes of
    Phi_ij / s_i (FP32 division, round to nearest, ties to the even code,
    saturating at 448).  Returns (s float32 [N], decoded values float64 [N, D])."""
    p32 = np.ascontiguousarray(phi, np.float32)
    s = (np.abs(p32).max(axis=1) / np.float32(448.0)).astype(np.float32)
    safe = np.where(s > 0, s, np.float32(1.0))
    x = np.where(s[:, None] > 0, p32 / safe[:, None], np.float32(0.0)).astype(np.float32).astype(np.float64)
    g = _e4m3_grid()
    a = np.minimum(np.abs(x), g[-1])
    hi = np.clip(np.searchsorted(g, a, side="left"), 0, len(g) - 1)
    lo = np.maximum(hi - 1, 0)
    dlo, dhi = a - g[lo], g[hi] - a
    pick = np.where(dlo < dhi, lo, np.where(dhi < dlo, hi, np.where(lo % 2 == 0, lo, hi)))
    return s, np.sign(x) * g[pick]


def gpu_fit(cf, prob, K, T, tol, maxit, seed=2, alpha0=None, host=False, want_res=False, **opts):
    D = prob.D
    if host:
        mu, s, al = (np.empty(D, np.float32) for _ in range(3))
        it = np.empty(T, np.int32)
        y = prob.y
        a0 = alpha0
        phi = prob.phi
    else:
        mu, s, al = (torch.empty(D, device=DEV) for _ in range(3))
        it = torch.empty(T, dtype=torch.int32, device=DEV)
        y = torch.from_numpy(prob.y).to(DEV)
        a0 = None if alpha0 is None else torch.from_numpy(alpha0).to(DEV)
        phi = torch.from_numpy(prob.phi).to(DEV)
    kind = cf.COFEM_OP_DENSE if prob.kind == "dense" else cf.COFEM_OP_TOEPLITZ
    with cf.CoFEM(prob.N, D, kind, phi, prob.L, seed=seed, **opts) as m:
        flags = cf.cofem_fit(m.h, y, prob.beta, a0, K, T, tol, maxit, mu, s, al, it)
        res = cf.cofem_true_residuals(m.h, T, K) if want_res else None
    cvt = (lambda v: v) if host else (lambda v: v.cpu().numpy())
    return dict(mu=cvt(mu), s=cvt(s), alpha=cvt(al), cg_iters=cvt(it), flags=flags, true_res=res)


def oracle_fit(prob, K, T, tol, maxit, seed=2, phi=None, **kw):
    if prob.kind == "dense":
        op = DenseOperator(prob.phi if phi is None else phi)
    else:
        op = ToeplitzOperator(prob.phi, prob.N)
    return oracle_cofem(op, prob.y, prob.beta, K, T, tol, maxit, seed, **kw)


def well_determined(r):
    """Coordinates where alpha = 1/max(mu^2 + s, 1/alpha_max) is well
    conditioned: alpha < 1e6, the second moment mu^2 + s at least 1e-2 of its
    largest value (the relative l2 error over a set is that of its largest
    alphas, whose second moments carry the largest relative error) and not a
    cancelling difference (>= 0.1 (mu^2 + |s|))."""
    mu, s_ = np.asarray(r["mu"], np.float64), np.asarray(r["s"], np.float64)
    m2 = 1.0 / np.asarray(r["alpha"], np.float64)
    return (r["alpha"] < 1e6) & (m2 >= 1e-2 * m2.max()) & (m2 >= 0.1 * (mu * mu + np.abs(s_)))


def assert_fit_close(g, r, tol_mu=1e-4, tol_s=1e-3, tol_a=1e-3):
    """mu, s and 1/alpha everywhere, and alpha itself where it is well
    determined (well_determined: the oracle keeps it active, its second moment
    is within 1e-2 of the largest and not a cancelling difference; with few
    probes s can be negative and large)."""
    act = well_determined(r)
    e = (rel(g["mu"], r["mu"]), rel(g["s"], r["s"]), rel(1.0 / g["alpha"], 1.0 / r["alpha"]),
         rel(g["alpha"][act], r["alpha"][act]) if act.any() else 0.0)
    assert e[0] <= tol_mu and e[1] <= tol_s and e[2] <= tol_a and e[3] <= tol_a, (e, g["cg_iters"], r["cg_iters"])
    return e


# ---------------------------------------------------------------------------
# a2: probes (bit-exact)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed,t,K,D", [(2, 1, 20, 1024), (2, 7, 3, 1), (99, 50, 5, 1000), (1, 0, 2, 70001)])
def test_probes_bit_exact(cf, seed, t, K, D):
    out = torch.empty((K, D), device=DEV)
    cf.cofem_probe_fill(seed, t, K, D, out)
    np.testing.assert_array_equal(out.cpu().numpy(), rademacher_probes(seed, t, K, D).astype(np.float32))


# ---------------------------------------------------------------------------
# a0 / a1: theta and b = beta Phi^T y
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,D", [(77, 301), (256, 1024), (1, 5), (300, 129)])
def test_theta_and_phity_dense(cf, N, D):
    p = dense_gaussian(N, D, max(1, D // 20), 20.0, seed=N + D)
    th = np.empty(D, np.float32)
    b = np.empty(D, np.float32)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, p.phi) as m:
        cf.cofem_get_theta(m.h, th)
        cf.cofem_phit_y(m.h, p.y, p.beta, b)
    op = DenseOperator(p.phi)
    np.testing.assert_allclose(th, op.column_sq_norms(), rtol=2e-6)
    assert rel(b, p.beta * op.apply_t(p.y.astype(np.float64))) < 2e-6


def test_theta_and_phity_toeplitz(cf):
    D, L = 5000, 256
    p = toeplitz_calcium(D, L, 0.02, 15.0, seed=3)
    th = np.empty(D, np.float32)
    b = np.empty(D, np.float32)
    with cf.CoFEM(D, D, cf.COFEM_OP_TOEPLITZ, p.phi, L) as m:
        cf.cofem_get_theta(m.h, th)
        cf.cofem_phit_y(m.h, p.y, p.beta, b)
    op = ToeplitzOperator(p.phi, D)
    np.testing.assert_allclose(th, op.column_sq_norms(), rtol=2e-6, atol=1e-12)
    assert th[-1] == 0.0          # h[0] = 0: the last column of Phi is zero
    assert rel(b, p.beta * op.apply_t(p.y.astype(np.float64))) < 2e-6


# ---------------------------------------------------------------------------
# a4: operator A V and pi = v^T A v
# ---------------------------------------------------------------------------
def _check_operator(cf, m, op, D, Q, seed, tol=2e-5):
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((Q, D)).astype(np.float32)
    alpha = np.exp(rng.uniform(-2, 6, D)).astype(np.float32)
    beta = 37.5
    Psi = torch.empty((Q, D), device=DEV)
    pi = cf.cofem_apply_operator(m.h, torch.from_numpy(V).to(DEV), Q, torch.from_numpy(alpha).to(DEV), beta, Psi)
    want = apply_A(op, V.T.astype(np.float64), alpha, beta).T
    got = Psi.cpu().numpy()
    for q in range(Q):
        assert rel(got[q], want[q]) < tol, (q, rel(got[q], want[q]))
    np.testing.assert_allclose(pi, np.sum(V.astype(np.float64) * want, axis=1), rtol=tol)


@pytest.mark.parametrize("precision", ["tf32x3", "simt"])
@pytest.mark.parametrize("N,D,Q", [(77, 301, 1), (77, 301, 7), (256, 1024, 21), (130, 700, 33), (64, 128, 64),
                                   (2500, 10000, 33), (1000, 3000, 17)])
def test_operator_dense_f32(cf, N, D, Q, precision):
    """FP32 dictionary: tensor cores with the error-compensated TF32 split, or
    FP32 FMA on the CUDA cores."""
    p = dense_gaussian(N, D, 3, 20.0, seed=Q)
    prec = cf.COFEM_F32_TF32X3 if precision == "tf32x3" else cf.COFEM_F32
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, torch.from_numpy(p.phi).to(DEV), precision=prec) as m:
        _check_operator(cf, m, DenseOperator(p.phi), D, Q, seed=Q)


PATHS = {"two_pass": 1, "single_pass": 2}


@pytest.mark.parametrize("path", ["two_pass", "single_pass"])
@pytest.mark.parametrize("N,D,Q", [(77, 301, 5), (256, 1024, 33), (1000, 3000, 17), (300, 700, 64),
                                   (2500, 10000, 33), (128, 128, 2), (1, 5, 1), (1153, 4000, 37), (640, 9000, 9)])
def test_operator_dense_bf16(cf, N, D, Q, path):
    """The BF16 form runs exactly on the quantised dictionary bf16(Phi), in
    both operator forms (the single-pass form takes 3Q <= 112)."""
    if path == "single_pass" and 3 * Q > 112:
        pytest.skip("single-pass form needs 3Q <= 112")
    p = dense_gaussian(N, D, 3, 20.0, seed=Q + 1)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_BF16, dense_path=PATHS[path]) as m:
        _check_operator(cf, m, DenseOperator(bf16_round(p.phi)), D, Q, seed=Q)
        assert cf.cofem_operator_info(m.h)[0] == PATHS[path]


@pytest.mark.parametrize("N,D", [(77, 301), (256, 1024), (1000, 3000), (1, 5)])
def test_fp8_dictionary_is_the_e4m3_quantisation(cf, N, D):
    """a0, FP8 form: the stored dictionary is s_i * e4m3(Phi_ij / s_i) bit for bit."""
    p = dense_gaussian(N, D, 3, 20.0, seed=N)
    s, dec = e4m3_quantise(p.phi)
    want = (s[:, None] * dec.astype(np.float32)).astype(np.float32)
    got = np.empty((N, D), np.float32)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_FP8_E4M3) as m:
        cf.cofem_get_dictionary(m.h, got)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("N,D,Q", [(77, 301, 5), (256, 1024, 33), (1000, 3000, 17), (2500, 10000, 33),
                                   (128, 128, 2), (1, 5, 1), (1153, 4000, 42)])
def test_operator_dense_fp8(cf, N, D, Q):
    """FP8 form: the operator on the quantised dictionary s_i e4m3(Phi_ij / s_i)."""
    p = dense_gaussian(N, D, 3, 20.0, seed=Q + 2)
    s, dec = e4m3_quantise(p.phi)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_FP8_E4M3) as m:
        _check_operator(cf, m, DenseOperator(s.astype(np.float64)[:, None] * dec), D, Q, seed=Q)


def test_single_pass_rejected_where_it_does_not_apply(cf):
    p = dense_gaussian(100, 300, 3, 20.0, seed=1)
    with cf.CoFEM(100, 300, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_BF16, dense_path=2) as m:
        V = torch.zeros((50, 300), device=DEV)
        with pytest.raises(cf.CofemError) as e:   # 3 x 50 > 128
            cf.cofem_apply_operator(m.h, V, 50, torch.ones(300, device=DEV), 1.0, torch.empty((50, 300), device=DEV))
        assert e.value.status == cf.COFEM_ERR_UNSUPPORTED
    with cf.CoFEM(100, 300, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_F32_TF32X3, dense_path=2) as m:
        V = torch.zeros((3, 300), device=DEV)
        with pytest.raises(cf.CofemError) as e:   # BF16 only
            cf.cofem_apply_operator(m.h, V, 3, torch.ones(300, device=DEV), 1.0, torch.empty((3, 300), device=DEV))
        assert e.value.status == cf.COFEM_ERR_UNSUPPORTED


@pytest.mark.parametrize("path", ["auto", "single_pass"])
def test_operator_dense_bf16_full_size_sampled(cf, path):
    """8192 x 32768 BF16 dictionary, 33 columns, in the launch configuration of
    the benchmark (the default, two-pass form) and in the single-pass form:
    sampled rows of Psi against FP64 on the quantised dictionary."""
    N, D, Q = 8192, 32768, 33
    p = dense_gaussian(N, D, 4, 30.0, seed=77)
    phq = bf16_round(p.phi)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((Q, D)).astype(np.float32)
    alpha = np.exp(rng.uniform(-2, 6, D)).astype(np.float32)
    beta = 1234.5
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, torch.from_numpy(p.phi).to(DEV), precision=cf.COFEM_BF16,
                  dense_path={"auto": 0, "single_pass": 2}[path]) as m:
        Psi = torch.empty((Q, D), device=DEV)
        pi = cf.cofem_apply_operator(m.h, torch.from_numpy(V).to(DEV), Q, torch.from_numpy(alpha).to(DEV),
                                     beta, Psi)
        assert cf.cofem_operator_info(m.h)[0] == (1 if path == "auto" else 2)
    got = Psi.cpu().numpy()
    T = np.zeros((N, Q))
    for i0 in range(0, N, 1024):                      # T = Phi~ V in FP64, by row blocks
        T[i0:i0 + 1024] = phq[i0:i0 + 1024].astype(np.float64) @ V.T.astype(np.float64)
    cols = np.sort(rng.choice(D, 2000, replace=False))
    want = beta * (phq[:, cols].astype(np.float64).T @ T) + alpha[cols, None].astype(np.float64) * V[:, cols].T
    for q in range(Q):
        assert rel(got[q, cols], want[:, q]) < 2e-5, q
    # pi_q = v^T A v = beta ||Phi~ v||^2 + sum alpha v^2 needs no sampling
    pi_want = beta * np.sum(T * T, axis=0) + np.sum(alpha[None, :].astype(np.float64) * V.astype(np.float64) ** 2,
                                                    axis=1)
    np.testing.assert_allclose(pi, pi_want, rtol=2e-5)


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("D,L,Q", [(5000, 256, 3), (3000, 256, 17), (200, 7, 2), (1793, 256, 1), (4097, 1, 4),
                                   (3000, 1024, 2), (20000, 256, 9), (8192, 64, 4)])
def test_operator_toeplitz(cf, D, L, Q, path):
    """Both forms of the convolution operator: the tiled direct convolution
    and the overlap-save FFTs (several 8192-point blocks at D = 20000)."""
    rng = np.random.default_rng(D + L)
    h = (double_exponential_filter(L) if L >= 16 else rng.standard_normal(L)).astype(np.float32)
    tp = cf.COFEM_TOEPLITZ_FFT if path == "fft" else cf.COFEM_TOEPLITZ_DIRECT
    with cf.CoFEM(D, D, cf.COFEM_OP_TOEPLITZ, h, L, toeplitz_path=tp) as m:
        _check_operator(cf, m, ToeplitzOperator(h, D), D, Q, seed=L)
        assert cf.cofem_operator_info(m.h)[0] == tp


# ---------------------------------------------------------------------------
# whole fits (a0-a8)
# ---------------------------------------------------------------------------
def test_fit_dense_n256_d1024_k20(cf):
    """Plain FP32 form on the 256 x 1024 Gaussian workload, K = 20, T = 50, tol 1e-5."""
    from synth import workload
    p, run = workload("dense_n256_d1024_k20")
    g = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"])
    r = oracle_fit(p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"])
    assert_fit_close(g, r)
    # FP32 CG loses orthogonality a little faster than FP64 CG near the tolerance
    assert np.all(np.abs(g["cg_iters"] - r["cg_iters"]) <= np.maximum(3, 0.1 * r["cg_iters"]))
    assert g["flags"] == r["flags"]


def test_fit_f32_forms_agree(cf):
    """The tensor-core (TF32 split) and CUDA-core FP32 forms give the same fit
    within the FP32 parity tolerance, and both match the oracle."""
    from synth import workload
    p, run = workload("dense_n256_d1024_k20")
    a = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_F32_TF32X3)
    b = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"], precision=cf.COFEM_F32)
    r = oracle_fit(p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"])
    assert_fit_close(a, r)
    assert_fit_close(b, r)


def test_fit_graph_and_direct_modes_identical(cf):
    p = dense_gaussian(77, 301, 9, 20.0, seed=5)
    a = gpu_fit(cf, p, 5, 6, 1e-6, 300, use_graph=1)
    b = gpu_fit(cf, p, 5, 6, 1e-6, 300, use_graph=0)
    for k in ("mu", "s", "alpha", "cg_iters"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["flags"] == b["flags"]


def test_fit_deterministic_and_host_pointers(cf):
    p = dense_gaussian(100, 400, 10, 25.0, seed=6)
    a = gpu_fit(cf, p, 8, 5, 1e-6, 300)
    b = gpu_fit(cf, p, 8, 5, 1e-6, 300, host=True)
    for k in ("mu", "s", "alpha", "cg_iters"):
        np.testing.assert_array_equal(a[k], b[k])


@pytest.mark.parametrize("K", [1, 5, 63])
def test_fit_ragged_sizes_and_probe_counts(cf, K):
    p = dense_gaussian(200, 501, 10, 15.0, seed=K)
    g = gpu_fit(cf, p, K, 8, 1e-5, 400)
    r = oracle_fit(p, K, 8, 1e-5, 400)
    assert_fit_close(g, r)


@pytest.mark.parametrize("variant", ["frobenius", "precond_one", "rr3", "alpha0"])
def test_fit_variants(cf, variant):
    p = dense_gaussian(250, 500, 10, 15.0, seed=11)
    kw_g, kw_o = {}, {}
    if variant == "rr3":
        # replacement needs a system whose FP32 recursive/true residual drift
        # stays below tol: an overdetermined dictionary (Phi^T Phi full rank)
        p = dense_gaussian(500, 400, 10, 15.0, seed=11)
    alpha0 = None
    if variant == "frobenius":
        kw_g["conv"], kw_o["conv"] = cf.COFEM_CONV_FROBENIUS, "frobenius"
    elif variant == "precond_one":
        kw_g["precond"], kw_o["precond"] = cf.COFEM_PRECOND_ONE, "one"
    elif variant == "rr3":
        kw_g["rr_period"], kw_o["rr_period"] = 3, 3
    else:
        alpha0 = np.exp(np.random.default_rng(0).uniform(-1, 3, 500)).astype(np.float32)
        kw_o["alpha0"] = alpha0.astype(np.float64)
    g = gpu_fit(cf, p, 16, 10, 1e-5, 400, alpha0=alpha0, **kw_g)
    r = oracle_fit(p, 16, 10, 1e-5, 400, **kw_o)
    assert_fit_close(g, r)


@pytest.mark.parametrize("case", ["dense_under", "dense_over", "toeplitz"])
def test_fit_precision_form_matches_oracle(cf, case):
    """Residual replacement with the accurate residual (X as an FP32 pair,
    B - A X in FP32-pair products) and the end-of-E-step check, against the
    oracle's replacement in FP64: the same fit, and every reported true
    residual within tol (none of these fits runs out of CG steps)."""
    if case == "toeplitz":
        p = toeplitz_calcium(6000, 256, 0.01, 15.0, seed=2)
        args = (8, 3, 1e-14, 25)          # fixed CG steps, as in the test below
    else:
        p = dense_gaussian(250, 500, 10, 15.0, seed=11) if case == "dense_under" else \
            dense_gaussian(500, 400, 10, 15.0, seed=11)
        args = (16, 10, 1e-5, 400)
    K, T = args[0], args[1]
    kind = cf.COFEM_OP_DENSE if p.kind == "dense" else cf.COFEM_OP_TOEPLITZ
    mu, s_, al = (np.empty(p.D, np.float32) for _ in range(3))
    it = np.empty(T, np.int32)
    with cf.CoFEM(p.N, p.D, kind, p.phi, p.L, rr_period=7) as m:
        flags = cf.cofem_fit(m.h, p.y, p.beta, None, *args, mu, s_, al, it)
        res = cf.cofem_true_residuals(m.h, T, K)
        n_rr, n_check = cf.cofem_fit_stats(m.h)
    g = dict(mu=mu, s=s_, alpha=al, cg_iters=it, flags=flags)
    r = oracle_fit(p, *args, rr_period=7)
    assert_fit_close(g, r)
    assert n_rr == sum(int(u) // 7 for u in it) and n_check >= T
    if case == "toeplitz":
        # fixed step count: the check reports the residual left after 25 steps
        np.testing.assert_allclose(res, r["true_res"], rtol=2e-2)
    else:
        assert not flags & cf.COFEM_FLAG_CG_NOT_CONVERGED and np.all(res <= args[2]), (flags, res.max())


def test_fit_check_residual_reports_the_true_residual(cf):
    """check_residual = 1 (no replacement; X held as the FP32 pair): the fit
    matches the oracle, and the reported true residual of the mu column equals
    its FP64 residual computed on the host from the returned mu (mu's own FP32
    rounding is far below it)."""
    p = dense_gaussian(250, 500, 10, 15.0, seed=11)
    K, T = 16, 6
    outs = [np.empty(p.D, np.float32) for _ in range(3)]
    it = np.empty(T, np.int32)
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, check_residual=1) as m:
        flags = cf.cofem_fit(m.h, p.y, p.beta, None, K, T, 1e-5, 400, *outs, it)
        res = cf.cofem_true_residuals(m.h, T, K)
    assert_fit_close(dict(mu=outs[0], s=outs[1], alpha=outs[2], cg_iters=it, flags=flags),
                     oracle_fit(p, K, T, 1e-5, 400))
    # mu of the last E-step solves A(alpha^(T)) mu = b
    Phi = p.phi.astype(np.float64)
    b = p.beta * (Phi.T @ p.y.astype(np.float64))
    mu = outs[0].astype(np.float64)
    r = b - p.beta * (Phi.T @ (Phi @ mu)) - outs[2].astype(np.float64) * mu
    host = np.linalg.norm(r) / np.linalg.norm(b.astype(np.float32).astype(np.float64))
    assert abs(res[-1, 0] - host) <= 1e-6 + 0.05 * host, (res[-1, 0], host)
    assert np.all(np.isfinite(res))
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi) as m:   # not measured without the option
        cf.cofem_fit(m.h, p.y, p.beta, None, K, 1, 1e-5, 400, *outs)
        with pytest.raises(cf.CofemError):
            cf.cofem_true_residuals(m.h, 1, K)


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_fit_warm_start_matches_oracle(cf, precision):
    """Warm start with probe reuse (every E-step draws the t = 1 probes; E-step
    t >= 2 starts from the previous X with R = B - A X): the same fit as the
    oracle's, CG step counts included (on these problems the warm start takes
    more CG steps than a cold start: the M-step makes the previous solution's
    components on the inactive coordinates stiff)."""
    p = dense_gaussian(250, 500, 10, 15.0, seed=11)
    K, T, tol = 16, 8, 1e-6
    prec = cf.COFEM_BF16 if precision == "bf16" else cf.COFEM_F32
    phi = bf16_round(p.phi) if precision == "bf16" else p.phi
    g = gpu_fit(cf, p, K, T, tol, 600, precision=prec, warm_start=1)
    r = oracle_fit(p, K, T, tol, 600, phi=phi, warm_start=True)
    assert_fit_close(g, r)
    assert np.all(np.abs(g["cg_iters"] - r["cg_iters"]) <= np.maximum(3, 0.15 * r["cg_iters"]))


@pytest.mark.parametrize("path", ["direct", "fft"])
def test_fit_toeplitz_small(cf, path):
    """The calcium-style convolution makes the E-step system so ill-conditioned
    that even FP64 CG needs > 1000 steps for tol 1e-5; compare the two CG
    trajectories at a fixed iteration count instead (tol unreachable)."""
    p = toeplitz_calcium(6000, 256, 0.01, 15.0, seed=2)
    tp = cf.COFEM_TOEPLITZ_FFT if path == "fft" else cf.COFEM_TOEPLITZ_DIRECT
    g = gpu_fit(cf, p, 8, 3, 1e-14, 25, toeplitz_path=tp)
    r = oracle_fit(p, 8, 3, 1e-14, 25)
    assert np.all(g["cg_iters"] == 25) and np.all(r["cg_iters"] == 25)
    assert_fit_close(g, r)


@pytest.mark.parametrize("kind", ["dense", "toeplitz"])
def test_fit_rectified_prior_matches_oracle(cf, kind):
    """Rectified Gaussian prior (non-negativity subsection): the M-step takes
    the truncated second moment (FP64, erfcx) on the GPU; the fit matches the
    oracle's.  The convolution case is the paper's calcium setting (non-negative
    spikes), compared at a fixed CG iteration count as in the test above."""
    if kind == "dense":
        p = dense_gaussian(200, 501, 10, 15.0, seed=5)
        args = (12, 8, 1e-5, 400)
    else:
        p = toeplitz_calcium(6000, 256, 0.01, 15.0, seed=2)
        args = (8, 3, 1e-14, 25)
    g = gpu_fit(cf, p, *args, prior=cf.COFEM_PRIOR_RECTIFIED)
    r = oracle_fit(p, *args, prior="rectified")
    assert_fit_close(g, r)
    # the prior changed the M-step: alpha differs from the Gaussian prior's
    ga = gpu_fit(cf, p, *args)
    assert not np.array_equal(ga["alpha"], g["alpha"])


@pytest.mark.parametrize("path", ["two_pass", "single_pass"])
def test_fit_bf16_matches_oracle_on_quantised_dictionary(cf, path):
    p = dense_gaussian(250, 500, 10, 15.0, seed=12)
    g = gpu_fit(cf, p, 16, 10, 1e-5, 400, precision=cf.COFEM_BF16, dense_path=PATHS[path])
    r = oracle_fit(p, 16, 10, 1e-5, 400, phi=bf16_round(p.phi))
    assert_fit_close(g, r)


def test_fit_fp8_matches_oracle_on_quantised_dictionary(cf):
    p = dense_gaussian(250, 500, 10, 15.0, seed=12)
    s, dec = e4m3_quantise(p.phi)
    g = gpu_fit(cf, p, 16, 10, 1e-5, 400, precision=cf.COFEM_FP8_E4M3)
    r = oracle_fit(p, 16, 10, 1e-5, 400, phi=s.astype(np.float64)[:, None] * dec)
    assert_fit_close(g, r)


def test_fit_single_pass_graph_direct_and_repeat_identical(cf):
    """The cooperative single-pass operator inside the CUDA graph and from the
    host loop, and twice in a row: identical bits (its reductions have a fixed
    order)."""
    p = dense_gaussian(700, 3000, 30, 20.0, seed=9)
    kw = dict(precision=cf.COFEM_BF16, dense_path=2)
    a = gpu_fit(cf, p, 12, 5, 1e-6, 300, use_graph=1, **kw)
    b = gpu_fit(cf, p, 12, 5, 1e-6, 300, use_graph=0, **kw)
    c = gpu_fit(cf, p, 12, 5, 1e-6, 300, use_graph=1, **kw)
    for k in ("mu", "s", "alpha", "cg_iters"):
        np.testing.assert_array_equal(a[k], b[k])
        np.testing.assert_array_equal(a[k], c[k])
    assert a["flags"] == b["flags"] == c["flags"] == 0


@pytest.mark.parametrize("precision", ["bf16", "tf32x3", "fp8"])
@pytest.mark.parametrize("rr_period", [0, 7])
def test_fit_overlapped_launch_identical(cf, precision, rr_period):
    """Programmatic dependent launch of the CG-step kernels (graph edges and
    direct launches) changes only when kernels start: the fit has the same bits
    as with plain stream order."""
    prec = {"bf16": cf.COFEM_BF16, "tf32x3": cf.COFEM_F32_TF32X3, "fp8": cf.COFEM_FP8_E4M3}[precision]
    p = dense_gaussian(700, 3000, 30, 20.0, seed=11)
    kw = dict(precision=prec, dense_path=1, rr_period=rr_period)
    if precision == "tf32x3" and rr_period > 0:
        # residual replacement needs products exact on the stored dictionary
        with pytest.raises(cf.CofemError) as e:
            cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, 0, **kw)
        assert e.value.status == cf.COFEM_ERR_UNSUPPORTED
        return
    ref = gpu_fit(cf, p, 12, 4, 1e-6, 300, use_graph=1, overlap_launch=0, **kw)
    for use_graph in (1, 0):
        g = gpu_fit(cf, p, 12, 4, 1e-6, 300, use_graph=use_graph, overlap_launch=1, **kw)
        for k in ("mu", "s", "alpha", "cg_iters"):
            np.testing.assert_array_equal(g[k], ref[k])
        assert g["flags"] == ref["flags"]
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, 0, **kw) as m:
        assert cf.cofem_graph_info(m.h) == (0, 0)
        m.fit(p.y, p.beta, 12, 2, 1e-6, 300)
        assert cf.cofem_graph_info(m.h) == (1, 1)


def test_fit_edge_cases(cf):
    p = dense_gaussian(50, 130, 5, 20.0, seed=1)
    a0 = np.linspace(0.5, 2.0, 130).astype(np.float32)
    # T = 1: no M-step, alpha^(T) = alpha0
    g = gpu_fit(cf, p, 3, 1, 1e-6, 200, alpha0=a0)
    np.testing.assert_array_equal(g["alpha"], a0)
    # cg_maxit = 1: not converged flag, one iteration per EM step
    g = gpu_fit(cf, p, 3, 2, 1e-12, 1)
    assert g["flags"] & cf.COFEM_FLAG_CG_NOT_CONVERGED and np.all(g["cg_iters"] == 1)
    r = oracle_fit(p, 3, 2, 1e-12, 1)
    assert_fit_close(g, r)
    # y = 0: b = 0, the mu column starts converged, mu = 0
    import dataclasses
    z = dataclasses.replace(p, y=np.zeros_like(p.y))
    g = gpu_fit(cf, z, 3, 2, 1e-6, 200)
    assert np.all(g["mu"] == 0.0)


def test_fit_breakdown_flagged_and_column_frozen(cf):
    """A column whose p^T A p is not a positive finite number is flagged and
    frozen, and the fit goes on: with Phi = 0 and alpha0 = 0 the Jacobi
    preconditioner M = beta theta + alpha is zero, so the probe columns start
    with an infinite direction and pi = NaN; mu stays 0 (b = 0), the M-step
    then clamps alpha at alpha_max and the next E-step is regular."""
    import dataclasses
    p = dense_gaussian(50, 130, 5, 20.0, seed=3)
    z = dataclasses.replace(p, phi=np.zeros_like(p.phi))
    g = gpu_fit(cf, z, 3, 3, 1e-6, 200, alpha0=np.zeros(130, np.float32))
    assert g["flags"] & cf.COFEM_FLAG_BREAKDOWN
    for k in ("mu", "s", "alpha"):
        assert np.all(np.isfinite(g[k])), k
    assert np.all(g["mu"] == 0.0)
    np.testing.assert_allclose(g["alpha"], 1e12, rtol=1e-5)


def test_fit_rejects_nonfinite_and_bad_args(cf):
    p = dense_gaussian(20, 40, 2, 20.0, seed=1)
    with cf.CoFEM(20, 40, cf.COFEM_OP_DENSE, p.phi) as m:
        out = [np.empty(40, np.float32) for _ in range(3)]
        bad = p.y.copy()
        bad[3] = np.nan
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_fit(m.h, bad, p.beta, None, 2, 2, 1e-5, 10, *out)
        assert e.value.status == cf.COFEM_ERR_NONFINITE
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_fit(m.h, p.y, -1.0, None, 2, 2, 1e-5, 10, *out)
        assert e.value.status == cf.COFEM_ERR_INVALID_ARG
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_fit(m.h, p.y, p.beta, None, 64, 2, 1e-5, 10, *out)
        assert e.value.status == cf.COFEM_ERR_INVALID_ARG
        # the handle still works after rejected calls
        cf.cofem_fit(m.h, p.y, p.beta, None, 2, 2, 1e-5, 10, *out)
    badphi = p.phi.copy()
    badphi[1, 1] = np.inf
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_create(20, 40, cf.COFEM_OP_DENSE, badphi, 0, cf.default_opts())
    assert e.value.status == cf.COFEM_ERR_NONFINITE


# ---------------------------------------------------------------------------
# Properties that hold at any size: the returned mu solves the last E-step
# system A(alpha^(T)) mu = beta Phi^T y to the CG tolerance (checked in FP64),
# and the returned alpha^(T) is what the M-step makes of the previous E-step.
# ---------------------------------------------------------------------------
def _mu_residual(phi, y, beta, alpha, mu):
    Phi = phi.astype(np.float64)
    b = beta * (Phi.T @ y.astype(np.float64))
    m = mu.astype(np.float64)
    Am = beta * (Phi.T @ (Phi @ m)) + alpha.astype(np.float64) * m
    return np.linalg.norm(b - Am) / np.linalg.norm(b)


def test_fit_dense_n2500_d10000_k32_properties(cf):
    """Full 2500 x 10000 FP32 workload (K = 32, T = 50) in its benchmark form
    (3xTF32 tensor-core products) and with FP32 FMA: every E-step converges, mu
    solves its system, NMSE is that of a converged SBL fit."""
    from synth import workload
    p, run = workload("dense_n2500_d10000_k32")
    assert run["precision"] == "tf32x3"
    g = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_F32_TF32X3)
    assert not g["flags"] & cf.COFEM_FLAG_CG_NOT_CONVERGED
    assert _mu_residual(p.phi, p.y, p.beta, g["alpha"], g["mu"]) < 10 * run["cg_tol"]
    nmse_tc = 20 * np.log10(np.linalg.norm(g["mu"] - p.z) / np.linalg.norm(p.z))
    assert nmse_tc < -20.0
    g = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"])
    assert not g["flags"] & cf.COFEM_FLAG_CG_NOT_CONVERGED
    assert _mu_residual(p.phi, p.y, p.beta, g["alpha"], g["mu"]) < 10 * run["cg_tol"]
    nmse_db = 20 * np.log10(np.linalg.norm(g["mu"] - p.z) / np.linalg.norm(p.z))
    assert nmse_db < -20.0
    assert abs(nmse_db - nmse_tc) < 0.1


def test_fit_dense_n8192_d32768_fp8_properties(cf):
    """The 8192 x 32768 problem with the FP8 E4M3 dictionary: every E-step
    converges, mu solves the E-step system of the quantised dictionary, and
    the NMSE stays within 4 dB of the BF16 form."""
    from synth import workload
    p, run = workload("dense_n8192_d32768_k32_bf16")
    g = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_FP8_E4M3)
    assert not g["flags"] & cf.COFEM_FLAG_CG_NOT_CONVERGED, g["cg_iters"]
    phq = np.empty(p.phi.shape, np.float32)
    for i0 in range(0, p.N, 512):                      # quantise by row blocks
        s, dec = e4m3_quantise(p.phi[i0:i0 + 512])
        phq[i0:i0 + 512] = s[:, None] * dec
    assert _mu_residual(phq, p.y, p.beta, g["alpha"], g["mu"]) < 10 * run["cg_tol"]
    b = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_BF16)
    nm = [20 * np.log10(np.linalg.norm(x["mu"] - p.z) / np.linalg.norm(p.z)) for x in (g, b)]
    assert nm[0] < nm[1] + 4.0, nm


def test_fit_dense_n8192_d32768_bf16_properties(cf):
    """Full 8192 x 32768 BF16 workload in the benchmark's launch configuration:
    mu solves the E-step system of the quantised dictionary, and the BF16 and
    FP32 forms reach the same NMSE within 0.1 dB."""
    from synth import workload
    p, run = workload("dense_n8192_d32768_k32_bf16")
    assert run["rr_period"] == 20
    g = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_BF16, rr_period=run["rr_period"], want_res=True)
    assert g["flags"] == 0, (g["flags"], g["cg_iters"])
    # the precision form: every column's true residual, measured on the GPU at
    # the end of every E-step, within the CG tolerance
    assert np.all(g["true_res"] <= run["cg_tol"]), g["true_res"].max()
    assert _mu_residual(bf16_round(p.phi), p.y, p.beta, g["alpha"], g["mu"]) < 10 * run["cg_tol"]
    f = gpu_fit(cf, p, run["K"], run["T"], run["cg_tol"], run["cg_maxit"], seed=run["seed"],
                precision=cf.COFEM_F32, rr_period=run["rr_period"])
    nm = [20 * np.log10(np.linalg.norm(x["mu"] - p.z) / np.linalg.norm(p.z)) for x in (g, f)]
    assert abs(nm[0] - nm[1]) < 0.1, nm


def test_bounded_device_waits_run_out_and_the_context_stays_usable(cf):
    """Failure detection without a GPU fault: the grid-counter wait and the
    mbarrier wait of the persistent kernels, run on a counter and an mbarrier
    that nothing completes, give up by their limits; the call reports
    COFEM_ERR_CUDA with COFEM_FLAG_DEVICE_TIMEOUT, and a fit on a fresh
    handle afterwards runs normally."""
    import time
    t0 = time.perf_counter()
    st, flags, msg = cf.cofem_selftest_bounded_wait(0.05)
    wall = time.perf_counter() - t0
    assert st == cf.COFEM_ERR_CUDA and flags & cf.COFEM_FLAG_DEVICE_TIMEOUT, (st, flags, msg)
    assert "timed out" in msg and wall < 30.0
    p = dense_gaussian(250, 500, 10, 15.0, seed=12)
    g = gpu_fit(cf, p, 16, 10, 1e-5, 400, precision=cf.COFEM_BF16)
    r = oracle_fit(p, 16, 10, 1e-5, 400, phi=bf16_round(p.phi))
    assert_fit_close(g, r)
    assert not g["flags"] & cf.COFEM_FLAG_DEVICE_TIMEOUT


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
def test_fit_replacement_on_the_last_cg_step_graph_matches_host(cf, precision):
    """The fit graph's CG loop ends at every replacement step and goes round
    again after the replacement; with the CG budget a multiple of the
    replacement period (and a tolerance no column meets) the last step is a
    replacement step: the graph gives the host loop's bits, flags and counts."""
    prec = {"bf16": cf.COFEM_BF16, "fp8": cf.COFEM_FP8_E4M3}[precision]
    p = dense_gaussian(300, 1200, 12, 20.0, seed=21)
    out = []
    for use_graph in (1, 0):
        with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, 0, precision=prec, rr_period=7,
                      use_graph=use_graph) as m:
            K, T = 8, 3
            mu, s, alpha = (np.zeros(p.D, np.float32) for _ in range(3))
            it = np.zeros(T, np.int32)
            flags = cf.cofem_fit(m.h, p.y, p.beta, None, K, T, 1e-12, 14, mu, s, alpha, it)
            out.append((mu, s, alpha, it, flags, cf.cofem_fit_stats(m.h)))
    (a, b) = out
    for x, y in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(x, y)
    assert a[4] == b[4] and a[4] & cf.COFEM_FLAG_CG_NOT_CONVERGED
    assert a[5] == b[5] and a[5][0] >= 2 * T
    assert np.all(a[3] >= 14)
