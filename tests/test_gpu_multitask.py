"""Multi-task CoFEM on the GPU (the multi-task subsection of Sec. III, the
shared-dictionary case) against the FP64 oracle's cofem_multitask with the
same per-task probes: L tasks share alpha and beta, their L (K+1) columns
run as one batched PCG, and the M-step is alpha_j = L / sum_l (mu_lj^2 + s_lj).
Tolerances as for single-task fits (relative l2: mu 1e-4, s 1e-3, 1/alpha
1e-3 and well-determined alpha 1e-3), per task."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import DenseOperator, ToeplitzOperator, cofem_multitask  # noqa: E402
from synth import dense_gaussian_multitask, double_exponential_filter  # noqa: E402


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def bf16_round(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def gpu_multitask(cf, kind, N, D, phi, L_filter, Y, beta, K, T, tol, maxit, **opts):
    Lt = Y.shape[0]
    mu = np.empty((Lt, D), np.float32)
    s = np.empty((Lt, D), np.float32)
    al = np.empty(D, np.float32)
    it = np.empty(T, np.int32)
    with cf.CoFEM(N, D, kind, phi, L_filter, **opts) as m:
        flags = cf.cofem_fit_multitask(m.h, Lt, np.ascontiguousarray(Y), beta, None, K, T, tol, maxit, mu, s, al,
                                       it)
    return dict(mu=mu, s=s, alpha=al, cg_iters=it, flags=flags)


def check(g, r):
    for l in range(g["mu"].shape[0]):
        e = (rel(g["mu"][l], r["mu"][l]), rel(g["s"][l], r["s"][l]))
        assert e[0] <= 1e-4 and e[1] <= 1e-3, (l, e)
    # alpha where it is well determined: active, second moment within 1e-2 of
    # the largest and not a cancelling difference
    m2 = 1.0 / r["alpha"]
    act = (r["alpha"] < 1e6) & (m2 >= 1e-2 * m2.max()) & (m2 >= 0.1 * np.mean(r["mu"] ** 2 + np.abs(r["s"]), axis=0))
    assert rel(1.0 / g["alpha"], 1.0 / r["alpha"]) <= 1e-3
    assert rel(g["alpha"][act], r["alpha"][act]) <= 1e-3


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_multitask_dense_matches_oracle(cf, precision):
    # 15 dB, tol 1e-6: the FP64 fit moves by < 1e-5 under a 100x tighter tol
    p = dense_gaussian_multitask(250, 500, 10, 15.0, 3, seed=4)
    K, T, tol, maxit = 15, 8, 1e-6, 600
    prec = cf.COFEM_BF16 if precision == "bf16" else cf.COFEM_F32
    g = gpu_multitask(cf, cf.COFEM_OP_DENSE, p.N, p.D, p.phi, 0, p.Y, p.beta, K, T, tol, maxit, precision=prec,
                      seed=7)
    phi = bf16_round(p.phi) if precision == "bf16" else p.phi
    r = cofem_multitask([DenseOperator(phi)] * p.L, list(p.Y), p.beta, K, T, tol, maxit, seed=7)
    check(g, r)
    # near tol 1e-6 FP32 CG may take a few more steps than FP64 CG
    assert np.all(np.abs(g["cg_iters"] - r["cg_iters"]) <= np.maximum(3, 0.15 * r["cg_iters"]))


def test_multitask_one_task_is_the_single_task_fit(cf):
    """L = 1 is cofem_fit bit for bit (task 0 draws the single-task probes)."""
    p = dense_gaussian_multitask(200, 501, 10, 15.0, 1, seed=5)
    a = gpu_multitask(cf, cf.COFEM_OP_DENSE, p.N, p.D, p.phi, 0, p.Y, p.beta, 12, 5, 1e-6, 300)
    mu, s, al = (np.empty(p.D, np.float32) for _ in range(3))
    it = np.empty(5, np.int32)
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi) as m:
        cf.cofem_fit(m.h, p.Y[0], p.beta, None, 12, 5, 1e-6, 300, mu, s, al, it)
    np.testing.assert_array_equal(a["mu"][0], mu)
    np.testing.assert_array_equal(a["s"][0], s)
    np.testing.assert_array_equal(a["alpha"], al)
    np.testing.assert_array_equal(a["cg_iters"], it)


def test_multitask_graph_and_host_loop_identical_and_wide_block(cf):
    """A 64-column block (L = 4 tasks of K = 15 probes) on the tensor-core
    operator: the CUDA graph and the host-driven loop give the same bits, and
    both match the oracle."""
    # 15 dB, tol 1e-7: the FP64 fit moves by < 2e-5 under a 100x tighter tol
    p = dense_gaussian_multitask(300, 700, 12, 15.0, 4, seed=6)
    K, T = 15, 5
    kw = dict(precision=cf.COFEM_BF16)
    a = gpu_multitask(cf, cf.COFEM_OP_DENSE, p.N, p.D, p.phi, 0, p.Y, p.beta, K, T, 1e-7, 600, use_graph=1, **kw)
    b = gpu_multitask(cf, cf.COFEM_OP_DENSE, p.N, p.D, p.phi, 0, p.Y, p.beta, K, T, 1e-7, 600, use_graph=0, **kw)
    for k in ("mu", "s", "alpha", "cg_iters"):
        np.testing.assert_array_equal(a[k], b[k])
    r = cofem_multitask([DenseOperator(bf16_round(p.phi))] * p.L, list(p.Y), p.beta, K, T, 1e-7, 600, seed=2)
    check(a, r)


def test_multitask_convolution_fixed_steps(cf):
    """Several calcium traces sharing one convolution filter (fixed CG step
    count, as for the single-task convolution parity test)."""
    D, L_f, Lt = 4000, 256, 2
    h = double_exponential_filter(L_f)
    rng = np.random.default_rng(3)
    op = ToeplitzOperator(h, D)
    Z = (rng.random((Lt, D)) < 0.01) * rng.exponential(1.0, (Lt, D))
    clean = np.stack([op.apply(z) for z in Z])
    sigma2 = float(np.mean(np.sum(clean ** 2, axis=1))) / (D * 10 ** 1.5)
    Y = (clean + rng.standard_normal(clean.shape) * np.sqrt(sigma2)).astype(np.float32)
    g = gpu_multitask(cf, cf.COFEM_OP_TOEPLITZ, D, D, h, L_f, Y, 1.0 / sigma2, 8, 3, 1e-14, 25)
    r = cofem_multitask([op] * Lt, list(Y), 1.0 / sigma2, 8, 3, 1e-14, 25, seed=2)
    assert np.all(g["cg_iters"] == 25) and np.all(r["cg_iters"] == 25)
    check(g, r)


def test_multitask_rejections(cf):
    p = dense_gaussian_multitask(40, 80, 3, 20.0, 5, seed=1)
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi) as m:
        out = (np.empty((5, 80), np.float32), np.empty((5, 80), np.float32), np.empty(80, np.float32))
        with pytest.raises(cf.CofemError) as e:    # 5 x 13 > 64 columns
            cf.cofem_fit_multitask(m.h, 5, p.Y, p.beta, None, 12, 2, 1e-5, 10, *out)
        assert e.value.status == cf.COFEM_ERR_INVALID_ARG
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, prior=cf.COFEM_PRIOR_RECTIFIED) as m:
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_fit_multitask(m.h, 2, p.Y[:2].copy(), p.beta, None, 4, 2, 1e-5, 10, out[0][:2].copy(),
                                   out[1][:2].copy(), out[2])
        assert e.value.status == cf.COFEM_ERR_UNSUPPORTED
