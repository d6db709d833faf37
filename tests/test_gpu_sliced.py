"""GPU parity of the precision form's accurate product (row a6) in both of its
forms: FP32 pairs on the CUDA cores (COFEM_RESIDUAL_FP32_PAIRS) and exact
integer slices on the tensor cores (COFEM_RESIDUAL_SLICED), through the C ABI
(cofem_accurate_product), against the oracle's FP64 dense operator on the same
BF16 dictionary; and whole precision-form fits with each form against the
oracle's FP64 replacement.

Tolerance of the product, element by element, with S1 = |Phi~|^T |Phi~| |x|
(the terms of the first product, which cancel when x lies near the null space
of Phi~) and S2 = |Phi~|^T |Phi~ x| (those of the second, which do not):
|out - ref| <= 2^-32 S1 + 2^-20 S2 for both forms.  The FP32-pair form
carries about 2^-48 S1 (error-free first product) plus FP32 sums of 32 terms
in the second product; the sliced form about 2^-37 S1 in all (40-bit digits
of x and of Phi~ x relative to their column's largest entry, 24-bit digits of
Phi~ relative to its row's largest, digit products of order above 4
dropped) and a little more in S2, checked as <= 2^-34 S1 + 2^-26 S2.  The
FP64 reference carries about
2^-53 sqrt(D) S1.  What residual replacement needs is B - A X to well below
tol ||b|| with |A| |x| up to 10^4 ||b||: about 2^-33 of S1."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import DenseOperator, cofem as oracle_cofem  # noqa: E402
from synth import dense_gaussian  # noqa: E402

DEV = "cuda:0"
TOL_S1, TOL_S2 = 2.0 ** -32, 2.0 ** -20


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


def bf16_round(x):
    """float32 -> nearest bfloat16 (ties to even), as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _pair_block(rng, Q, D):
    """Q x D vectors as FP32 pairs (hi + lo of an FP64 value): column scales
    from 1e-6 to 1e3, one sparse column and (Q > 2) one zero column."""
    X = rng.standard_normal((Q, D)) * np.logspace(-6, 3, Q)[:, None]
    if Q > 1:
        X[1] *= rng.random(D) < 0.03
    if Q > 2:
        X[2] = 0.0
    Xh = X.astype(np.float32)
    Xl = (X - Xh.astype(np.float64)).astype(np.float32)
    return Xh, Xl


def _bounds(phi_b, x):
    """(reference product in FP64, S1, S2) for one vector x."""
    op, absop = DenseOperator(phi_b), DenseOperator(np.abs(phi_b))
    t = op.apply(x)
    return op.apply_t(t), absop.apply_t(absop.apply(np.abs(x))), absop.apply_t(np.abs(t))


def _check_product(out, phi_b, Xh, Xl, cols=None, tol1=TOL_S1, tol2=TOL_S2):
    """Every element of the sampled columns within tol1 S1 + tol2 S2."""
    cols = range(Xh.shape[0]) if cols is None else cols
    for q in cols:
        x = Xh[q].astype(np.float64) + Xl[q].astype(np.float64)
        ref, s1, s2 = _bounds(phi_b, x)
        err = np.abs(out[q] - ref)
        bound = tol1 * s1 + tol2 * s2
        assert np.all(err <= bound), (q, float(np.max(err / np.where(bound > 0, bound, 1.0))))


# The sliced form, tighter: about 2^-37 S1 from the first product and, in the
# second, digits of the transposed dictionary relative to each column's
# largest entry (an entry below 2^-15 of it keeps 24 bits below that point
# only: about 2^-25 of the largest entry, 2^-29 S2 at N = 256).
SLICED_TOL = (2.0 ** -34, 2.0 ** -26)


def _stored_dictionary(phi, precision):
    """The dictionary the handle computes with, FP64: bf16(Phi), or the FP8
    form's diag(s) decode(codes) (the parity module's E4M3 quantiser)."""
    if precision == "bf16":
        return bf16_round(phi).astype(np.float64)
    from test_gpu_parity import e4m3_quantise
    sc, dec = e4m3_quantise(phi)
    return sc.astype(np.float64)[:, None] * dec


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("path", ["sliced", "pairs"])
@pytest.mark.parametrize("N,D,Q", [(256, 1024, 1), (300, 1000, 17), (512, 2048, 33), (640, 1536, 48),
                                   (129, 4100, 21)])
def test_accurate_product_matches_fp64(cf, precision, path, N, D, Q):
    if precision == "fp8" and 3 * Q > 128:
        pytest.skip("the FP8 operator takes 3(K+1) <= 128")
    rng = np.random.default_rng(N * 7 + Q)
    phi = (rng.standard_normal((N, D)) / np.sqrt(N)).astype(np.float32)
    Xh, Xl = _pair_block(rng, Q, D)
    rp = cf.COFEM_RESIDUAL_SLICED if path == "sliced" else cf.COFEM_RESIDUAL_FP32_PAIRS
    prec = cf.COFEM_BF16 if precision == "bf16" else cf.COFEM_FP8_E4M3
    out = np.empty((Q, D), np.float64)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi, precision=prec, check_residual=1, residual_path=rp) as m:
        cf.cofem_accurate_product(m.h, Xh, Xl, Q, out)
        out2 = np.empty_like(out)
        cf.cofem_accurate_product(m.h, Xh, Xl, Q, out2)   # the same bits on a second call
    np.testing.assert_array_equal(out, out2)
    pb = _stored_dictionary(phi, precision)
    _check_product(out, pb, Xh, Xl)
    if path == "sliced":
        _check_product(out, pb, Xh, Xl, None, *SLICED_TOL)


def _ilogb(v):
    return np.floor(np.log2(v)).astype(np.int64)


def _dict_digits(v, e):
    """Three signed base-256 digits of each bfloat16 entry relative to 2^e of
    its row (round to nearest at each step, in FP32 as the scheme states)."""
    w = (v.astype(np.float32) * (2.0 ** (8 - e)).astype(np.float32)).astype(np.float32)
    out = []
    for _ in range(3):
        d = np.rint(w).astype(np.float32)
        out.append(d.astype(np.int64))
        w = ((w - d) * np.float32(256)).astype(np.float32)
    return out


def _int_digits(I):
    """Five signed base-256 digits of 64-bit integers (lowest in [-128, 127])."""
    out = [None] * 5
    for b in range(4, 0, -1):
        r = ((I + 128) & 255) - 128
        out[b] = r
        I = (I - r) >> 8
    out[0] = I
    return out


def _sliced_model(M, e, digits):
    """Z = sum over digit products a + b <= 4 of 2^(8 (4 - a - b)) M_a V_b in
    exact 64-bit integer arithmetic."""
    A = _dict_digits(M, e[:, None])
    acc = [sum(A[a] @ digits[d - a] for a in range(3) if 0 <= d - a <= 4) for d in range(5)]
    return sum(acc[d] * (1 << (8 * (4 - d))) for d in range(5))


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("N,D,Q", [(256, 1024, 1), (300, 1000, 17), (512, 2048, 33)])
def test_sliced_product_is_the_exact_integer_scheme(cf, precision, N, D, Q):
    """The tensor cores sum the digit products exactly: the sliced product
    equals, bit for bit, the same slicing evaluated in 64-bit integers on the
    host (both products, exponents and digits as the kernels define them; the
    FP8 form slices the codes' values and scales t by s_i^2)."""
    rng = np.random.default_rng(N * 7 + Q)
    phi = (rng.standard_normal((N, D)) / np.sqrt(N)).astype(np.float32)
    Xh, Xl = _pair_block(rng, Q, D)
    out = np.empty((Q, D), np.float64)
    prec = cf.COFEM_BF16 if precision == "bf16" else cf.COFEM_FP8_E4M3
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi, precision=prec, check_residual=1,
                  residual_path=cf.COFEM_RESIDUAL_SLICED) as m:
        cf.cofem_accurate_product(m.h, Xh, Xl, Q, out)
    if precision == "bf16":
        pb, rs2 = bf16_round(phi), None
    else:
        from test_gpu_parity import e4m3_quantise
        sc, dec = e4m3_quantise(phi)
        pb, rs2 = dec.astype(np.float32), sc.astype(np.float64) ** 2
    E1 = _ilogb(np.abs(pb).max(axis=1)) + 2
    E2 = _ilogb(np.abs(pb).max(axis=0)) + 2
    mx = np.abs(Xh).max(axis=1)
    F = np.where(mx > 0, _ilogb(np.where(mx > 0, mx, 1.0)) + 3, 0)
    sc = 2.0 ** (40 - F[:, None])
    I = np.rint(Xh.astype(np.float64) * sc).astype(np.int64) + np.rint(Xl.astype(np.float64) * sc).astype(np.int64)
    Z1 = _sliced_model(pb, E1, [d.T for d in _int_digits(I)])                      # N x Q
    t = Z1.astype(np.float64) * 2.0 ** (E1[:, None] + F[None, :] - 48)
    if rs2 is not None:
        t = t * rs2[:, None]
    tm = np.abs(t).max(axis=0)
    G = np.where(tm > 0, _ilogb(np.where(tm > 0, tm, 1.0)) + 3, 0)
    It = np.rint(t * 2.0 ** (40 - G[None, :])).astype(np.int64)
    Z2 = _sliced_model(np.ascontiguousarray(pb.T), E2, _int_digits(It))           # D x Q
    U = Z2.astype(np.float64) * 2.0 ** (E2[:, None] + G[None, :] - 48)
    np.testing.assert_array_equal(out, U.T)


def test_accurate_product_forms_agree_on_device_buffers(cf):
    """Device-resident inputs and output; the two forms agree within the
    tolerance, and the sliced form meets its tighter one."""
    rng = np.random.default_rng(5)
    N, D, Q = 1024, 4096, 33
    phi = torch.from_numpy((rng.standard_normal((N, D)) / np.sqrt(N)).astype(np.float32)).to(DEV)
    Xh, Xl = _pair_block(rng, Q, D)
    xh, xl = torch.from_numpy(Xh).to(DEV), torch.from_numpy(Xl).to(DEV)
    outs = []
    for rp in (cf.COFEM_RESIDUAL_SLICED, cf.COFEM_RESIDUAL_FP32_PAIRS):
        o = torch.empty((Q, D), dtype=torch.float64, device=DEV)
        with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi, precision=cf.COFEM_BF16, rr_period=20, residual_path=rp) as m:
            cf.cofem_accurate_product(m.h, xh, xl, Q, o)
        outs.append(o.cpu().numpy())
    pb = bf16_round(phi.cpu().numpy()).astype(np.float64)
    _check_product(outs[0], pb, Xh, Xl, None, *SLICED_TOL)
    for q in range(Q):
        _, s1, s2 = _bounds(pb, Xh[q].astype(np.float64) + Xl[q].astype(np.float64))
        assert np.all(np.abs(outs[0][q] - outs[1][q]) <= TOL_S1 * s1 + TOL_S2 * s2), q


def test_accurate_product_full_size_sampled(cf):
    """The 8192 x 32768 dictionary with 33 columns (the benchmark's precision
    form), sampled columns compared with the FP64 product."""
    rng = np.random.default_rng(8)
    N, D, Q = 8192, 32768, 33
    phi32 = torch.randn((N, D), device=DEV, generator=torch.Generator(device=DEV).manual_seed(3)) / np.sqrt(N)
    Xh, Xl = _pair_block(rng, Q, D)
    out = torch.empty((Q, D), dtype=torch.float64, device=DEV)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi32, precision=cf.COFEM_BF16, check_residual=1,
                  residual_path=cf.COFEM_RESIDUAL_SLICED) as m:
        cf.cofem_accurate_product(m.h, torch.from_numpy(Xh).to(DEV), torch.from_numpy(Xl).to(DEV), Q, out)
    pb = bf16_round(phi32.cpu().numpy()).astype(np.float64)
    del phi32
    _check_product(out.cpu().numpy(), pb, Xh, Xl, [0, 1, 2, 16, 32], *SLICED_TOL)


def _oracle_fit(p, K, T, tol, maxit, **kw):
    return oracle_cofem(DenseOperator(bf16_round(p.phi)), p.y, p.beta, K, T, tol, maxit, 2, **kw)


@pytest.mark.parametrize("path", ["sliced", "pairs"])
@pytest.mark.parametrize("case", ["dense_under", "dense_over"])
def test_fit_precision_form_bf16_matches_oracle(cf, path, case):
    """BF16 dictionary, replacement every 7 CG steps and the end-of-E-step
    check, with each accurate residual form: the fit matches the oracle's FP64
    replacement on bf16(Phi) (same tolerances as every fit), and every reported
    true residual is within tol."""
    from test_gpu_parity import assert_fit_close
    p = dense_gaussian(250, 500, 10, 15.0, seed=11) if case == "dense_under" else \
        dense_gaussian(500, 400, 10, 15.0, seed=11)
    K, T, tol, maxit = 16, 10, 1e-5, 400
    rp = cf.COFEM_RESIDUAL_SLICED if path == "sliced" else cf.COFEM_RESIDUAL_FP32_PAIRS
    mu, s_, al = (np.empty(p.D, np.float32) for _ in range(3))
    it = np.empty(T, np.int32)
    with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, precision=cf.COFEM_BF16, rr_period=7,
                  residual_path=rp) as m:
        flags = cf.cofem_fit(m.h, p.y, p.beta, None, K, T, tol, maxit, mu, s_, al, it)
        res = cf.cofem_true_residuals(m.h, T, K)
        n_rr, _ = cf.cofem_fit_stats(m.h)
        _, _, k_rr, _ = cf.cofem_operator_info(m.h)
    assert k_rr == (7 if path == "sliced" else 4)
    g = dict(mu=mu, s=s_, alpha=al, cg_iters=it, flags=flags)
    r = _oracle_fit(p, K, T, tol, maxit, rr_period=7)
    assert_fit_close(g, r)
    assert n_rr == sum(int(u) // 7 for u in it)
    assert not flags & cf.COFEM_FLAG_CG_NOT_CONVERGED and np.all(res <= tol), (flags, res.max())


def test_sliced_form_rejected_where_it_does_not_apply(cf):
    """SLICED needs a BF16 dense dictionary and K + 1 <= 48: otherwise the
    first fit reports UNSUPPORTED; AUTO falls back to the FP32 pairs."""
    p = dense_gaussian(120, 300, 6, 20.0, seed=4)
    outs = [np.empty(p.D, np.float32) for _ in range(3)]
    for prec, K in ((cf.COFEM_F32, 8), (cf.COFEM_BF16, 50)):
        with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, precision=prec, rr_period=5,
                      residual_path=cf.COFEM_RESIDUAL_SLICED) as m:
            with pytest.raises(cf.CofemError) as e:
                cf.cofem_fit(m.h, p.y, p.beta, None, K, 1, 1e-5, 50, *outs)
            assert e.value.status == cf.COFEM_ERR_UNSUPPORTED
        with cf.CoFEM(p.N, p.D, cf.COFEM_OP_DENSE, p.phi, precision=prec, rr_period=5) as m:
            cf.cofem_fit(m.h, p.y, p.beta, None, K, 1, 1e-5, 50, *outs)
            assert cf.cofem_operator_info(m.h)[2] == 4   # the FP32-pair form
