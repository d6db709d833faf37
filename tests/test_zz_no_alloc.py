"""The allocation-free operator entry point (cofem_apply_dense_noalloc).

It serves callers that cannot allocate device memory (inside a stream capture,
under another framework's memory pool, or on a path that must not enter the
driver's allocator), keeping the product Phi V in a fixed device array of the
library.  Its output must equal the regular entry point's, within the operator
tolerance of the parity tests, on two calls in a row (the second with other
sizes, so leftovers of the first call in the shared array would show)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 2e-5   # relative l2 per column, as for the other operator parity tests


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


def test_noalloc_matches_regular_operator_on_two_calls(cf):
    from synth import dense_gaussian
    dev = torch.device("cuda", 0)
    for call, (N, D, Q) in enumerate([(300, 1000, 9), (517, 2049, 33)]):
        p = dense_gaussian(N, D, 5, 20.0, seed=100 + call)
        rng = np.random.default_rng(call)
        V = torch.from_numpy(rng.standard_normal((Q, D)).astype(np.float32)).to(dev)
        alpha = torch.from_numpy(np.exp(rng.uniform(-2, 4, D)).astype(np.float32)).to(dev)
        beta = 12.5 + call
        phi = torch.from_numpy(p.phi).to(dev)
        ref = torch.empty((Q, D), device=dev)
        with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi) as m:
            cf.cofem_apply_operator(m.h, V, Q, alpha, beta, ref, want_pi=False)
        out = torch.full((Q, D), float("nan"), device=dev)
        cf.cofem_apply_dense_noalloc(phi, N, D, D, V, Q, alpha, beta, out)
        torch.cuda.synchronize(dev)
        got, want = out.cpu().numpy(), ref.cpu().numpy()
        for q in range(Q):
            assert _rel(got[q], want[q]) < TOL, (call, q, _rel(got[q], want[q]))


def test_noalloc_rejects_sizes_beyond_its_array(cf):
    dev = torch.device("cuda", 0)
    N, D, Q = 40000, 8, 33          # N*Q = 1 320 000 > 1 048 576
    phi = torch.zeros((N, D), device=dev)
    V = torch.zeros((Q, D), device=dev)
    alpha = torch.ones(D, device=dev)
    out = torch.zeros((Q, D), device=dev)
    with pytest.raises(cf.CofemError) as e:
        cf.cofem_apply_dense_noalloc(phi, N, D, D, V, Q, alpha, 1.0, out)
    assert e.value.status == cf.COFEM_ERR_INVALID_ARG
    assert "exceeds the static scratch" in str(e.value)
