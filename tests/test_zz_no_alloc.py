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


def test_noalloc_is_captured_by_a_cuda_graph_and_allocates_nothing(cf):
    """After one call on the device (which looks up the scratch array), a call
    allocates no device memory (torch's allocator and the driver's free bytes
    are unchanged across it), and a call inside a stream capture (torch's
    strictest mode) records into the graph: replays give the regular
    operator's result for the inputs in place at replay time."""
    from synth import dense_gaussian
    dev = torch.device("cuda", 0)
    N, D, Q = 400, 1500, 12
    p = dense_gaussian(N, D, 5, 20.0, seed=7)
    rng = np.random.default_rng(7)
    phi = torch.from_numpy(p.phi).to(dev)
    alpha = torch.from_numpy(np.exp(rng.uniform(-2, 4, D)).astype(np.float32)).to(dev)
    V = torch.empty((Q, D), device=dev)
    out = torch.empty((Q, D), device=dev)
    beta = 9.0
    V.copy_(torch.from_numpy(rng.standard_normal((Q, D)).astype(np.float32)))
    cf.cofem_apply_dense_noalloc(phi, N, D, D, V, Q, alpha, beta, out)   # first call: scratch lookup
    torch.cuda.synchronize(dev)
    used, free = torch.cuda.memory_allocated(dev), torch.cuda.mem_get_info(dev)[0]
    cf.cofem_apply_dense_noalloc(phi, N, D, D, V, Q, alpha, beta, out)
    torch.cuda.synchronize(dev)
    assert torch.cuda.memory_allocated(dev) == used
    assert torch.cuda.mem_get_info(dev)[0] == free

    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            cf.cofem_apply_dense_noalloc(phi, N, D, D, V, Q, alpha, beta, out, stream=side)
    torch.cuda.synchronize(dev)
    with cf.CoFEM(N, D, cf.COFEM_OP_DENSE, phi) as m:
        for rep in range(2):
            V.copy_(torch.from_numpy(rng.standard_normal((Q, D)).astype(np.float32)))
            out.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize(dev)
            ref = torch.empty((Q, D), device=dev)
            cf.cofem_apply_operator(m.h, V, Q, alpha, beta, ref, want_pi=False)
            got, want = out.cpu().numpy(), ref.cpu().numpy()
            for q in range(Q):
                assert _rel(got[q], want[q]) < TOL, (rep, q, _rel(got[q], want[q]))
