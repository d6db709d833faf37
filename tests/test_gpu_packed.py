"""Packed serving (cofem_server_create_packed) through the C ABI: the CG steps
of all admitted fits run in shared launches (one packed GEMM per product, one
launch of each vector kernel), so a request's result must not depend on the
requests it shares the launches with (the same bits alone and in a mix), and
must match the FP64 oracle on the dictionary it computes with, within the fit
tolerances of the other parity tests (mu <= 1e-4, s, 1/alpha and
well-determined alpha <= 1e-3, relative l2)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import DenseOperator, cofem as oracle_cofem  # noqa: E402
from synth import dense_gaussian  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


def bf16_round(x):
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def _make(cf, p, K, T, precision, tol=1e-5, seed=2):
    D = p.D
    out = dict(mu=torch.empty(D, device=DEV), s=torch.empty(D, device=DEV), alpha=torch.empty(D, device=DEV),
               it=torch.empty(T, dtype=torch.int32, device=DEV), phi=torch.from_numpy(p.phi).to(DEV),
               y=torch.from_numpy(p.y).to(DEV))
    out["req"] = cf.make_request(cf.COFEM_OP_DENSE, p.N, D, out["phi"], out["y"], p.beta, K, T, tol, 400,
                                 out["mu"], out["s"], out["alpha"], out["it"], precision=precision, seed=seed)
    return out


def _np(o):
    return {k: o[k].cpu().numpy() for k in ("mu", "s", "alpha", "it")}


def _prec(cf, name):
    return cf.COFEM_BF16 if name == "bf16" else cf.COFEM_F32_TF32X3


def _oracle(p, K, T, precision_name, tol=1e-5):
    phi = bf16_round(p.phi) if precision_name == "bf16" else p.phi
    return oracle_cofem(DenseOperator(phi), p.y, p.beta, K, T, tol, 400, 2)


def _close(g, r):
    from test_gpu_parity import assert_fit_close
    return assert_fit_close(dict(mu=g["mu"], s=g["s"], alpha=g["alpha"], cg_iters=g["it"]), r)


@pytest.mark.parametrize("precision", ["bf16", "tf32x3"])
def test_packed_same_alone_and_in_mix_and_matches_oracle(cf, precision):
    prec = _prec(cf, precision)
    target = dense_gaussian(250, 500, 10, 15.0, seed=11)
    # mix members 0 and 4 are conditioned like the target (their own FP32
    # fits are within the parity tolerances of FP64: 15 dB, N / D = 1/2);
    # the larger ones only share the launches
    others = [dense_gaussian(n, d, max(1, d // 50), 15.0 if i in (0, 4) else 20.0, seed=30 + i)
              for i, (n, d) in enumerate([(300, 600), (1024, 4096), (512, 2048), (2048, 8192),
                                          (400, 800), (800, 3200), (1500, 6000)])]
    srv = cf.cofem_server_create_packed(40 << 30, 16, 4)
    try:
        a = _make(cf, target, 16, 10, prec)
        r = cf.cofem_wait(srv, cf.cofem_submit(srv, a["req"]))
        assert r.status == 0, r.message
        alone = _np(a)
        b = _make(cf, target, 16, 10, prec)
        mix = [_make(cf, p, 8 + 8 * (i % 3), 6, prec) for i, p in enumerate(others)]
        tickets = [cf.cofem_submit(srv, m["req"]) for m in mix[:4]]
        tb = cf.cofem_submit(srv, b["req"])
        tickets += [cf.cofem_submit(srv, m["req"]) for m in mix[4:]]
        rb = cf.cofem_wait(srv, tb)
        rs = [cf.cofem_wait(srv, t) for t in tickets]
        assert rb.status == 0, rb.message
        assert all(x.status == 0 for x in rs), [x.message for x in rs if x.status != 0]
        in_mix = _np(b)
    finally:
        cf.cofem_server_destroy(srv)
    for k in ("mu", "s", "alpha", "it"):
        np.testing.assert_array_equal(alone[k], in_mix[k])
    _close(alone, _oracle(target, 16, 10, precision))
    # the mix's requests are fits of their own problems too
    for i in (0, 4):
        _close(_np(mix[i]), _oracle(others[i], 8 + 8 * (i % 3), 6, precision))


def test_packed_many_requests_with_arrivals(cf):
    """Requests of different sizes and probe counts submitted while others
    run (admission between steps), more of them at once than the step tables
    first hold (so the tables and the step graph grow): every one completes,
    and a sample matches its own fit alone on a fresh packed server bit for
    bit."""
    rng = np.random.default_rng(4)
    probs = []
    for i in range(48):
        D = int(rng.integers(256, 3073))
        probs.append((dense_gaussian(max(1, D // 4), D, max(1, int(0.03 * D)), float(rng.uniform(15, 30)),
                                     seed=100 + i), int(rng.choice([8, 16, 32]))))
    srv = cf.cofem_server_create_packed(40 << 30, 40, 4)
    import time
    try:
        reqs, tickets = [], []
        for i, (p, K) in enumerate(probs):
            reqs.append(_make(cf, p, K, 5, cf.COFEM_BF16))
            tickets.append(cf.cofem_submit(srv, reqs[-1]["req"]))
            if i % 12 == 11:
                time.sleep(0.05)
        rs = [cf.cofem_wait(srv, t) for t in tickets]
        stats = cf.cofem_server_get_stats(srv)
    finally:
        cf.cofem_server_destroy(srv)
    assert all(r.status == 0 for r in rs), [r.message for r in rs if r.status != 0]
    assert stats["fit_steps"] > 16 * stats["launches"], stats   # steps served many fits at once
    srv = cf.cofem_server_create_packed(8 << 30, 1, 1)
    try:
        for i in (0, 7, 19, 47):
            p, K = probs[i]
            a = _make(cf, p, K, 5, cf.COFEM_BF16)
            assert cf.cofem_wait(srv, cf.cofem_submit(srv, a["req"])).status == 0
            for k in ("mu", "s", "alpha", "it"):
                np.testing.assert_array_equal(_np(a)[k], _np(reqs[i])[k])
    finally:
        cf.cofem_server_destroy(srv)


def test_packed_rejects_what_it_does_not_take(cf):
    p = dense_gaussian(64, 256, 4, 20.0, seed=1)
    srv = cf.cofem_server_create_packed(1 << 30, 4, 1)
    try:
        for prec, kw in ((cf.COFEM_F32, {}), (cf.COFEM_BF16, dict(rr_period=5))):
            r = _make(cf, p, 4, 2, prec)
            if kw:
                r["req"].rr_period = kw["rr_period"]
            with pytest.raises(cf.CofemError) as e:
                cf.cofem_submit(srv, r["req"])
            assert e.value.status == cf.COFEM_ERR_UNSUPPORTED
    finally:
        cf.cofem_server_destroy(srv)


def test_packed_failing_request_is_isolated(cf):
    good = dense_gaussian(256, 1024, 20, 20.0, seed=3)
    bad = dense_gaussian(256, 1024, 20, 20.0, seed=4)
    bad.y[7] = np.nan
    srv = cf.cofem_server_create_packed(8 << 30, 4, 2)
    try:
        g = _make(cf, good, 8, 4, cf.COFEM_BF16)
        b = _make(cf, bad, 8, 4, cf.COFEM_BF16)
        tb = cf.cofem_submit(srv, b["req"])
        tg = cf.cofem_submit(srv, g["req"])
        rb, rg = cf.cofem_wait(srv, tb), cf.cofem_wait(srv, tg)
    finally:
        cf.cofem_server_destroy(srv)
    assert rb.status == cf.COFEM_ERR_NONFINITE and b"y contains NaN" in rb.message
    assert rg.status == 0 and np.all(np.isfinite(g["mu"].cpu().numpy()))


def test_packed_host_loop_matches_graph(cf):
    """The host-driven step loop (COFEM_SERVE_HOST_LOOP: the same kernels
    launched one step at a time, no graph) gives the same bits as the graph's
    device-side loop; dictionaries of 8192 to 16384 columns (together larger
    than L2, as for a profiler's capture of the packed GEMM)."""
    probs = [(dense_gaussian(D // 4, D, D // 50, 20.0, seed=200 + i), K)
             for i, (D, K) in enumerate([(16384, 16), (8192, 32), (12288, 8), (16384, 32)])]
    outs = []
    for flags in (0, cf.COFEM_SERVE_HOST_LOOP):
        srv = cf.cofem_server_create_packed(40 << 30, 8, 2, flags)
        try:
            reqs = [_make(cf, p, K, 2, cf.COFEM_BF16) for p, K in probs]
            rs = [cf.cofem_wait(srv, t) for t in [cf.cofem_submit(srv, r["req"]) for r in reqs]]
            assert all(r.status == 0 for r in rs), [r.message for r in rs if r.status != 0]
            outs.append([_np(r) for r in reqs])
        finally:
            cf.cofem_server_destroy(srv)
    for a, b in zip(*outs):
        for k in ("mu", "s", "alpha", "it"):
            np.testing.assert_array_equal(a[k], b[k])
