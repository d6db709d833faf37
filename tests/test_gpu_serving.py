"""Serving loop (continuous batching) through the C ABI: a request's result is
the same alone and in a mix of concurrent requests, admission respects the
memory budget, and one failing request does not disturb the others."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from synth import dense_gaussian  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def cf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2105_10439_gb300 as m
    return m


def _make(cf, p, K, T, precision, seed=2):
    D = p.D
    out = dict(mu=torch.empty(D, device=DEV), s=torch.empty(D, device=DEV), alpha=torch.empty(D, device=DEV),
               it=torch.empty(T, dtype=torch.int32, device=DEV), phi=torch.from_numpy(p.phi).to(DEV),
               y=torch.from_numpy(p.y).to(DEV))
    out["req"] = cf.make_request(cf.COFEM_OP_DENSE, p.N, D, out["phi"], out["y"], p.beta, K, T, 1e-5, 400,
                                 out["mu"], out["s"], out["alpha"], out["it"], precision=precision, seed=seed)
    return out


def _np(o):
    return {k: o[k].cpu().numpy() for k in ("mu", "s", "alpha", "it")}


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_result_same_alone_and_in_mix(cf, precision):
    prec = cf.COFEM_BF16 if precision == "bf16" else cf.COFEM_F32
    target = dense_gaussian(600, 2048, 40, 20.0, seed=5)
    others = [dense_gaussian(n, d, max(1, d // 30), 20.0, seed=10 + i)
              for i, (n, d) in enumerate([(256, 1024), (1024, 4096), (512, 2048), (2048, 8192),
                                          (300, 1500), (800, 3200), (1500, 6000)])]
    srv = cf.cofem_server_create(40 << 30, 4)
    try:
        a = _make(cf, target, 16, 8, prec)
        r = cf.cofem_wait(srv, cf.cofem_submit(srv, a["req"]))
        assert r.status == 0, r.message
        alone = _np(a)
        b = _make(cf, target, 16, 8, prec)
        mix = [_make(cf, p, 8 + 4 * (i % 3), 8, prec) for i, p in enumerate(others)]
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
    # and the same as a direct fit on a handle
    with cf.CoFEM(target.N, target.D, cf.COFEM_OP_DENSE, torch.from_numpy(target.phi).to(DEV),
                  precision=prec, seed=2) as m:
        c = _make(cf, target, 16, 8, prec)
        cf.cofem_fit(m.h, c["y"], target.beta, None, 16, 8, 1e-5, 400, c["mu"], c["s"], c["alpha"], c["it"])
    direct = _np(c)
    for k in ("mu", "s", "alpha", "it"):
        np.testing.assert_array_equal(alone[k], direct[k])


def test_admission_respects_budget(cf):
    ps = [dense_gaussian(1024, 4096, 40, 20.0, seed=20 + i) for i in range(3)]
    est = cf.cofem_estimate_bytes(cf.COFEM_OP_DENSE, 1024, 4096, 0, cf.COFEM_F32, 8)
    srv = cf.cofem_server_create(int(est * 1.5), 3)    # room for one request at a time
    try:
        reqs = [_make(cf, p, 8, 6, cf.COFEM_F32) for p in ps]
        ts = [cf.cofem_submit(srv, r["req"]) for r in reqs]
        rs = [cf.cofem_wait(srv, t) for t in ts]
    finally:
        cf.cofem_server_destroy(srv)
    assert all(r.status == 0 for r in rs)
    # one at a time: each request waited at least for the runs before it
    assert rs[1].queue_ms >= 0.9 * rs[0].run_ms
    assert rs[2].queue_ms >= 0.9 * (rs[0].run_ms + rs[1].run_ms)


def test_oversized_request_rejected(cf):
    p = dense_gaussian(64, 256, 4, 20.0, seed=1)
    srv = cf.cofem_server_create(1 << 20, 2)
    try:
        r = _make(cf, p, 4, 2, cf.COFEM_F32)
        with pytest.raises(cf.CofemError) as e:
            cf.cofem_submit(srv, r["req"])
        assert e.value.status == cf.COFEM_ERR_NOMEM
    finally:
        cf.cofem_server_destroy(srv)


def test_failing_request_is_isolated(cf):
    good = dense_gaussian(256, 1024, 20, 20.0, seed=3)
    bad = dense_gaussian(256, 1024, 20, 20.0, seed=4)
    bad.y[7] = np.nan
    srv = cf.cofem_server_create(8 << 30, 2)
    try:
        g = _make(cf, good, 8, 4, cf.COFEM_F32)
        b = _make(cf, bad, 8, 4, cf.COFEM_F32)
        tb = cf.cofem_submit(srv, b["req"])
        tg = cf.cofem_submit(srv, g["req"])
        rb, rg = cf.cofem_wait(srv, tb), cf.cofem_wait(srv, tg)
    finally:
        cf.cofem_server_destroy(srv)
    assert rb.status == cf.COFEM_ERR_NONFINITE and b"y contains NaN" in rb.message
    assert rg.status == 0 and np.all(np.isfinite(g["mu"].cpu().numpy()))
