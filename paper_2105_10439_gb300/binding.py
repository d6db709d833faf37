"""ctypes binding of libcofem (include/cofem.h).

Argument marshalling only: every function here converts Python arguments to
the C types of the same-named entry point and raises on a non-zero status.
Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); both must be contiguous float32 (int32 for cg_iters).  No computation
happens on this side.  If libcofem.so has not been built, importing the
package raises immediately: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcofem.so")

COFEM_OK = 0
COFEM_ERR_INVALID_ARG = 1
COFEM_ERR_NOMEM = 2
COFEM_ERR_CUDA = 3
COFEM_ERR_NONFINITE = 4
COFEM_ERR_UNSUPPORTED = 5
COFEM_ERR_NOT_FOUND = 6

COFEM_OP_DENSE = 0
COFEM_OP_TOEPLITZ = 1
COFEM_OP_DCT = 2
COFEM_F32 = 0
COFEM_BF16 = 1
COFEM_F32_TF32X3 = 2
COFEM_FP8_E4M3 = 3
COFEM_PRECOND_JACOBI = 0
COFEM_PRECOND_ONE = 1
COFEM_PRECOND_NONE = 2
COFEM_CONV_PER_COLUMN = 0
COFEM_CONV_FROBENIUS = 1
COFEM_PATH_AUTO = 0
COFEM_PATH_TWO_PASS = 1
COFEM_PATH_SINGLE_PASS = 2
COFEM_TOEPLITZ_AUTO = 0
COFEM_TOEPLITZ_DIRECT = 1
COFEM_TOEPLITZ_FFT = 2
COFEM_PRIOR_GAUSSIAN = 0
COFEM_PRIOR_RECTIFIED = 1
COFEM_SERVE_HOST_LOOP = 1
COFEM_RESIDUAL_AUTO = 0
COFEM_RESIDUAL_FP32_PAIRS = 1
COFEM_RESIDUAL_SLICED = 2
COFEM_FLAG_CG_NOT_CONVERGED = 1
COFEM_FLAG_ALPHA_CLAMPED = 2
COFEM_FLAG_BREAKDOWN = 4
COFEM_FLAG_DEVICE_TIMEOUT = 8


class cofem_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("precond", C.c_int),
        ("conv", C.c_int),
        ("rr_period", C.c_int),
        ("alpha_max", C.c_double),
        ("seed", C.c_ulonglong),
        ("stream", C.c_void_p),
        ("use_graph", C.c_int),
        ("dense_path", C.c_int),
        ("max_sms", C.c_int),
        ("overlap_launch", C.c_int),
        ("prior", C.c_int),
        ("check_residual", C.c_int),
        ("warm_start", C.c_int),
        ("toeplitz_path", C.c_int),
        ("residual_path", C.c_int),
    ]


class cofem_request(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("N", C.c_longlong), ("D", C.c_longlong), ("L", C.c_longlong),
        ("phi", C.c_void_p), ("y", C.c_void_p), ("beta", C.c_double), ("alpha0", C.c_void_p),
        ("K", C.c_int), ("T_em", C.c_int), ("cg_tol", C.c_double), ("cg_maxit", C.c_int),
        ("precision", C.c_int), ("precond", C.c_int), ("conv", C.c_int), ("rr_period", C.c_int),
        ("alpha_max", C.c_double), ("seed", C.c_ulonglong),
        ("mu", C.c_void_p), ("s", C.c_void_p), ("alpha", C.c_void_p), ("cg_iters", C.c_void_p),
        ("max_sms", C.c_int), ("prior", C.c_int),
    ]


class cofem_result(C.Structure):
    _fields_ = [("status", C.c_int), ("flags", C.c_uint), ("queue_ms", C.c_double), ("run_ms", C.c_double),
                ("message", C.c_char * 160)]


class cofem_server_stats(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("steps", C.c_longlong), ("fit_steps", C.c_longlong),
                ("graphs_built", C.c_longlong)]


class CofemError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"libcofem status {status}: {message}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(LIB_PATH)
    vp, i, ll, d, ull = C.c_void_p, C.c_int, C.c_longlong, C.c_double, C.c_ulonglong
    sig = {
        "cofem_default_opts": (None, [C.POINTER(cofem_opts)]),
        "cofem_create": (i, [C.POINTER(vp), ll, ll, i, vp, ll, C.POINTER(cofem_opts)]),
        "cofem_create_dct": (i, [C.POINTER(vp), ll, ll, vp, C.POINTER(cofem_opts)]),
        "cofem_fit": (i, [vp, vp, d, vp, i, i, d, i, vp, vp, vp, vp, vp]),
        "cofem_fit_multitask": (i, [vp, i, vp, d, vp, i, i, d, i, vp, vp, vp, vp, vp]),
        "cofem_destroy": (i, [vp]),
        "cofem_status_string": (C.c_char_p, [i]),
        "cofem_last_error": (C.c_char_p, []),
        "cofem_probe_fill": (i, [ull, i, i, ll, vp, vp]),
        "cofem_apply_operator": (i, [vp, vp, i, vp, d, vp, vp]),
        "cofem_get_theta": (i, [vp, vp]),
        "cofem_phit_y": (i, [vp, vp, d, vp]),
        "cofem_device_bytes": (ll, [vp]),
        "cofem_get_dictionary": (i, [vp, vp]),
        "cofem_operator_info": (i, [vp, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "cofem_graph_info": (i, [vp, C.POINTER(i), C.POINTER(i)]),
        "cofem_true_residuals": (i, [vp, vp]),
        "cofem_fit_stats": (i, [vp, C.POINTER(i), C.POINTER(i)]),
        "cofem_selftest_bounded_wait": (i, [d, C.POINTER(C.c_uint)]),
        "cofem_time_true_residual": (i, [vp, i, i, C.POINTER(d), C.POINTER(d)]),
        "cofem_accurate_product": (i, [vp, vp, vp, i, vp]),
        "cofem_time_operator": (i, [vp, i, i, C.POINTER(d)]),
        "cofem_apply_dense_noalloc": (i, [vp, ll, ll, ll, vp, i, vp, d, vp, vp]),
        "cofem_estimate_bytes": (ll, [i, ll, ll, ll, i, i]),
        "cofem_server_create": (i, [C.POINTER(vp), ll, i]),
        "cofem_server_create_packed": (i, [C.POINTER(vp), ll, i, i, i]),
        "cofem_server_get_stats": (i, [vp, C.POINTER(cofem_server_stats)]),
        "cofem_submit": (i, [vp, C.POINTER(cofem_request), C.POINTER(C.c_ulonglong)]),
        "cofem_poll": (i, [vp, C.c_ulonglong, C.POINTER(i)]),
        "cofem_wait": (i, [vp, C.c_ulonglong, C.POINTER(cofem_result)]),
        "cofem_server_destroy": (i, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _check(status: int):
    if status != COFEM_OK:
        msg = lib.cofem_last_error().decode(errors="replace")
        raise CofemError(status, msg or lib.cofem_status_string(status).decode())


def _ptr(x, dtype=np.float32, allow_none=False):
    """Address of a contiguous array (numpy host array or torch tensor)."""
    if x is None:
        if allow_none:
            return None
        raise ValueError("array argument is None")
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"need a C-contiguous {np.dtype(dtype).name} array")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        import torch  # only for the dtype check
        want = {np.float32: torch.float32, np.int32: torch.int32, np.float64: torch.float64}[dtype]
        if x.dtype != want or not x.is_contiguous():
            raise TypeError(f"need a contiguous {want} tensor")
        return x.data_ptr()
    raise TypeError(f"unsupported array type {type(x)}")


def default_opts(**kw) -> cofem_opts:
    o = cofem_opts()
    lib.cofem_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream if hasattr(v, "cuda_stream") else int(v)
        setattr(o, k, v)
    return o


def cofem_create(N: int, D: int, kind: int, phi, L: int = 0, opts: cofem_opts | None = None) -> int:
    h = C.c_void_p()
    _check(lib.cofem_create(C.byref(h), N, D, kind, _ptr(phi), L, C.byref(opts) if opts is not None else None))
    return h.value


def cofem_create_dct(N: int, D: int, rows, opts: cofem_opts | None = None) -> int:
    """rows: N distinct int32 indices in [0, D) (host or device)."""
    h = C.c_void_p()
    _check(lib.cofem_create_dct(C.byref(h), N, D, _ptr(rows, np.int32), C.byref(opts) if opts is not None else None))
    return h.value


def cofem_fit(h: int, y, beta: float, alpha0, K: int, T_em: int, cg_tol: float, cg_maxit: int,
              mu, s, alpha, cg_iters=None) -> int:
    """Returns the COFEM_FLAG_* bits of the fit."""
    flags = C.c_uint(0)
    _check(lib.cofem_fit(h, _ptr(y), float(beta), _ptr(alpha0, allow_none=True), int(K), int(T_em),
                         float(cg_tol), int(cg_maxit), _ptr(mu), _ptr(s), _ptr(alpha),
                         _ptr(cg_iters, np.int32, allow_none=True), C.byref(flags)))
    return flags.value


def cofem_fit_multitask(h: int, L: int, Y, beta: float, alpha0, K: int, T_em: int, cg_tol: float, cg_maxit: int,
                        mu, s, alpha, cg_iters=None) -> int:
    """L tasks sharing the handle's dictionary and alpha; Y, mu, s are L x N /
    L x D row-major.  Returns the COFEM_FLAG_* bits of the fit."""
    flags = C.c_uint(0)
    _check(lib.cofem_fit_multitask(h, int(L), _ptr(Y), float(beta), _ptr(alpha0, allow_none=True), int(K),
                                   int(T_em), float(cg_tol), int(cg_maxit), _ptr(mu), _ptr(s), _ptr(alpha),
                                   _ptr(cg_iters, np.int32, allow_none=True), C.byref(flags)))
    return flags.value


def cofem_destroy(h: int) -> None:
    _check(lib.cofem_destroy(h))


def cofem_probe_fill(seed: int, t: int, K: int, D: int, out, stream=None) -> None:
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.cofem_probe_fill(seed, t, K, D, _ptr(out), st))


def cofem_apply_operator(h: int, V, Q: int, alpha, beta: float, Psi, want_pi: bool = True):
    pi = np.zeros(Q, dtype=np.float64) if want_pi else None
    _check(lib.cofem_apply_operator(h, _ptr(V), Q, _ptr(alpha), float(beta), _ptr(Psi),
                                    pi.ctypes.data if pi is not None else None))
    return pi


def cofem_get_theta(h: int, theta) -> None:
    _check(lib.cofem_get_theta(h, _ptr(theta)))


def cofem_phit_y(h: int, y, beta: float, b) -> None:
    _check(lib.cofem_phit_y(h, _ptr(y), float(beta), _ptr(b)))


def cofem_time_operator(h: int, Q: int, reps: int) -> float:
    ms = C.c_double(0.0)
    _check(lib.cofem_time_operator(h, Q, reps, C.byref(ms)))
    return ms.value


def cofem_apply_dense_noalloc(phi, N: int, D: int, ld: int, V, Q: int, alpha, beta: float, Psi,
                              stream=None) -> None:
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib.cofem_apply_dense_noalloc(_ptr(phi), N, D, ld, _ptr(V), Q, _ptr(alpha), float(beta), _ptr(Psi), st))


def cofem_estimate_bytes(kind: int, N: int, D: int, L: int, precision: int, K: int) -> int:
    return int(lib.cofem_estimate_bytes(kind, N, D, L, precision, K))


def cofem_server_create(hbm_budget_bytes: int, max_slots: int) -> int:
    h = C.c_void_p()
    _check(lib.cofem_server_create(C.byref(h), int(hbm_budget_bytes), int(max_slots)))
    return h.value


def cofem_server_create_packed(hbm_budget_bytes: int, max_fits: int, prep_threads: int = 4, flags: int = 0) -> int:
    h = C.c_void_p()
    _check(lib.cofem_server_create_packed(C.byref(h), int(hbm_budget_bytes), int(max_fits), int(prep_threads),
                                          int(flags)))
    return h.value


def cofem_server_get_stats(srv: int) -> dict:
    st = cofem_server_stats()
    _check(lib.cofem_server_get_stats(srv, C.byref(st)))
    return {k: getattr(st, k) for k, _ in cofem_server_stats._fields_}


def make_request(kind, N, D, phi, y, beta, K, T_em, cg_tol, cg_maxit, mu, s, alpha, cg_iters=None, L=0,
                 alpha0=None, max_sms=0, **opts) -> cofem_request:
    o = default_opts(**opts)
    return cofem_request(kind=kind, N=N, D=D, L=L, phi=_ptr(phi), y=_ptr(y), beta=float(beta),
                         alpha0=_ptr(alpha0, allow_none=True), K=K, T_em=T_em, cg_tol=float(cg_tol),
                         cg_maxit=cg_maxit, precision=o.precision, precond=o.precond, conv=o.conv,
                         rr_period=o.rr_period, alpha_max=o.alpha_max, seed=o.seed, mu=_ptr(mu), s=_ptr(s),
                         alpha=_ptr(alpha), cg_iters=_ptr(cg_iters, np.int32, allow_none=True), max_sms=max_sms,
                         prior=o.prior)


def cofem_submit(srv: int, req: cofem_request) -> int:
    t = C.c_ulonglong(0)
    _check(lib.cofem_submit(srv, C.byref(req), C.byref(t)))
    return t.value


def cofem_poll(srv: int, ticket: int) -> bool:
    d = C.c_int(0)
    _check(lib.cofem_poll(srv, ticket, C.byref(d)))
    return bool(d.value)


def cofem_wait(srv: int, ticket: int) -> cofem_result:
    r = cofem_result()
    _check(lib.cofem_wait(srv, ticket, C.byref(r)))
    return r


def cofem_server_destroy(srv: int) -> None:
    _check(lib.cofem_server_destroy(srv))


def cofem_device_bytes(h: int) -> int:
    return int(lib.cofem_device_bytes(h))


def cofem_get_dictionary(h: int, out) -> None:
    """The dictionary the handle computes with, FP32 N x D (host or device array)."""
    _check(lib.cofem_get_dictionary(h, _ptr(out)))


def cofem_operator_info(h: int) -> tuple[int, int, int, int]:
    """(path, kernels per CG-loop operator application, per residual
    replacement, kernels of the CG update/direction per step)."""
    path, kc, kr, ks = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(lib.cofem_operator_info(h, C.byref(path), C.byref(kc), C.byref(kr), C.byref(ks)))
    return path.value, kc.value, kr.value, ks.value


def cofem_true_residuals(h: int, T_em: int, K: int) -> np.ndarray:
    """(T_em, K+1) FP64 array of the last fit's true relative residuals
    ||b_q - A x_q|| / ||b_q|| per EM iteration and column."""
    out = np.empty((T_em, K + 1), dtype=np.float64)
    _check(lib.cofem_true_residuals(h, out.ctypes.data))
    return out


def cofem_accurate_product(h: int, Xh, Xl, Q: int, out) -> None:
    """out (Q x D float64) = Phi~^T Phi~ (Xh + Xl) by the handle's accurate
    residual form; Xh, Xl are Q x D float32 (host or device)."""
    _check(lib.cofem_accurate_product(h, _ptr(Xh), _ptr(Xl), int(Q), _ptr(out, np.float64)))


def cofem_time_true_residual(h: int, Q: int, reps: int) -> tuple[float, float]:
    """(ms per accurate residual, ms per first product Phi~ X)."""
    a, b = C.c_double(0.0), C.c_double(0.0)
    _check(lib.cofem_time_true_residual(h, Q, reps, C.byref(a), C.byref(b)))
    return a.value, b.value


def cofem_selftest_bounded_wait(seconds: float) -> tuple[int, int, str]:
    """Runs the bounded-wait self-test: (status, flags, message), without
    raising (the waits are meant to run out: COFEM_ERR_CUDA with
    COFEM_FLAG_DEVICE_TIMEOUT)."""
    f = C.c_uint(0)
    st = lib.cofem_selftest_bounded_wait(float(seconds), C.byref(f))
    return st, f.value, lib.cofem_last_error().decode(errors="replace")


def cofem_fit_stats(h: int) -> tuple[int, int]:
    """(residual replacements, true-residual checks) of the last fit."""
    r, c = C.c_int(), C.c_int()
    _check(lib.cofem_fit_stats(h, C.byref(r), C.byref(c)))
    return r.value, c.value


def cofem_graph_info(h: int) -> tuple[int, int]:
    """(fit graph built, its CG-step kernels joined by programmatic edges)."""
    built, ov = C.c_int(), C.c_int()
    _check(lib.cofem_graph_info(h, C.byref(built), C.byref(ov)))
    return built.value, ov.value


class CoFEM:
    """Owning wrapper of one handle (closes it on exit / garbage collection).
    kind COFEM_OP_DCT takes the kept rows (int32) in place of phi."""

    def __init__(self, N, D, kind, phi, L=0, **opts):
        self.N, self.D, self.kind = int(N), int(D), kind
        self.opts = default_opts(**opts)
        if kind == COFEM_OP_DCT:
            self.h = cofem_create_dct(N, D, phi, self.opts)
        else:
            self.h = cofem_create(N, D, kind, phi, L, self.opts)

    def fit(self, y, beta, K, T, cg_tol, cg_maxit, alpha0=None, out=None):
        """Host-array convenience: returns dict(mu, s, alpha, cg_iters, flags)."""
        if out is None:
            out = dict(mu=np.empty(self.D, np.float32), s=np.empty(self.D, np.float32),
                       alpha=np.empty(self.D, np.float32), cg_iters=np.empty(T, np.int32))
        out["flags"] = cofem_fit(self.h, y, beta, alpha0, K, T, cg_tol, cg_maxit, out["mu"], out["s"],
                                 out["alpha"], out["cg_iters"])
        return out

    def close(self):
        if getattr(self, "h", None):
            cofem_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
