// C ABI of libcofem: handle lifetime, workspace, and the fit driver.  A fit is
// one CUDA-graph launch: an EM WHILE loop whose body runs the PCG
// initialisation, a CG WHILE loop (operator, fused update, an IF branch for
// residual replacement, direction update) and the fused M-step; the loop
// conditions are set on the device (cudaGraphSetConditional), so the host is
// only involved at the start and the end of the fit.
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <cstring>
#include <cmath>

#include "cofem_internal.cuh"

namespace {

thread_local char g_err[512] = "";

cofem_status fail(cofem_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

cofem_status cuda_fail(cudaError_t e, const char* what) {
    cudaGetLastError();  // clear sticky-free errors
    return fail(e == cudaErrorMemoryAllocation ? COFEM_ERR_NOMEM : COFEM_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// Device memory of a handle is stream-ordered (cudaMallocAsync / cudaFreeAsync
// on the handle's stream): unlike cudaFree, releasing it does not synchronise the
// whole device, so handles on different streams (concurrent requests) do not
// serialise each other.
template <typename T>
cofem_status dalloc(cofem_ctx* c, T** p, size_t count) {
    if (*p) return COFEM_OK;
    const size_t bytes = count * sizeof(T) > 0 ? count * sizeof(T) : 16;
    cudaError_t e = cudaMallocAsync((void**)p, bytes, c->stream);
    if (e != cudaSuccess) {
        *p = nullptr;
        return cuda_fail(e, "cudaMalloc");
    }
    c->bytes += (long long)bytes;
    c->alloc_bytes[(void*)*p] = bytes;
    return COFEM_OK;
}

template <typename T>
void dfree(cofem_ctx* c, T** p, size_t /*count*/) {
    if (*p) {
        cudaFreeAsync(*p, c->stream);
        auto it = c->alloc_bytes.find((void*)*p);
        if (it != c->alloc_bytes.end()) {
            c->bytes -= (long long)it->second;
            c->alloc_bytes.erase(it);
        }
        *p = nullptr;
    }
}

void free_graph(cofem_ctx* c) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->gexec = nullptr;
    c->graph = nullptr;
    c->graph_Q = -1;
}

// Sizes of the Q-dependent workspace (recomputed on every (re)allocation).
struct WsSizes {
    size_t xrp, u, t, tpart, part, ttpart, counters;
};

WsSizes ws_sizes(cofem_ctx* c, int Qcap) {
    WsSizes w{};
    w.xrp = (size_t)Qcap * c->Dp;
    const int QP = ((Qcap + 7) / 8) * 8;
    if (c->kind == COFEM_OP_DENSE && c->use_tc) {
        w.u = (size_t)Qcap * c->Dp;
        w.t = 0;
        w.tpart = 0;
        w.ttpart = (size_t)Qcap * ((c->Np + 1023) / 1024 + 1);
    } else if (c->kind == COFEM_OP_DENSE) {
        w.u = (size_t)c->S2 * Qcap * c->Dp;
        w.t = (size_t)c->Np * QP;
        w.tpart = (size_t)c->S1 * c->Np * QP;
        w.ttpart = (size_t)Qcap * (c->Np / 64 + 1);
    } else if (c->kind == COFEM_OP_DCT) {
        w.u = (size_t)Qcap * c->Dp;
        w.t = 0;
        w.tpart = 0;
        w.ttpart = (size_t)Qcap + 1;
    } else {
        w.u = (size_t)Qcap * c->Dp;
        w.t = 0;
        w.tpart = 0;
        const long long Bout = 2048 - (c->L - 1);
        w.ttpart = (size_t)Qcap * ((c->Dp + Bout - 1) / Bout + 1);
    }
    w.part = (size_t)3 * Qcap * c->nch;
    w.counters = 16 + (size_t)(c->Np / 64 + 1);
    return w;
}

// The precision form: X kept as an FP32 pair, accurate residual replacement
// (rr_period > 0) and the true-residual check at the end of each E-step.
bool precise(const cofem_ctx* c) { return c->opts.rr_period > 0 || c->opts.check_residual != 0; }

void free_precise(cofem_ctx* c) {
    sl_release(c);
    if (!c->Xlo) return;
    const DfSizes z = df_configure(c, c->Qcap);
    dfree(c, &c->Xlo, (size_t)c->Qcap * c->Dp);
    dfree(c, &c->Rt, (size_t)c->Qcap * c->Dp);
    dfree(c, &c->df_T, z.T);
    dfree(c, &c->df_thi, z.t);
    dfree(c, &c->df_tlo, z.t);
    dfree(c, &c->df_U, z.U);
}

void free_workspace(cofem_ctx* c) {
    if (c->Qcap == 0) return;
    free_precise(c);
    const WsSizes w = ws_sizes(c, c->Qcap);
    dfree(c, &c->X, w.xrp);
    dfree(c, &c->R, w.xrp);
    dfree(c, &c->P, w.xrp);
    dfree(c, &c->U, w.u);
    dfree(c, &c->T, w.t);
    dfree(c, &c->Tpart, w.tpart);
    dfree(c, &c->part, w.part);
    dfree(c, &c->tt_part, w.ttpart);
    dfree(c, &c->counters, w.counters);
    tc_release(c);
    c->Qcap = 0;
    free_graph(c);
}

// Make sure the fit workspace holds Q columns (the split configuration
// depends on Q, so any change of Q re-derives it and rebuilds the graph).
cofem_status ensure_workspace(cofem_ctx* c, int Q) {
    if (c->Qcap == Q && (!c->use_tc || c->tc)) return COFEM_OK;
    free_workspace(c);
    if (c->kind == COFEM_OP_DENSE) dense_configure(c, Q);
    const WsSizes w = ws_sizes(c, Q);
    cofem_status st;
    if ((st = dalloc(c, &c->X, w.xrp)) || (st = dalloc(c, &c->R, w.xrp)) || (st = dalloc(c, &c->P, w.xrp)) ||
        (st = dalloc(c, &c->U, w.u)) || (st = dalloc(c, &c->part, w.part)) ||
        (st = dalloc(c, &c->tt_part, w.ttpart)) || (st = dalloc(c, &c->counters, w.counters))) {
        c->Qcap = Q;
        free_workspace(c);
        return st;
    }
    if (c->kind == COFEM_OP_DENSE && !c->use_tc) {
        if ((st = dalloc(c, &c->T, w.t)) || (st = dalloc(c, &c->Tpart, w.tpart))) {
            c->Qcap = Q;
            free_workspace(c);
            return st;
        }
    }
    c->Qcap = Q;
    if (precise(c)) {
        const DfSizes z = df_configure(c, Q);
        c->df_QP = z.QP;
        c->df_S1 = z.S1;
        c->df_S2 = z.S2;
        c->df_k1 = z.k1;
        c->df_k2 = z.k2;
        if ((st = dalloc(c, &c->Xlo, w.xrp)) || (st = dalloc(c, &c->Rt, w.xrp)) ||
            (c->kind == COFEM_OP_DENSE && (st = dalloc(c, &c->df_T, z.T))) || (st = dalloc(c, &c->df_thi, z.t)) ||
            (st = dalloc(c, &c->df_tlo, z.t)) || (st = dalloc(c, &c->df_U, z.U))) {
            free_workspace(c);
            return st;
        }
        CK(cudaMemsetAsync(c->Xlo, 0, w.xrp * sizeof(float), c->stream));
        CK(cudaMemsetAsync(c->Rt, 0, w.xrp * sizeof(float), c->stream));
    }
    if (c->kind == COFEM_OP_DENSE && c->use_tc) {
        cudaError_t e = tc_setup(c, Q);
        if (e != cudaSuccess) {
            free_workspace(c);
            if (e == cudaErrorNotSupported)
                return fail(COFEM_ERR_UNSUPPORTED,
                            c->phi8 ? "the FP8 dense operator needs 3(K+1) <= 128"
                                    : "the single-pass dense operator needs BF16, 3(K+1) <= 112 and D <= 256 x SMs");
            return cuda_fail(e, "tensor-core operator set-up");
        }
    }
    if (precise(c)) {
        if (sl_applies(c, Q)) {
            cudaError_t e = sl_setup(c, Q);
            if (e != cudaSuccess) {
                free_workspace(c);
                return cuda_fail(e, "sliced accurate residual set-up");
            }
        } else if (c->opts.residual_path == COFEM_RESIDUAL_SLICED) {
            free_workspace(c);
            return fail(COFEM_ERR_UNSUPPORTED,
                        "the sliced accurate residual needs a BF16 or FP8 dense dictionary, K + 1 <= 48 and N, "
                        "D <= 40960");
        }
    }
    CK(cudaMemsetAsync(c->counters, 0, w.counters * sizeof(unsigned), c->stream));
    CK(cudaMemsetAsync(c->X, 0, w.xrp * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->R, 0, w.xrp * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->P, 0, w.xrp * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->U, 0, w.u * sizeof(float), c->stream));
    return COFEM_OK;
}

cofem_status ensure_iters(cofem_ctx* c, int T) {
    if (c->iters_cap >= T) return COFEM_OK;
    dfree(c, &c->iters_dev, (size_t)c->iters_cap);
    dfree(c, &c->res_dev, (size_t)c->iters_cap * COFEM_QMAX);
    c->iters_cap = 0;
    cofem_status st = dalloc(c, &c->iters_dev, (size_t)T);
    if (st || (st = dalloc(c, &c->res_dev, (size_t)T * COFEM_QMAX))) return st;
    c->iters_cap = T;
    return COFEM_OK;
}

// Record the whole fit (after the host-side prologue) into a graph.
cofem_status build_graph(cofem_ctx* c, int Q, bool pdl) {
    free_graph(c);
    CK(cudaGraphCreate(&c->graph, 0));
    Sink root;
    root.stream = c->stream;
    root.graph = c->graph;
    root.pdl = pdl;
    launch_fit_setup(root, c, Q);
    const cudaGraphConditionalHandle h_em = root.make_handle(1u, true);
    Sink em = root.conditional(h_em, cudaGraphCondTypeWhile);
    // precision form: the CG loop sits in a verification loop whose body ends
    // with the true-residual check (which may restart columns and go round
    // again).  The initialisation sets the verification loop's condition in
    // every EM iteration (a handle's default value is applied only when the
    // whole graph is launched); the gate kernel sets the CG loop's entry
    // condition, a handle of the verification body
    const bool verify = precise(c);
    // warm start: A X of the previous E-step's X for the initial residual (at
    // t = 1 the initialisation ignores it and starts from X = 0)
    if (c->opts.warm_start) launch_operator(em, c, Q, c->X, OP_PLAIN);
    Sink vf;
    cudaGraphConditionalHandle h_vf = 0, h_cg = 0;
    // two-pass tensor-core operator: the loop is rotated so that the first
    // product of the next CG step follows the direction kernel inside the
    // body (a programmatic edge: its prologue and first dictionary tiles
    // overlap the direction kernel); the first step's product runs before the
    // loop.  When the loop ends, the product of the step not taken is unused.
    const bool rot = tc_rotatable(c);
    // residual replacement (precision form): no conditional node inside the
    // CG loop, so that every step keeps its programmatic edges.  The loop
    // instead ends at a replacement step: its direction and next first
    // product are deferred (they do nothing at such a step), and after the
    // loop an IF node runs the replacement, the direction and the first
    // product; a "run" loop around both goes back into the CG loop.  Per run
    // a gate sets the CG loop's entry condition (and clears the replacement
    // condition), and a gate after the IF node the run loop's condition.  The
    // kernels of every step are those of the host-driven loop, in the same
    // order.  (Measured at 8192 x 32768, K = 32, 10 EM iterations: 1.2 %
    // less fit time than an IF node between the update and the direction at
    // every step.  Timeline stamps around a replacement: the loop exit, the
    // IF node, the gates and the re-entry take about 25 us in all.)
    const bool with_rr = c->opts.rr_period > 0;   // implies verify
    cudaGraphConditionalHandle h_run = 0;
    if (verify) {
        h_vf = em.make_handle(0u, false);
        launch_cg_init(em, c, Q, h_vf);
        vf = em.conditional(h_vf, cudaGraphCondTypeWhile);
        if (with_rr) {
            h_run = vf.make_handle(0u, false);
            launch_cg_gate(vf, c, h_run);
        } else {
            h_cg = vf.make_handle(0u, false);
            launch_cg_gate(vf, c, h_cg);
        }
        if (rot) launch_tc_first_product(vf, c);
    } else {
        h_cg = em.make_handle(0u, false);
        launch_cg_init(em, c, Q, h_cg);
        if (rot) launch_tc_first_product(em, c);
    }
    Sink& outer = verify ? vf : em;
    Sink run;
    cudaGraphConditionalHandle h_rr = 0;
    if (with_rr) {
        run = outer.conditional(h_run, cudaGraphCondTypeWhile);
        h_cg = run.make_handle(0u, false);
        h_rr = run.make_handle(0u, false);
        launch_cg_gate(run, c, h_cg, h_rr);
    }
    Sink cg = (with_rr ? run : outer).conditional(h_cg, cudaGraphCondTypeWhile);
    if (rot) launch_tc_rest(cg, c, Q, OP_CG);
    else launch_operator(cg, c, Q, c->P, OP_CG);
    launch_cg_update(cg, c, Q, h_rr, h_cg);
    launch_cg_direction(cg, c, Q, h_cg, with_rr);
    if (rot) launch_tc_first_product(cg, c, with_rr);
    Sink rr;
    if (with_rr) {
        rr = run.conditional(h_rr, cudaGraphCondTypeIf);
        launch_true_residual(rr, c, Q, DF_RR);
        launch_cg_direction(rr, c, Q, 0);
        if (rot) launch_tc_first_product(rr, c);
        launch_cg_gate(run, c, h_run);
    }
    if (verify) {
        launch_true_residual(vf, c, Q, DF_CHECK);
        launch_df_check(vf, c, Q, h_vf);
    }
    launch_mstep(em, c, Q, h_em);
    cudaError_t e = root.err ? root.err
                             : (em.err ? em.err
                                       : (vf.err ? vf.err : (run.err ? run.err : (cg.err ? cg.err : rr.err))));
    if (e != cudaSuccess) {
        free_graph(c);
        return cuda_fail(e, "recording the fit graph");
    }
    e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
    if (e != cudaSuccess) {
        free_graph(c);
        return cuda_fail(e, "cudaGraphInstantiate");
    }
    c->graph_Q = Q;
    c->graph_pdl = pdl;
    return COFEM_OK;
}

cofem_status read_ctl(cofem_ctx* c) {
    CK(cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

// The same sequence as the graph, driven from the host (one sync per CG iteration).
cofem_status run_fit_direct(cofem_ctx* c, int Q, int T) {
    Sink s;
    s.stream = c->stream;
    s.pdl = c->opts.overlap_launch != 0;
    launch_fit_setup(s, c, Q);
    const bool verify = precise(c);
    for (int t = 1; t <= T; ++t) {
        if (c->opts.warm_start) launch_operator(s, c, Q, c->X, OP_PLAIN);
        launch_cg_init(s, c, Q, 0);
        if (s.err) return cuda_fail(s.err, "launch");
        cofem_status st = read_ctl(c);
        if (st) return st;
        do {
            while (c->ctl_host->any_active && c->ctl_host->u < c->ctl_host->maxit) {
                launch_operator(s, c, Q, c->P, OP_CG);
                launch_cg_update(s, c, Q, 0, 0);
                if (s.err) return cuda_fail(s.err, "launch");
                if ((st = read_ctl(c))) return st;
                const int u = c->ctl_host->u;
                if (c->ctl_host->rr_period > 0 && u % c->ctl_host->rr_period == 0)
                    launch_true_residual(s, c, Q, DF_RR);
                launch_cg_direction(s, c, Q, 0);
                if (s.err) return cuda_fail(s.err, "launch");
                if ((st = read_ctl(c))) return st;
            }
            if (!verify) break;
            launch_true_residual(s, c, Q, DF_CHECK);
            launch_df_check(s, c, Q, 0);
            if (s.err) return cuda_fail(s.err, "launch");
            if ((st = read_ctl(c))) return st;
        } while (c->ctl_host->verify_again);
        launch_mstep(s, c, Q, 0);
        if (s.err) return cuda_fail(s.err, "launch");
    }
    return COFEM_OK;
}

cofem_status check_finite_dev(cofem_ctx* c, const float* x, long long n, const char* name) {
    unsigned* dbad = c->check_flag;
    CK(cudaMemsetAsync(dbad, 0, sizeof(unsigned), c->stream));
    launch_check_finite(c->stream, x, n, dbad);
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, dbad, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (h) return fail(COFEM_ERR_NONFINITE, "%s contains NaN or Inf", name);
    return COFEM_OK;
}

// Kernel attributes that are device-wide (dynamic shared-memory limits) are set
// once per device, before the first handle on it runs anything.
std::mutex g_attr_mu;
bool g_attr_done[64] = {};

cofem_status set_kernel_attributes(int dev) {
    if (dev < 0 || dev >= 64) return fail(COFEM_ERR_UNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (g_attr_done[dev]) return COFEM_OK;
    int optin = 0;
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CK(tc_kernel_attributes(optin));
    CK(toeplitz_kernel_attributes());
    CK(dct_kernel_attributes());
    CK(fftconv_kernel_attributes());
    CK(df_kernel_attributes());
    CK(sl_kernel_attributes(optin));
    g_attr_done[dev] = true;
    return COFEM_OK;
}

cofem_status check_device(int* dev, int* sms) {
    CK(cudaGetDevice(dev));
    int major = 0, minor = 0;
    CK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, *dev));
    CK(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, *dev));
    if (!(major == 10 && minor == 3))
        return fail(COFEM_ERR_UNSUPPORTED, "libcofem is built for sm_103a (GB300); device %d is sm_%d%d", *dev,
                    major, minor);
    CK(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, *dev));
    return set_kernel_attributes(*dev);
}

}  // namespace

// Lets other translation units record a failure message for cofem_last_error().
cofem_status cofem_set_error(cofem_status st, const char* msg) { return fail(st, "%s", msg); }

extern "C" {

void cofem_default_opts(cofem_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = COFEM_F32;
    o->precond = COFEM_PRECOND_JACOBI;
    o->conv = COFEM_CONV_PER_COLUMN;
    o->rr_period = 0;
    o->alpha_max = 1e12;
    o->seed = 2;
    o->stream = nullptr;
    o->use_graph = 1;
    o->overlap_launch = 1;
    o->check_residual = 0;
    o->warm_start = 0;
    o->toeplitz_path = COFEM_TOEPLITZ_AUTO;
}

const char* cofem_status_string(cofem_status s) {
    switch (s) {
        case COFEM_OK: return "ok";
        case COFEM_ERR_INVALID_ARG: return "invalid argument";
        case COFEM_ERR_NOMEM: return "out of device memory";
        case COFEM_ERR_CUDA: return "CUDA error";
        case COFEM_ERR_NONFINITE: return "non-finite value";
        case COFEM_ERR_UNSUPPORTED: return "unsupported";
        case COFEM_ERR_NOT_FOUND: return "not found";
        default: return "unknown status";
    }
}

const char* cofem_last_error(void) { return g_err; }

}  // extern "C"

// Handle creation for every dictionary kind: `data` is the dense matrix or the
// convolution filter (floats), or the DCT dictionary's row indices (ints).
static cofem_status create_impl(cofem_ctx** out, long long N, long long D, int kind, const void* data, long long L,
                                const cofem_opts* opts) {
    g_err[0] = 0;
    if (!out) return fail(COFEM_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (N < 1 || D < 1 || N > 0x7fffffffLL || D > 0x7fffffffLL) return fail(COFEM_ERR_INVALID_ARG, "bad N/D");
    if (!data) return fail(COFEM_ERR_INVALID_ARG, kind == COFEM_OP_DCT ? "rows is NULL" : "phi is NULL");
    const float* phi = (const float*)data;
    cofem_opts o;
    cofem_default_opts(&o);
    if (opts) o = *opts;
    if (kind == COFEM_OP_DENSE) {
        if (L != 0) return fail(COFEM_ERR_INVALID_ARG, "L must be 0 for a dense dictionary");
        if (o.max_sms < 0) return fail(COFEM_ERR_INVALID_ARG, "max_sms must be >= 0");
        if (o.dense_path < COFEM_PATH_AUTO || o.dense_path > COFEM_PATH_SINGLE_PASS)
            return fail(COFEM_ERR_INVALID_ARG, "dense_path must be AUTO, TWO_PASS or SINGLE_PASS");
        if (o.precision != COFEM_F32 && o.precision != COFEM_BF16 && o.precision != COFEM_F32_TF32X3 &&
            o.precision != COFEM_FP8_E4M3)
            return fail(COFEM_ERR_INVALID_ARG,
                        "precision must be COFEM_F32, COFEM_BF16, COFEM_F32_TF32X3 or COFEM_FP8_E4M3");
        // the 3xTF32 products hold the FP32 dictionary only to about 2^-22: CG
        // then iterates on another dictionary than the one the accurate
        // residual measures, a mismatch that the cancellation in Phi^T Phi x
        // lifts far above the CG tolerance, so replacement cannot converge
        if (o.precision == COFEM_F32_TF32X3 && o.rr_period > 0)
            return fail(COFEM_ERR_UNSUPPORTED, "residual replacement needs products exact on the stored dictionary "
                                               "(COFEM_F32, COFEM_BF16, COFEM_FP8_E4M3), not 3xTF32");
    } else if (kind == COFEM_OP_TOEPLITZ) {
        if (N != D) return fail(COFEM_ERR_INVALID_ARG, "a convolutional dictionary needs N == D");
        if (L < 1 || L > 1024 || L > N) return fail(COFEM_ERR_INVALID_ARG, "need 1 <= L <= min(1024, N)");
        if (o.precision != COFEM_F32) return fail(COFEM_ERR_INVALID_ARG, "convolutional dictionary is FP32 only");
        if (o.toeplitz_path < COFEM_TOEPLITZ_AUTO || o.toeplitz_path > COFEM_TOEPLITZ_FFT)
            return fail(COFEM_ERR_INVALID_ARG, "toeplitz_path must be AUTO, DIRECT or FFT");
    } else if (kind == COFEM_OP_DCT) {
        if (D < 16 || D > COFEM_DCT_MAX_D || (D & (D - 1)))
            return fail(COFEM_ERR_INVALID_ARG, "a DCT dictionary needs D a power of two, 16 <= D <= %d",
                        COFEM_DCT_MAX_D);
        if (N > D) return fail(COFEM_ERR_INVALID_ARG, "a DCT dictionary keeps N <= D rows");
        if (L != 0) return fail(COFEM_ERR_INVALID_ARG, "L must be 0 for a DCT dictionary");
        if (o.precision != COFEM_F32) return fail(COFEM_ERR_INVALID_ARG, "the DCT dictionary is FP32 only");
        if (o.rr_period != 0 || o.check_residual != 0)
            return fail(COFEM_ERR_UNSUPPORTED, "the precision form (rr_period, check_residual) is not built for "
                                               "the DCT dictionary");
    } else {
        return fail(COFEM_ERR_INVALID_ARG, "unknown dictionary kind %d", kind);
    }
    if (o.precond != COFEM_PRECOND_JACOBI && o.precond != COFEM_PRECOND_ONE && o.precond != COFEM_PRECOND_NONE)
        return fail(COFEM_ERR_INVALID_ARG, "bad precond");
    if (o.conv != COFEM_CONV_PER_COLUMN && o.conv != COFEM_CONV_FROBENIUS)
        return fail(COFEM_ERR_INVALID_ARG, "bad conv");
    if (o.rr_period < 0) return fail(COFEM_ERR_INVALID_ARG, "rr_period < 0");
    if (o.check_residual != 0 && o.check_residual != 1)
        return fail(COFEM_ERR_INVALID_ARG, "check_residual must be 0 or 1");
    if (o.warm_start != 0 && o.warm_start != 1) return fail(COFEM_ERR_INVALID_ARG, "warm_start must be 0 or 1");
    if (o.residual_path < COFEM_RESIDUAL_AUTO || o.residual_path > COFEM_RESIDUAL_SLICED)
        return fail(COFEM_ERR_INVALID_ARG, "residual_path must be AUTO, FP32_PAIRS or SLICED");
    if (o.overlap_launch != 0 && o.overlap_launch != 1) return fail(COFEM_ERR_INVALID_ARG, "overlap_launch must be 0 or 1");
    if (o.prior != COFEM_PRIOR_GAUSSIAN && o.prior != COFEM_PRIOR_RECTIFIED)
        return fail(COFEM_ERR_INVALID_ARG, "prior must be COFEM_PRIOR_GAUSSIAN or COFEM_PRIOR_RECTIFIED");
    if (!(o.alpha_max > 0.0) || !std::isfinite(o.alpha_max)) return fail(COFEM_ERR_INVALID_ARG, "bad alpha_max");

    int dev = 0, sms = 0;
    cofem_status st = check_device(&dev, &sms);
    if (st) return st;

    cofem_ctx* c = new cofem_ctx();
    c->N = N;
    c->D = D;
    c->kind = kind;
    c->L = (int)L;
    c->opts = o;
    c->device = dev;
    c->num_sms = (o.max_sms > 0 && o.max_sms < sms) ? o.max_sms : sms;
    c->Np = round_up(N, 128);
    c->Dp = round_up(D, 128);
    c->use_tc = kind == COFEM_OP_DENSE && o.precision != COFEM_F32;
    c->nch = vec_chunks(c->Dp);
    if (o.stream) {
        c->stream = (cudaStream_t)o.stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return cuda_fail(e, "cudaStreamCreate");
        }
        c->own_stream = true;
    }
    auto bail = [&](cofem_status s2) {
        cofem_destroy(c);
        return s2;
    };
#define CKB(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call)); \
    } while (0)

    if ((st = dalloc(c, &c->ctl, 1))) return bail(st);
    c->ctl_host = new DevCtl();
    memset(c->ctl_host, 0, sizeof(DevCtl));
    if ((st = dalloc(c, &c->theta, (size_t)c->Dp)) || (st = dalloc(c, &c->alpha, (size_t)c->Dp)) ||
        (st = dalloc(c, &c->minv, (size_t)c->Dp)) || (st = dalloc(c, &c->b, (size_t)c->Dp)) ||
        (st = dalloc(c, &c->mu_out, (size_t)c->Dp)) || (st = dalloc(c, &c->s_out, (size_t)c->Dp)) ||
        (st = dalloc(c, &c->yv, (size_t)c->Np)))
        return bail(st);
    CKB(cudaMemsetAsync(c->alpha, 0, c->Dp * sizeof(float), c->stream));
    CKB(cudaMemsetAsync(c->yv, 0, c->Np * sizeof(float), c->stream));
    // one device word for the finiteness checks of inputs (the fit workspace,
    // and the tensor-core plan with it, is made by the first call that needs it)
    if ((st = dalloc(c, &c->check_flag, 1))) return bail(st);

    if (kind == COFEM_OP_DENSE) {
        // upload into a padded FP32 copy (zero rows/columns beyond N, D)
        float* tmp = nullptr;
        if ((st = dalloc(c, &tmp, (size_t)c->Np * c->Dp))) return bail(st);
        CKB(cudaMemsetAsync(tmp, 0, (size_t)c->Np * c->Dp * sizeof(float), c->stream));
        CKB(cudaMemcpy2DAsync(tmp, c->Dp * sizeof(float), phi, D * sizeof(float), D * sizeof(float), N,
                              cudaMemcpyDefault, c->stream));
        if ((st = check_finite_dev(c, tmp, (long long)c->Np * c->Dp, "phi"))) {
            dfree(c, &tmp, (size_t)c->Np * c->Dp);
            return bail(st);
        }
        if (o.precision == COFEM_BF16) {
            if ((st = dalloc(c, &c->phi16, (size_t)c->Np * c->Dp))) {
                dfree(c, &tmp, (size_t)c->Np * c->Dp);
                return bail(st);
            }
            launch_quantize_bf16(c->stream, tmp, c->Np, c->Dp, c->Dp, c->phi16, c->Np, c->Dp);
            CKB(cudaStreamSynchronize(c->stream));
            dfree(c, &tmp, (size_t)c->Np * c->Dp);
        } else if (o.precision == COFEM_FP8_E4M3) {
            if ((st = dalloc(c, &c->phi8, (size_t)c->Np * c->Dp)) || (st = dalloc(c, &c->scale8, (size_t)c->Np))) {
                dfree(c, &tmp, (size_t)c->Np * c->Dp);
                return bail(st);
            }
            launch_quantize_fp8(c->stream, tmp, c->Dp, c->N, c->D, c->Np, c->Dp, c->phi8, c->scale8);
            CKB(cudaStreamSynchronize(c->stream));
            dfree(c, &tmp, (size_t)c->Np * c->Dp);
        } else {
            c->phi32 = tmp;
        }
        launch_dense_colreduce(c->stream, c, nullptr, 1.0, c->theta);
    } else if (kind == COFEM_OP_DCT) {
        // rows: N distinct indices in [0, D), checked on the host
        std::vector<int> rows((size_t)N);
        CKB(cudaMemcpy(rows.data(), data, (size_t)N * sizeof(int), cudaMemcpyDefault));
        std::vector<char> seen((size_t)D, 0);
        for (long long i = 0; i < N; ++i) {
            const int r = rows[(size_t)i];
            if (r < 0 || r >= D || seen[(size_t)r]) {
                cofem_destroy(c);
                return fail(COFEM_ERR_INVALID_ARG, "rows must be N distinct indices in [0, D)");
            }
            seen[(size_t)r] = 1;
        }
        if ((st = dalloc(c, &c->dct_rows, (size_t)N)) || (st = dalloc(c, &c->dct_mask, (size_t)c->Dp)) ||
            (st = dalloc(c, &c->dct_tw, (size_t)(D / 4 > 0 ? D / 4 : 1))))
            return bail(st);
        CKB(cudaMemcpyAsync(c->dct_rows, rows.data(), (size_t)N * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        launch_dct_setup(c->stream, c);
        CKB(cudaStreamSynchronize(c->stream));   // rows (host vector) is read by the copy
    } else {
        if ((st = dalloc(c, &c->h, (size_t)L))) return bail(st);
        CKB(cudaMemcpyAsync(c->h, phi, L * sizeof(float), cudaMemcpyDefault, c->stream));
        if ((st = check_finite_dev(c, c->h, L, "h"))) return bail(st);
        CKB(toeplitz_prepare(c->L));
        launch_toeplitz_theta(c->stream, c);
        // AUTO takes the direct form: on GB300 the tiled direct convolution
        // (420 us per application at D = 10^6, L = 256, Q = 17) beats the
        // shared-memory FFT form (890 us), whose radix-2 stages are bound by
        // shared-memory traffic and barriers, not by its O(log F) flops
        c->use_fftconv = o.toeplitz_path == COFEM_TOEPLITZ_FFT;
        if (c->use_fftconv) {
            if ((st = dalloc(c, &c->fc_H, (size_t)1 << COFEM_FFTCONV_LOGF)) ||
                (st = dalloc(c, &c->fc_tw, (size_t)1 << (COFEM_FFTCONV_LOGF - 1))))
                return bail(st);
            launch_fftconv_setup(c->stream, c);
        }
    }
    CKB(cudaGetLastError());
    if (o.precond == COFEM_PRECOND_ONE) {
        std::vector<float> ones((size_t)c->Dp, 0.0f);
        for (long long j = 0; j < D; ++j) ones[(size_t)j] = 1.0f;
        CKB(cudaMemcpyAsync(c->theta, ones.data(), c->Dp * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    }
    CKB(cudaStreamSynchronize(c->stream));
#undef CKB
    *out = c;
    return COFEM_OK;
}

extern "C" {

cofem_status cofem_create(cofem_ctx** out, long long N, long long D, int kind, const float* phi, long long L,
                          const cofem_opts* opts) {
    if (kind == COFEM_OP_DCT) {
        g_err[0] = 0;
        return fail(COFEM_ERR_INVALID_ARG, "a DCT dictionary is created with cofem_create_dct");
    }
    return create_impl(out, N, D, kind, phi, L, opts);
}

cofem_status cofem_create_dct(cofem_ctx** out, long long N, long long D, const int* rows, const cofem_opts* opts) {
    return create_impl(out, N, D, COFEM_OP_DCT, rows, 0, opts);
}

cofem_status cofem_destroy(cofem_ctx* c) {
    if (!c) return COFEM_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_workspace(c);
    free_graph(c);
    dfree(c, &c->phi32, (size_t)c->Np * c->Dp);
    dfree(c, &c->phi16, (size_t)c->Np * c->Dp);
    dfree(c, &c->phi8, (size_t)c->Np * c->Dp);
    dfree(c, &c->scale8, (size_t)c->Np);
    dfree(c, &c->h, (size_t)c->L);
    dfree(c, &c->fc_H, (size_t)1 << COFEM_FFTCONV_LOGF);
    dfree(c, &c->fc_tw, (size_t)1 << (COFEM_FFTCONV_LOGF - 1));
    dfree(c, &c->dct_rows, (size_t)c->N);
    dfree(c, &c->dct_mask, (size_t)c->Dp);
    dfree(c, &c->dct_tw, (size_t)(c->D / 4 > 0 ? c->D / 4 : 1));
    dfree(c, &c->theta, (size_t)c->Dp);
    dfree(c, &c->alpha, (size_t)c->Dp);
    dfree(c, &c->minv, (size_t)c->Dp);
    dfree(c, &c->b, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->mu_out, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->s_out, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->yv, (size_t)c->Lcap * c->Np);
    dfree(c, &c->iters_dev, (size_t)c->iters_cap);
    dfree(c, &c->res_dev, (size_t)c->iters_cap * COFEM_QMAX);
    dfree(c, &c->check_flag, 1);
    dfree(c, &c->ctl, 1);
    delete c->ctl_host;
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return COFEM_OK;
}

// Per-task buffers (b, y, mu, s) for L tasks; growing them drops the fit
// graph, which holds their addresses.
static cofem_status ensure_tasks(cofem_ctx* c, int L) {
    if (L <= c->Lcap) return COFEM_OK;
    dfree(c, &c->b, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->mu_out, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->s_out, (size_t)c->Lcap * c->Dp);
    dfree(c, &c->yv, (size_t)c->Lcap * c->Np);
    free_graph(c);
    c->Lcap = 0;
    cofem_status st;
    if ((st = dalloc(c, &c->b, (size_t)L * c->Dp)) || (st = dalloc(c, &c->mu_out, (size_t)L * c->Dp)) ||
        (st = dalloc(c, &c->s_out, (size_t)L * c->Dp)) || (st = dalloc(c, &c->yv, (size_t)L * c->Np)))
        return st;
    CK(cudaMemsetAsync(c->yv, 0, (size_t)L * c->Np * sizeof(float), c->stream));
    c->Lcap = L;
    return COFEM_OK;
}

// b_l = beta Phi^T y_l into row l of c->b, after y_l (row l of Y, N floats
// each) is staged in row l of c->yv.
static cofem_status stage_y_and_b(cofem_ctx* c, const float* Y, double beta, int L = 1) {
    CK(cudaMemcpy2DAsync(c->yv, c->Np * sizeof(float), Y, c->N * sizeof(float), c->N * sizeof(float), L,
                         cudaMemcpyDefault, c->stream));
    for (int l = 0; l < L; ++l) {
        cofem_status st = check_finite_dev(c, c->yv + (size_t)l * c->Np, c->N, "y");
        if (st) return st;
        float* yl = c->yv + (size_t)l * c->Np;
        float* bl = c->b + (size_t)l * c->Dp;
        if (c->kind == COFEM_OP_DENSE) launch_dense_colreduce(c->stream, c, yl, beta, bl);
        else if (c->kind == COFEM_OP_DCT) launch_dct_phit_y(c->stream, c, yl, beta, bl, c->s_out + (size_t)l * c->Dp);
        else launch_toeplitz_phit_y(c->stream, c, yl, beta, bl);
    }
    CK(cudaGetLastError());
    return COFEM_OK;
}

// Arguments, workspace, control block, b = beta Phi^T y and alpha^(1) of a
// fit of L tasks (everything before the E-steps).
static cofem_status fit_begin(cofem_ctx* c, int L, const float* Y, double beta, const float* alpha0, int K,
                              int T_em, double cg_tol, int cg_maxit, float* mu, float* s, float* alpha) {
    if (!c) return fail(COFEM_ERR_INVALID_ARG, "handle is NULL");
    if (!Y || !mu || !s || !alpha) return fail(COFEM_ERR_INVALID_ARG, "y, mu, s and alpha are required");
    if (L < 1) return fail(COFEM_ERR_INVALID_ARG, "need L >= 1");
    if (K < 1 || L * (K + 1) > COFEM_QMAX)
        return fail(COFEM_ERR_INVALID_ARG, L == 1 ? "need 1 <= K <= %d" : "need K >= 1 and L (K + 1) <= %d",
                    L == 1 ? COFEM_QMAX - 1 : COFEM_QMAX);
    if (T_em < 1) return fail(COFEM_ERR_INVALID_ARG, "need T_em >= 1");
    if (cg_maxit < 1) return fail(COFEM_ERR_INVALID_ARG, "need cg_maxit >= 1");
    if (!(cg_tol > 0.0) || !std::isfinite(cg_tol)) return fail(COFEM_ERR_INVALID_ARG, "need cg_tol > 0");
    if (!std::isfinite(beta)) return fail(COFEM_ERR_NONFINITE, "beta is not finite");
    if (!(beta > 0.0)) return fail(COFEM_ERR_INVALID_ARG, "need beta > 0");
    if (L > 1 && c->opts.prior != COFEM_PRIOR_GAUSSIAN)
        return fail(COFEM_ERR_UNSUPPORTED, "the multi-task M-step is defined for the Gaussian prior only");
    CK(cudaSetDevice(c->device));
    const int Q = L * (K + 1);
    cofem_status st;
    if ((st = ensure_workspace(c, Q)) || (st = ensure_iters(c, T_em)) || (st = ensure_tasks(c, L))) return st;

    DevCtl* hc = c->ctl_host;
    memset(hc, 0, sizeof(DevCtl));
    hc->beta = beta;
    hc->tol = cg_tol;
    hc->alpha_max = c->opts.alpha_max;
    hc->seed = c->opts.seed;
    hc->T = T_em;
    hc->K = K;
    hc->L = L;
    hc->Q = Q;
    hc->maxit = cg_maxit;
    hc->conv = c->opts.conv;
    hc->rr_period = c->opts.rr_period;
    hc->prior = c->opts.prior;
    hc->fix_residual = c->opts.rr_period > 0;
    hc->precond_none = c->opts.precond == COFEM_PRECOND_NONE;
    hc->warm = c->opts.warm_start;
    hc->ap_part = c->part + (size_t)2 * Q * c->nch;   // slab 2 of the CG partials
    hc->ap_n = c->nch;
    CK(cudaMemcpyAsync(c->ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, c->stream));
    // true residuals not measured stay NaN (all bits set)
    CK(cudaMemsetAsync(c->res_dev, 0xFF, (size_t)T_em * COFEM_QMAX * sizeof(double), c->stream));
    c->last_T = T_em;
    c->last_Q = Q;
    if ((st = stage_y_and_b(c, Y, beta, L))) return st;
    if (alpha0) {
        CK(cudaMemcpyAsync(c->alpha, alpha0, c->D * sizeof(float), cudaMemcpyDefault, c->stream));
        if ((st = check_finite_dev(c, c->alpha, c->D, "alpha0"))) return st;
    } else {
        std::vector<float> ones((size_t)c->D, 1.0f);
        CK(cudaMemcpyAsync(c->alpha, ones.data(), c->D * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return COFEM_OK;
}

// Results of the last E-step (mu, s of each task, alpha^(T), cg_iters) and the flags.
static cofem_status fit_finish(cofem_ctx* c, int L, int T_em, float* mu, float* s, float* alpha, int* cg_iters,
                               unsigned* flags) {
    DevCtl* hc = c->ctl_host;
    CK(cudaMemcpy2DAsync(mu, c->D * sizeof(float), c->mu_out, c->Dp * sizeof(float), c->D * sizeof(float), L,
                         cudaMemcpyDefault, c->stream));
    CK(cudaMemcpy2DAsync(s, c->D * sizeof(float), c->s_out, c->Dp * sizeof(float), c->D * sizeof(float), L,
                         cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(alpha, c->alpha, c->D * sizeof(float), cudaMemcpyDefault, c->stream));
    if (cg_iters) CK(cudaMemcpyAsync(cg_iters, c->iters_dev, T_em * sizeof(int), cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(hc, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    if (flags) *flags = hc->flags;
    c->last_rr = hc->n_rr;
    c->last_check = hc->n_check;
    if (hc->flags & COFEM_FLAG_DEVICE_TIMEOUT)
        return fail(COFEM_ERR_CUDA, "a bounded on-device wait timed out (tensor-core pipeline)");
    return COFEM_OK;
}

// One fit of L tasks sharing the dictionary and alpha (L = 1: Alg. 1 as
// printed; L > 1: the multi-task CoFEM of Sec. III with the L (K+1) columns
// in one batched PCG).
static cofem_status fit_impl(cofem_ctx* c, int L, const float* Y, double beta, const float* alpha0, int K,
                             int T_em, double cg_tol, int cg_maxit, float* mu, float* s, float* alpha,
                             int* cg_iters, unsigned* flags) {
    g_err[0] = 0;
    cofem_status st = fit_begin(c, L, Y, beta, alpha0, K, T_em, cg_tol, cg_maxit, mu, s, alpha);
    if (st) return st;
    const int Q = L * (K + 1);
    if (c->opts.use_graph) {
        if (c->graph_Q != Q || c->graph_L != L || !c->gexec) {
            // programmatic edges where the driver takes them, else plain ones
            const bool pdl = c->opts.overlap_launch != 0;
            if (!pdl || build_graph(c, Q, true) != COFEM_OK) {
                (void)cudaGetLastError();
                if ((st = build_graph(c, Q, false))) return st;
            }
            c->graph_L = L;
        }
        CK(cudaGraphLaunch(c->gexec, c->stream));
    } else {
        if ((st = run_fit_direct(c, Q, T_em))) return st;
    }
    return fit_finish(c, L, T_em, mu, s, alpha, cg_iters, flags);
}

}  // extern "C"

// Packed serving: the fit's prologue, the fixed segments of its products and
// the first E-step's initialisation on the handle's stream; the packed steps
// take it from there (phase PH_CG, or PH_START if no column needs CG).
cofem_status packed_prepare(cofem_ctx* c, const cofem_request& r) {
    g_err[0] = 0;
    if (c->kind != COFEM_OP_DENSE || !c->use_tc || c->phi8)
        return fail(COFEM_ERR_UNSUPPORTED, "packed serving takes dense BF16 or 3xTF32 dictionaries");
    cofem_status st = fit_begin(c, 1, r.y, r.beta, r.alpha0, r.K, r.T_em, r.cg_tol, r.cg_maxit, r.mu, r.s, r.alpha);
    if (st) return st;
    cudaError_t e = tc_pack_setup(c);
    if (e == cudaErrorNotSupported)
        return fail(COFEM_ERR_UNSUPPORTED, "packed serving needs the two-pass tensor-core operator");
    if (e != cudaSuccess) return cuda_fail(e, "packed segments");
    Sink s;
    s.stream = c->stream;
    launch_fit_setup(s, c, r.K + 1);
    launch_cg_init(s, c, r.K + 1, 0);
    if (s.err) return cuda_fail(s.err, "launch");
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status packed_finish(cofem_ctx* c, const cofem_request& r, unsigned* flags) {
    return fit_finish(c, 1, r.T_em, r.mu, r.s, r.alpha, r.cg_iters, flags);
}

extern "C" {

cofem_status cofem_fit(cofem_ctx* c, const float* y, double beta, const float* alpha0, int K, int T_em,
                       double cg_tol, int cg_maxit, float* mu, float* s, float* alpha, int* cg_iters,
                       unsigned* flags) {
    return fit_impl(c, 1, y, beta, alpha0, K, T_em, cg_tol, cg_maxit, mu, s, alpha, cg_iters, flags);
}

cofem_status cofem_fit_multitask(cofem_ctx* c, int L, const float* Y, double beta, const float* alpha0, int K,
                                 int T_em, double cg_tol, int cg_maxit, float* mu, float* s, float* alpha,
                                 int* cg_iters, unsigned* flags) {
    return fit_impl(c, L, Y, beta, alpha0, K, T_em, cg_tol, cg_maxit, mu, s, alpha, cg_iters, flags);
}

cofem_status cofem_probe_fill(unsigned long long seed, int t, int K, long long D, float* out, void* stream) {
    g_err[0] = 0;
    if (!out || K < 1 || D < 1 || t < 0) return fail(COFEM_ERR_INVALID_ARG, "bad arguments");
    if (K > 65535) return fail(COFEM_ERR_INVALID_ARG, "K too large");
    cudaStream_t st = (cudaStream_t)stream;
    launch_probe_fill(st, seed, t, K, D, D, out);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(st));
    return COFEM_OK;
}

cofem_status cofem_apply_operator(cofem_ctx* c, const float* V, int Q, const float* alpha, double beta,
                                  float* Psi, double* pi) {
    g_err[0] = 0;
    if (!c || !V || !alpha || !Psi) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (Q < 1 || Q > COFEM_QMAX) return fail(COFEM_ERR_INVALID_ARG, "need 1 <= Q <= %d", COFEM_QMAX);
    if (!std::isfinite(beta)) return fail(COFEM_ERR_NONFINITE, "beta is not finite");
    CK(cudaSetDevice(c->device));
    float* out = Psi;
    int out_kind = 0;   // 0 host, 1 device memory of this handle's device (or managed), 2 another device's
    {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, Psi) != cudaSuccess) {
            cudaGetLastError();
        } else if (a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == c->device)) {
            out_kind = 1;
        } else if (a.type == cudaMemoryTypeDevice) {
            out_kind = 2;
        }
    }
    if (out_kind == 2)
        return fail(COFEM_ERR_INVALID_ARG, "Psi is device memory of another device than the handle's (%d)", c->device);
    cofem_status st = ensure_workspace(c, Q);
    if (st) return st;
    // stage V (Q x D, stride D) into the padded P block and alpha into c->alpha
    CK(cudaMemsetAsync(c->P, 0, (size_t)Q * c->Dp * sizeof(float), c->stream));
    CK(cudaMemcpy2DAsync(c->P, c->Dp * sizeof(float), V, c->D * sizeof(float), c->D * sizeof(float), Q,
                         cudaMemcpyDefault, c->stream));
    CK(cudaMemcpyAsync(c->alpha, alpha, c->D * sizeof(float), cudaMemcpyDefault, c->stream));
    DevCtl* hc = c->ctl_host;
    memset(hc, 0, sizeof(DevCtl));
    hc->beta = beta;
    hc->Q = Q;
    CK(cudaMemcpyAsync(c->ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, c->stream));
    Sink s;
    s.stream = c->stream;
    launch_operator(s, c, Q, c->P, OP_PLAIN);
    if (s.err) return cuda_fail(s.err, "operator launch");
    const bool dev_out = out_kind == 1;
    if (!dev_out) out = c->X;   // stage in the X block (Q x D fits in Q x Dp)
    launch_plain_psi(c->stream, c, Q, c->P, c->alpha, beta, out);
    CK(cudaGetLastError());
    if (pi) {
        double* dpi = c->part;   // Q doubles of scratch
        launch_dot_rows(c->stream, c->P, c->Dp, out, c->D, c->D, Q, dpi);
        CK(cudaMemcpyAsync(pi, dpi, Q * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    if (!dev_out) CK(cudaMemcpyAsync(Psi, out, (size_t)Q * c->D * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status cofem_get_theta(cofem_ctx* c, float* theta) {
    g_err[0] = 0;
    if (!c || !theta) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpyAsync(theta, c->theta, c->D * sizeof(float), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status cofem_phit_y(cofem_ctx* c, const float* y, double beta, float* b) {
    g_err[0] = 0;
    if (!c || !y || !b) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (!std::isfinite(beta)) return fail(COFEM_ERR_NONFINITE, "beta is not finite");
    CK(cudaSetDevice(c->device));
    cofem_status st = stage_y_and_b(c, y, beta);
    if (st) return st;
    CK(cudaMemcpyAsync(b, c->b, c->D * sizeof(float), cudaMemcpyDefault, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status cofem_time_operator(cofem_ctx* c, int Q, int reps, double* ms_per_apply) {
    g_err[0] = 0;
    if (!c || !ms_per_apply || reps < 1) return fail(COFEM_ERR_INVALID_ARG, "bad arguments");
    if (Q != c->Qcap) return fail(COFEM_ERR_INVALID_ARG, "Q must match the last fit (%d)", c->Qcap);
    CK(cudaSetDevice(c->device));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    Sink s;
    s.stream = c->stream;
    launch_operator(s, c, Q, c->P, OP_TIME);   // warm-up
    CK(cudaEventRecord(e0, c->stream));
    for (int r = 0; r < reps; ++r) launch_operator(s, c, Q, c->P, OP_TIME);
    CK(cudaEventRecord(e1, c->stream));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s.err) return cuda_fail(s.err, "operator launch");
    *ms_per_apply = (double)ms / reps;
    return COFEM_OK;
}

cofem_status cofem_time_true_residual(cofem_ctx* c, int Q, int reps, double* ms_residual, double* ms_first) {
    g_err[0] = 0;
    if (!c || reps < 1 || (!ms_residual && !ms_first)) return fail(COFEM_ERR_INVALID_ARG, "bad arguments");
    if (!precise(c)) return fail(COFEM_ERR_INVALID_ARG, "the handle has neither rr_period > 0 nor check_residual = 1");
    if (Q != c->Qcap || c->last_T == 0) return fail(COFEM_ERR_INVALID_ARG, "Q must match the last fit (%d)", c->Qcap);
    CK(cudaSetDevice(c->device));
    cudaEvent_t e[4];
    for (auto& x : e) CK(cudaEventCreate(&x));
    Sink s;
    s.stream = c->stream;
    launch_true_residual(s, c, Q, DF_CHECK);   // warm-up
    CK(cudaEventRecord(e[0], c->stream));
    for (int r = 0; r < reps; ++r) launch_true_residual(s, c, Q, DF_CHECK);
    CK(cudaEventRecord(e[1], c->stream));
    if (c->kind == COFEM_OP_DENSE) {
        CK(cudaEventRecord(e[2], c->stream));
        for (int r = 0; r < reps; ++r) launch_df_first_product(s, c, Q);
        CK(cudaEventRecord(e[3], c->stream));
    }
    CK(cudaEventSynchronize(c->kind == COFEM_OP_DENSE ? e[3] : e[1]));
    float a = 0.0f, b = 0.0f;
    CK(cudaEventElapsedTime(&a, e[0], e[1]));
    if (c->kind == COFEM_OP_DENSE) CK(cudaEventElapsedTime(&b, e[2], e[3]));
    for (auto& x : e) cudaEventDestroy(x);
    if (s.err) return cuda_fail(s.err, "accurate residual launch");
    if (ms_residual) *ms_residual = (double)a / reps;
    if (ms_first) *ms_first = c->kind == COFEM_OP_DENSE ? (double)b / reps : 0.0;
    return COFEM_OK;
}

cofem_status cofem_accurate_product(cofem_ctx* c, const float* Xh, const float* Xl, int Q, double* out) {
    g_err[0] = 0;
    if (!c || !Xh || !Xl || !out) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (Q < 1 || Q > COFEM_QMAX) return fail(COFEM_ERR_INVALID_ARG, "need 1 <= Q <= %d", COFEM_QMAX);
    if (c->kind != COFEM_OP_DENSE) return fail(COFEM_ERR_INVALID_ARG, "the accurate product is built for dense dictionaries");
    if (!precise(c)) return fail(COFEM_ERR_INVALID_ARG, "the handle has neither rr_period > 0 nor check_residual = 1");
    CK(cudaSetDevice(c->device));
    for (const void* ptr : {(const void*)Xh, (const void*)Xl, (const void*)out}) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
            cudaGetLastError();
        } else if (a.type == cudaMemoryTypeDevice && a.device != c->device) {
            return fail(COFEM_ERR_INVALID_ARG, "device memory of another device than the handle's (%d)", c->device);
        }
    }
    cofem_status st = ensure_workspace(c, Q);
    if (st) return st;
    // the pair into the padded X, Xlo blocks (padding stays zero)
    CK(cudaMemsetAsync(c->X, 0, (size_t)Q * c->Dp * sizeof(float), c->stream));
    CK(cudaMemsetAsync(c->Xlo, 0, (size_t)Q * c->Dp * sizeof(float), c->stream));
    CK(cudaMemcpy2DAsync(c->X, c->Dp * sizeof(float), Xh, c->D * sizeof(float), c->D * sizeof(float), Q,
                         cudaMemcpyDefault, c->stream));
    CK(cudaMemcpy2DAsync(c->Xlo, c->Dp * sizeof(float), Xl, c->D * sizeof(float), c->D * sizeof(float), Q,
                         cudaMemcpyDefault, c->stream));
    if ((st = check_finite_dev(c, c->X, (long long)Q * c->Dp, "Xh"))) return st;
    if ((st = check_finite_dev(c, c->Xlo, (long long)Q * c->Dp, "Xl"))) return st;
    double* dout = nullptr;
    if ((st = dalloc(c, &dout, (size_t)Q * c->D))) return st;
    DevCtl* hc = c->ctl_host;
    memset(hc, 0, sizeof(DevCtl));
    hc->Q = Q;
    CK(cudaMemcpyAsync(c->ctl, hc, sizeof(DevCtl), cudaMemcpyHostToDevice, c->stream));
    Sink s;
    s.stream = c->stream;
    launch_df_gram(s, c, Q, dout);
    cudaError_t e = s.err;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, dout, (size_t)Q * c->D * sizeof(double), cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, &dout, (size_t)Q * c->D);
    if (e != cudaSuccess) return cuda_fail(e, "accurate product");
    if (hc->flags & COFEM_FLAG_DEVICE_TIMEOUT)
        return fail(COFEM_ERR_CUDA, "a bounded on-device wait timed out (tensor-core pipeline)");
    return COFEM_OK;
}

long long cofem_device_bytes(cofem_ctx* c) { return c ? c->bytes : 0; }

cofem_status cofem_get_dictionary(cofem_ctx* c, float* out) {
    g_err[0] = 0;
    if (!c || !out) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (c->kind != COFEM_OP_DENSE) return fail(COFEM_ERR_INVALID_ARG, "the handle holds a convolution filter");
    CK(cudaSetDevice(c->device));
    if (c->phi32) {
        CK(cudaMemcpy2DAsync(out, c->D * sizeof(float), c->phi32, c->Dp * sizeof(float), c->D * sizeof(float), c->N,
                             cudaMemcpyDefault, c->stream));
    } else {
        float* tmp = nullptr;
        cofem_status st = dalloc(c, &tmp, (size_t)c->N * c->D);
        if (st) return st;
        if (c->phi8) launch_dequant_fp8(c->stream, c->phi8, c->scale8, c->N, c->D, c->Dp, tmp);
        else launch_bf16_to_f32(c->stream, c->phi16, c->N, c->D, c->Dp, tmp);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out, tmp, (size_t)c->N * c->D * sizeof(float), cudaMemcpyDefault, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dfree(c, &tmp, (size_t)c->N * c->D);
        if (e != cudaSuccess) return cuda_fail(e, "reading the dictionary");
    }
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status cofem_operator_info(cofem_ctx* c, int* path, int* kernels_cg, int* kernels_rr, int* kernels_step) {
    g_err[0] = 0;
    if (!c) return fail(COFEM_ERR_INVALID_ARG, "handle is NULL");
    if (c->Qcap == 0) return fail(COFEM_ERR_INVALID_ARG, "no fit or application yet");
    int pth = COFEM_PATH_AUTO, kc = 1, kr = 1;
    if (c->kind == COFEM_OP_DENSE && c->use_tc) {
        tc_operator_info(c, &pth, &kc, &kr);
    } else if (c->kind == COFEM_OP_DENSE) {
        kc = 2;   // k_gemm1_simt, k_gemm2_simt
        kr = true_residual_kernels(c);
    } else {
        if (c->kind == COFEM_OP_TOEPLITZ) pth = c->use_fftconv ? COFEM_TOEPLITZ_FFT : COFEM_TOEPLITZ_DIRECT;
        kr = true_residual_kernels(c);
    }
    if (path) *path = pth;
    if (kernels_cg) *kernels_cg = kc;
    if (kernels_rr) *kernels_rr = kr;
    if (kernels_step) *kernels_step = 2;   // k_cg_update, k_cg_direction
    return COFEM_OK;
}

cofem_status cofem_true_residuals(cofem_ctx* c, double* out) {
    g_err[0] = 0;
    if (!c || !out) return fail(COFEM_ERR_INVALID_ARG, "NULL argument");
    if (c->last_T == 0) return fail(COFEM_ERR_INVALID_ARG, "no fit yet");
    if (!precise(c)) return fail(COFEM_ERR_INVALID_ARG, "the handle has neither rr_period > 0 nor check_residual = 1");
    CK(cudaSetDevice(c->device));
    CK(cudaMemcpy2DAsync(out, c->last_Q * sizeof(double), c->res_dev, COFEM_QMAX * sizeof(double),
                         c->last_Q * sizeof(double), c->last_T, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return COFEM_OK;
}

cofem_status cofem_fit_stats(cofem_ctx* c, int* replacements, int* checks) {
    g_err[0] = 0;
    if (!c) return fail(COFEM_ERR_INVALID_ARG, "handle is NULL");
    if (c->last_T == 0) return fail(COFEM_ERR_INVALID_ARG, "no fit yet");
    if (replacements) *replacements = c->last_rr;
    if (checks) *checks = c->last_check;
    return COFEM_OK;
}

cofem_status cofem_graph_info(cofem_ctx* c, int* built, int* overlapped) {
    g_err[0] = 0;
    if (!c) return fail(COFEM_ERR_INVALID_ARG, "handle is NULL");
    if (built) *built = c->gexec ? 1 : 0;
    if (overlapped) *overlapped = c->gexec && c->graph_pdl ? 1 : 0;
    return COFEM_OK;
}

}  // extern "C"
