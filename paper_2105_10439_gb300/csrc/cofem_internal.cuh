// Internal declarations shared by the libcofem translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/cofem.h"

#define COFEM_QMAX 64          // K <= 63
#define COFEM_VEC_CHUNK 1024   // elements of one column handled by a vector-kernel block
#define COFEM_VEC_THREADS 256

// ---------------------------------------------------------------------------
// Device-resident control block: fit parameters plus the per-column CG scalars
// of Alg. 2 (rho, pi, gamma, eta) and the loop counters.  Kept on the device so
// the EM and CG loops run without host round trips.
// ---------------------------------------------------------------------------
struct DevCtl {
    double beta, tol, alpha_max;
    unsigned long long seed;
    int T, K, Q, maxit, conv, rr_period;
    int t;            // current EM iteration, 1-based
    int u;            // CG iterations done in EM iteration t
    int any_active;   // some column still iterating
    unsigned flags;   // COFEM_FLAG_* bits
    int active[COFEM_QMAX];
    double rho[COFEM_QMAX];     // r^T M^-1 r
    double pi[COFEM_QMAX];      // p^T A p
    double gamma[COFEM_QMAX];   // rho / pi
    double eta[COFEM_QMAX];     // rho_new / rho_old
    double bnorm2[COFEM_QMAX];  // ||b_q||^2
    double rnorm2[COFEM_QMAX];  // ||r_q||^2
    double ap[COFEM_QMAX];      // p^T diag(alpha) p
    double tt[COFEM_QMAX];      // ||Phi p||^2
};

// Modes of the operator kernels.
enum OpMode { OP_CG = 0, OP_RR = 1, OP_PLAIN = 2 };

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the probe rule:
// key (seed, 0), counter (j >> 8, k, t, 0), bit j & 255 of the 256-bit block,
// p = +1 for bit 0, -1 for bit 1.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
    const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
        const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
        const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// The 64-bit word of the probe block that holds bits for j .. (j | 63).
__device__ __forceinline__ uint64_t probe_word(unsigned long long seed, int t, int k, long long j) {
    uint64_t c[4] = {(uint64_t)(j >> 8), (uint64_t)k, (uint64_t)t, 0ull};
    philox4x64_10(c, seed, 0ull);
    const int w = (int)((j & 255) >> 6);
    return w == 0 ? c[0] : (w == 1 ? c[1] : (w == 2 ? c[2] : c[3]));
}

__device__ __forceinline__ float probe_sign_from_word(uint64_t word, long long j) {
    return ((word >> (j & 63)) & 1ull) ? -1.0f : 1.0f;
}

// ---------------------------------------------------------------------------
// Reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; every thread gets the result.  `sh` needs blockDim/32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < nw; ++i) r += sh[i];   // fixed order: deterministic
    return r;
}

// "Last block done" arrival (threadfence reduction pattern, no spinning):
// every thread fences its own partial writes, thread 0 counts arrivals, the
// block that arrives last gets true and resets the counter for the next launch.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, unsigned total) {
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == total - 1);
        if (s_last) *counter = 0u;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// ---------------------------------------------------------------------------
// Launch sink: the same launch sequence either runs directly on a stream or is
// recorded as kernel nodes of a CUDA graph (linear chain), with conditional
// WHILE / IF bodies for the device-side loops.
// ---------------------------------------------------------------------------
struct Sink {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;   // null -> direct launches
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;

    bool recording() const { return graph != nullptr; }

    template <typename... P, typename... A>
    void launch(void (*f)(P...), dim3 grid, dim3 block, size_t smem, A... args) {
        if (err != cudaSuccess) return;
        if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
        // convert to the exact parameter types, then take addresses
        launch_typed<P...>(f, grid, block, smem, static_cast<P>(args)...);
    }

    template <typename... P>
    void launch_typed(void (*f)(P...), dim3 grid, dim3 block, size_t smem, P... args) {
        void* ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1] = {(void*)&args...};
        if (!graph) {
            err = cudaLaunchKernel((const void*)f, grid, block, ptrs, smem, stream);
            return;
        }
        cudaKernelNodeParams p = {};
        p.func = (void*)f;
        p.gridDim = grid;
        p.blockDim = block;
        p.sharedMemBytes = (unsigned)smem;
        p.kernelParams = ptrs;
        p.extra = nullptr;
        cudaGraphNode_t n;
        err = cudaGraphAddKernelNode(&n, graph, last ? &last : nullptr, last ? 1 : 0, &p);
        if (err == cudaSuccess) last = n;
    }

    // Conditional handle owned by this sink's graph (0 in direct mode).
    cudaGraphConditionalHandle make_handle(unsigned default_value, bool assign_default) {
        cudaGraphConditionalHandle h = 0;
        if (err != cudaSuccess || !graph) return 0;
        err = cudaGraphConditionalHandleCreate(&h, graph, default_value,
                                               assign_default ? cudaGraphCondAssignDefault : 0);
        return h;
    }

    // Append a conditional node (WHILE or IF) and return a sink recording its body.
    Sink conditional(cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type) {
        Sink body;
        body.stream = stream;
        if (err != cudaSuccess || !graph) { body.err = err ? err : cudaErrorInvalidValue; return body; }
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = type;
        np.conditional.size = 1;
        cudaGraphNode_t n;
        err = cudaGraphAddNode(&n, graph, last ? &last : nullptr, nullptr, last ? 1 : 0, &np);
        if (err != cudaSuccess) { body.err = err; return body; }
        last = n;
        body.graph = np.conditional.phGraph_out[0];
        return body;
    }
};

// Sets a graph conditional from one device thread (no-op for a zero handle,
// used in the direct-launch mode).
__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int v) {
    if (h) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
struct cofem_ctx {
    long long N = 0, D = 0;     // problem sizes
    long long Np = 0, Dp = 0;   // padded: Np multiple of 128, Dp multiple of 128
    int kind = COFEM_OP_DENSE;
    int L = 0;
    cofem_opts opts{};
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;

    // operator storage
    float* phi32 = nullptr;          // dense FP32, Np x Dp row-major, zero padded
    __nv_bfloat16* phi16 = nullptr;  // dense BF16, Np x Dp row-major, zero padded
    __nv_bfloat16* phiT16 = nullptr; // its transpose, Dp x Np row-major (tensor-core GEMM2 operand)
    void* tc = nullptr;              // tensor-core operator plan (kernels_tc.cu)
    float* h = nullptr;              // Toeplitz filter, L floats
    float* theta = nullptr;          // Dp

    // fit workspace (sized for Qcap columns)
    int Qcap = 0;
    int QP = 0;                      // padded column count of the dense intermediate T
    float *X = nullptr, *R = nullptr, *P = nullptr;   // Qcap x Dp each
    float *U = nullptr;              // operator output partials, S2 x Qcap x Dp
    float *alpha = nullptr, *minv = nullptr, *b = nullptr, *yv = nullptr;   // Dp (yv: Np)
    float *mu_out = nullptr, *s_out = nullptr;        // Dp
    float *T = nullptr;              // dense: Np x QP
    float *Tpart = nullptr;          // dense: S1 x Np x QP
    double* part = nullptr;          // vector-kernel partials: 3 x Qcap x nch
    double* tt_part = nullptr;       // operator partials of ||Phi p||^2
    unsigned* counters = nullptr;    // last-block counters
    int* iters_dev = nullptr;        // T_em
    int iters_cap = 0;
    DevCtl* ctl = nullptr;
    DevCtl* ctl_host = nullptr;      // pinned mirror
    int S1 = 1, S2 = 1;              // dense split factors
    long long chunk1 = 0, rchunk2 = 0;
    int nch = 0;                     // vector chunks per column

    // graph cache
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_Q = -1;

    long long bytes = 0;
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
// kernels_vec.cu
void launch_fit_setup(Sink& s, cofem_ctx* c, int Q);                 // alpha -> minv, ctl t = 1
void launch_cg_init(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg);
void launch_cg_update(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_rr);
void launch_rr_residual(Sink& s, cofem_ctx* c, int Q);
void launch_cg_direction(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg);
void launch_mstep(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_em);
void launch_probe_fill(cudaStream_t st, unsigned long long seed, int t, int K, long long D,
                       long long ld, float* out);
void launch_plain_psi(cudaStream_t st, cofem_ctx* c, int Q, const float* V, const float* alpha,
                      double beta, float* Psi);
void launch_quantize_bf16(cudaStream_t st, const float* src, long long rows, long long cols,
                          long long ld_src, __nv_bfloat16* dst, long long rows_dst, long long ld_dst);
void launch_check_finite(cudaStream_t st, const float* x, long long n, unsigned* bad);
void launch_dot_rows(cudaStream_t st, const float* a, long long lda, const float* b, long long ldb, long long n,
                     int rows, double* out);

// kernels_dense.cu
void dense_configure(cofem_ctx* c, int Q);
void launch_dense_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
void launch_dense_colreduce(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out);

// kernels_tc.cu (BF16 dictionary on tcgen05 tensor cores)
cudaError_t tc_setup(cofem_ctx* c, int Q);
void tc_release(cofem_ctx* c);
cudaError_t tc_make_transpose(cofem_ctx* c, cudaStream_t st);
void launch_tc_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);

// kernels_toeplitz.cu
size_t toeplitz_smem_bytes(int L);
cudaError_t toeplitz_prepare(int L);
void launch_toeplitz_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
void launch_toeplitz_theta(cudaStream_t st, cofem_ctx* c);
void launch_toeplitz_phit_y(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out);

// dispatch
inline void launch_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    if (c->kind == COFEM_OP_DENSE) launch_dense_operator(s, c, Q, V, mode);
    else launch_toeplitz_operator(s, c, Q, V, mode);
}

// Finish an operator application (run by the last block of an operator kernel):
// reduce the ||Phi p_q||^2 partials (layout [q][nparts]) into ctl->tt and, in
// OP_CG mode, form pi_q = p^T A p = beta ||Phi p_q||^2 + p^T diag(alpha) p and
// gamma_q = rho_q / pi_q (Alg. 2, "pi" and "gamma").  Writing pi through Phi p
// instead of sum_j P_jq Psi_jq is the same number in exact arithmetic and is a
// sum of non-negative terms.  A column with pi <= 0 or non-finite is frozen
// and flagged (CG breakdown).
__device__ __forceinline__ void op_finalize_block(DevCtl* ctl, const double* tt_part, int nparts,
                                                   int Q, int mode) {
    __shared__ double s_tt[COFEM_QMAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = w; q < Q; q += nw) {
        double v = 0.0;
        for (int i = lane; i < nparts; i += 32) v += __ldcg(&tt_part[(size_t)q * nparts + i]);
        v = warp_sum(v);
        if (lane == 0) s_tt[q] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double beta = ctl->beta;
        int any = 0;
        for (int q = 0; q < Q; ++q) {
            ctl->tt[q] = s_tt[q];
            if (mode == OP_CG && ctl->active[q]) {
                const double pi = beta * s_tt[q] + ctl->ap[q];
                ctl->pi[q] = pi;
                if (!(pi > 0.0) || !isfinite(pi)) {
                    ctl->flags |= COFEM_FLAG_BREAKDOWN;
                    ctl->active[q] = 0;
                    ctl->gamma[q] = 0.0;
                } else {
                    ctl->gamma[q] = ctl->rho[q] / pi;
                }
            }
            any |= ctl->active[q];
        }
        if (mode == OP_CG) ctl->any_active = any;
    }
}

// Records a failure message for cofem_last_error() (cofem_api.cu) and returns st.
cofem_status cofem_set_error(cofem_status st, const char* msg);

// Vector-kernel geometry
inline int vec_chunks(long long Dp) { return (int)((Dp + COFEM_VEC_CHUNK - 1) / COFEM_VEC_CHUNK); }
