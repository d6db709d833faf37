// Internal declarations shared by the libcofem translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/cofem.h"

#define COFEM_QMAX 64          // K <= 63
#ifndef COFEM_VEC_CHUNK
#define COFEM_VEC_CHUNK 4096   // elements of one column handled by a vector-kernel block
#endif
#define COFEM_VEC_THREADS 256
#define COFEM_DCT_MAX_D 32768  // largest DCT dictionary (D/2 complex points in shared memory)
#define COFEM_FFTCONV_LOGF 13  // FFT convolution: 8192-point overlap-save blocks

// ---------------------------------------------------------------------------
// Device-resident control block: fit parameters plus the per-column CG scalars
// of Alg. 2 (rho, pi, gamma, eta) and the loop counters.  Kept on the device so
// the EM and CG loops run without host round trips.
// ---------------------------------------------------------------------------
struct DevCtl {
    double beta, tol, alpha_max;
    unsigned long long seed;
    int T, K, Q, maxit, conv, rr_period, prior;
    int L;            // tasks (multi-task fit: Q = L (K + 1), column l (K+1) + k of task l)
    int precond_none; // M = I (unpreconditioned CG) instead of M = beta theta + alpha
    int warm;         // warm start with probe reuse: E-step t >= 2 starts from the previous X
                      // and every E-step draws the probes of t = 1
    int t;            // current EM iteration, 1-based
    int u;            // CG iterations done in EM iteration t
    int any_active;   // some column still iterating
    unsigned flags;   // COFEM_FLAG_* bits
    int active[COFEM_QMAX];
    double rho[2][COFEM_QMAX];  // r^T M^-1 r of the residual after u CG iterations, at [u & 1]
    double pi[COFEM_QMAX];      // p^T A p
    double gamma[COFEM_QMAX];   // rho / pi
    double eta[COFEM_QMAX];     // rho_new / rho_old
    double bnorm2[COFEM_QMAX];  // ||b_q||^2
    double rnorm2[COFEM_QMAX];  // ||r_q||^2
    double ap[COFEM_QMAX];      // p^T diag(alpha) p
    double tt[COFEM_QMAX];      // ||Phi p||^2
    const double* ap_part;      // per-block partials of p^T diag(alpha) p: [q][ap_n]
    int ap_n;
    const double* tt_part;      // the CG operator's partials of ||Phi p||^2: [q][tt_n]
    int tt_n;
    // precision form: accurate residual replacement and the true-residual check
    int fix_residual;           // 1: a column whose true residual misses tol restarts from it
    int verify_again;           // the last check restarted some column
    int n_rr, n_check;          // replacements and checks during the fit
    int broken[COFEM_QMAX];     // column frozen by a breakdown in this EM iteration
    int restart[COFEM_QMAX];    // column restarted by the last check
    double rt2[COFEM_QMAX];     // ||B - A X||^2 of the last check (FP32-pair product)
    int phase;                  // packed serving: what the next step does for this fit (PH_*)
};

// Phase of a fit in a packed serving step (cofem_server in packed mode): the
// kernels of one step (operator, update, direction) run only for PH_CG fits;
// the M-step runs for fits whose CG loop ended (or was never entered,
// PH_START), the initialisation for PH_INIT fits.  The initialisation and the
// M-step of every fit record it; only the packed step reads it.
#define PH_NONE 0
#define PH_CG 1
#define PH_START 2
#define PH_INIT 3
#define PH_DONE 4

// Column q of the block: task q / (K+1), and k = q mod (K+1) (0: the mu system
// beta Phi^T y_task, k >= 1: probe k of that task).
__device__ __forceinline__ void column_task(const DevCtl* ctl, int q, int& task, int& k) {
    const int Qt = ctl->K + 1;
    task = q / Qt;
    k = q - task * Qt;
}

// Modes of the accurate residual (kernels_accurate.cu).
#define DF_RR 0      // residual replacement: R = B - A X for the active columns
#define DF_CHECK 1   // true-residual check: Rt = B - A X for every column

// Modes of the operator kernels.
// OP_CG: apply to P inside the CG loop (forms pi, gamma; the tensor-core path
//        reads the split of P written by the direction kernel and leaves Psi as
//        segment partials for the update kernel);
// OP_PLAIN: stand-alone application (split made here, Psi summed into U);
// OP_TIME: the OP_CG launch sequence without touching the CG scalars (timing).
enum OpMode { OP_CG = 0, OP_PLAIN = 2, OP_TIME = 3 };

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

// The 64-bit word of the probe block that holds bits for j .. (j | 63); task
// is the counter's last word (multi-task fits; 0 for a single task).
__device__ __forceinline__ uint64_t probe_word(unsigned long long seed, int t, int k, long long j, int task = 0) {
    uint64_t c[4] = {(uint64_t)(j >> 8), (uint64_t)k, (uint64_t)t, (uint64_t)task};
    philox4x64_10(c, seed, 0ull);
    const int w = (int)((j & 255) >> 6);
    return w == 0 ? c[0] : (w == 1 ? c[1] : (w == 2 ? c[2] : c[3]));
}

__device__ __forceinline__ float probe_sign_from_word(uint64_t word, long long j) {
    return ((word >> (j & 63)) & 1ull) ? -1.0f : 1.0f;
}

// Right-hand side B[j][q] of the accurate residual: b of the column's task
// (k = 0) or its probe k of EM iteration t (of t = 1 under the warm start).
__device__ __forceinline__ double accurate_rhs(const DevCtl* ctl, const float* b, int q, long long j, long long D,
                                               long long Dp) {
    int task, k;
    column_task(ctl, q, task, k);
    if (k == 0) return (double)b[(size_t)task * Dp + j];
    if (j >= D) return 0.0;
    return (double)probe_sign_from_word(probe_word(ctl->seed, ctl->warm ? 1 : ctl->t, k, j, task), j);
}

// ---------------------------------------------------------------------------
// Reductions.  GB300 runs FP64 at a small fraction of the FP32 rate, so the
// per-element work of every inner product stays in FP32 and only the
// cross-warp, cross-block and grid levels are FP64.  All CG inner products of
// this path (r^T r, r^T M^-1 r, p^T diag(alpha) p, ||Phi p||^2, b^T b) are sums
// of non-negative terms, so the FP32 warp sums carry no cancellation.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of n per-block partials by one warp: lane l adds partials l, l + 32, ...
// in order, then a butterfly over the lanes; every lane, and every block that
// sums the same partials, gets the same bits.
__device__ __forceinline__ double warp_sum_parts(const double* src, int n) {
    double v = 0.0;
#pragma unroll 4
    for (int i = threadIdx.x & 31; i < n; i += 32) v += __ldcg(src + i);
    return warp_sum(v);
}

// Block sum of per-thread FP32 values: FP32 within each warp, FP64 across warps
// (fixed order, deterministic).  The result is valid in thread 0.  `sh` needs
// blockDim/32 doubles.
__device__ __forceinline__ double block_sum_f(float v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum_f(v);
    __syncthreads();   // sh may still be read by a previous call
    if (lane == 0) sh[wid] = (double)v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// Block sum of FP64 values (cold paths), result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    return r;
}

// "Last block done" arrival (threadfence reduction pattern, no spinning): the
// block barrier orders every thread's partial writes before thread 0's
// device-scope fence, thread 0 counts arrivals, and the block that arrives last
// gets true (after a second fence, so its reads see all partials) and resets
// the counter for the next launch.  One fence per block, not per thread.
__device__ __forceinline__ bool last_block_arrive(unsigned* counter, unsigned total) {
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        s_last = (prev == total - 1);
        if (s_last) {
            __threadfence();
            *counter = 0u;
        }
    }
    __syncthreads();
    return s_last != 0;
}

// ---------------------------------------------------------------------------
// Tensor-core operand formats (used by kernels_tc.cu and by the vector kernels
// that write the split direction block directly).
// ---------------------------------------------------------------------------
// Offset (in elements) of element (row, col) inside a tiled, 128-byte-swizzled
// image of a matrix with `rows_per_tile` rows per 64-column tile: tile k = col/64
// holds rows_per_tile x 64 bf16, row r at r * 64, 16-byte chunk c of the row at
// chunk position c ^ (r & 7).
__device__ __forceinline__ size_t swz_offset(int row, long long col, int rows_per_tile) {
    const long long k = col >> 6;
    const int cc = (int)(col & 63);
    return (size_t)k * rows_per_tile * 64 + (size_t)row * 64 + (size_t)((((cc >> 3) ^ (row & 7)) << 3) | (cc & 7));
}

// v = hi + mid + lo with hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid)
__device__ __forceinline__ void split3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// Write the three bf16 terms of v.x..v.w (columns j..j+3 of column q; j % 4 == 0,
// so the four share one 16-byte chunk) into the tiled image Vs.
__device__ __forceinline__ void store_split4(__nv_bfloat16* Vs, int QS, int q, long long j, float4 v) {
    __nv_bfloat16 t[3][4];
    split3(v.x, t[0][0], t[1][0], t[2][0]);
    split3(v.y, t[0][1], t[1][1], t[2][1]);
    split3(v.z, t[0][2], t[1][2], t[2][2]);
    split3(v.w, t[0][3], t[1][3], t[2][3]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        *reinterpret_cast<uint2*>(Vs + swz_offset(3 * q + k, j, QS)) = *reinterpret_cast<const uint2*>(t[k]);
}

// FP32 counterpart of swz_offset: 32-column tiles of 128-byte rows, 4 floats
// per 16-byte chunk.
__device__ __forceinline__ size_t swz32_offset(int row, long long col, int rows_per_tile) {
    const long long k = col >> 5;
    const int cc = (int)(col & 31);
    return (size_t)k * rows_per_tile * 32 + (size_t)row * 32 + (size_t)((((cc >> 2) ^ (row & 7)) << 2) | (cc & 3));
}

// Round to the nearest TF32 value (10 explicit mantissa bits, ties away from
// zero), kept as an FP32 bit pattern whose low 13 bits are zero, so the tensor
// core reads it exactly.
__device__ __forceinline__ float tf32_rn(float x) {
    return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// TF32 split v = hi + lo with hi = tf32_rn(v) and lo = tf32_rn(v - hi): hi at row
// q, lo at row QH + q of the tiled fp32 image (columns j..j+3, j % 4 == 0: one
// 16-byte chunk).
__device__ __forceinline__ void store_split_tf32(float* Vs, int QS, int QH, int q, long long j, float4 v) {
    float4 hi, lo;
    hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
    lo = make_float4(tf32_rn(v.x - hi.x), tf32_rn(v.y - hi.y), tf32_rn(v.z - hi.z), tf32_rn(v.w - hi.w));
    *reinterpret_cast<float4*>(Vs + swz32_offset(q, j, QS)) = hi;
    *reinterpret_cast<float4*>(Vs + swz32_offset(QH + q, j, QS)) = lo;
}

// Where the CG direction kernels write the split of P for the tensor-core
// GEMM (fmt 0: no tensor-core operator, 1: bf16 3-term image, 2: TF32 image).
struct SplitOut {
    void* Vs;
    int fmt, QS, QH;
    float scale = 1.0f;   // power of two applied before the split (FP8 operator: 2^64)
};

__device__ __forceinline__ void store_split(const SplitOut& so, int q, long long j, float4 v) {
    if (so.scale != 1.0f) v = make_float4(v.x * so.scale, v.y * so.scale, v.z * so.scale, v.w * so.scale);
    if (so.fmt == 1) store_split4((__nv_bfloat16*)so.Vs, so.QS, q, j, v);
    else if (so.fmt == 2) store_split_tf32((float*)so.Vs, so.QS, so.QH, q, j, v);
}

// Operator output: either S2 dense slices U_s (Q x Dp each, stride sstride) or,
// for the tensor-core path, stream-K segment partials part[seg][Q][GR] with
// the segments of row group g listed in grp_seg[2g], grp_seg[2g+1].
struct OpOut {
    const float* U;
    int S2;
    size_t sstride;
    const int* grp_seg;   // null for dense slices
    int GR;
    float uscale = 1.0f;  // power of two the partials carry (FP8 operator: 2^56)
};

// The operator partials for elements j..j+3: the segment range [s0, s0 + ns) of
// their row group (tensor-core path), or the S2 dense slices.
__device__ __forceinline__ void op_range(const OpOut& o, long long j, int& s0, int& ns) {
    if (o.grp_seg) {
        const int g = (int)(j / o.GR);
        s0 = o.grp_seg[2 * g];
        ns = o.grp_seg[2 * g + 1];
    } else {
        s0 = 0;
        ns = o.S2;
    }
}

// Sum of those partials in segment order; the loads of the first four are
// issued together (one memory round trip for the usual two to four).
__device__ __forceinline__ float4 op_sum4(const OpOut& o, int Q, int q, long long Dp, long long j, int s0, int ns) {
    float4 w[4];
    const float* base;
    size_t step;
    if (o.grp_seg) {
        base = o.U + ((size_t)s0 * Q + q) * o.GR + (size_t)(j % o.GR);
        step = (size_t)Q * o.GR;
    } else {
        base = o.U + (size_t)q * Dp + j;
        step = o.sstride;
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (s < ns) w[s] = *reinterpret_cast<const float4*>(base + (size_t)s * step);
    float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (s < ns) { u.x += w[s].x; u.y += w[s].y; u.z += w[s].z; u.w += w[s].w; }
    for (int s = 4; s < ns; ++s) {
        const float4 x = *reinterpret_cast<const float4*>(base + (size_t)s * step);
        u.x += x.x; u.y += x.y; u.z += x.z; u.w += x.w;
    }
    return u;
}

// ---------------------------------------------------------------------------
// Packed serving: the kernels of one CG step of several fits in one launch
// each (serve.cu builds the tables; kernels_tc.cu and kernels_vec.cu run them).
// ---------------------------------------------------------------------------
// One fit's product for the packed GEMM, and a segment of it.
struct TcSlot {
    const uint8_t* A;     // tiled A image of the fit's product
    const uint8_t* B;     // its B image (split block), k tile at k QS 128 bytes
    const DevCtl* ctl;    // the fit's phase: only PH_CG fits run
    float* part;          // the fit's segment partials [segment][Q][G 128]
    uint32_t idesc, idesc_lo;
    int K_tiles, M_tiles, QS, QH, Q;
};
struct TcSeg {
    int slot, g, k0, k1;  // fit, row group, k tiles [k0, k1)
    int out;              // segment index within the fit's partials
};
struct TcBatch {
    const TcSlot* slots;
    const TcSeg* segs;
    const int* cta_seg;   // CTA c runs segments [cta_seg[c], cta_seg[c + 1])
    int G, acc_stride, QSmax;
    unsigned* flags;
};

// One fit's vectors and control block for the packed vector kernels.
struct VSlot {
    DevCtl* ctl;
    const float* b;
    const float* theta;
    float *alpha, *minv, *X, *R, *P, *mu_out, *s_out;
    int* iters;
    long long D, Dp, Np;
    int nch, Q;
    double* part;          // CG partials, 3 x Q x nch
    unsigned* counters;    // the fit's last-block counters
    SplitOut so;           // split image of P (the first product's B operand)
    OpOut uo;              // the second product's segment partials
    const float* t_part;   // the first product's segment partials [segment][Q][GR]
    const int* t_grp;      // their (first segment, count) per row group
    int GR;
    SplitOut st;           // split image of T (the second product's B operand)
    double* tt_part;       // partials of ||Phi p||^2, [q][ceil(Np / 1024)]
};

// ---------------------------------------------------------------------------
// Launch sink: the same launch sequence either runs directly on a stream or is
// recorded as kernel nodes of a CUDA graph (linear chain), with conditional
// WHILE / IF bodies for the device-side loops.
// ---------------------------------------------------------------------------
struct Sink {
    cudaStream_t stream = nullptr;
    cudaGraph_t graph = nullptr;   // null -> direct launches
    cudaGraphNode_t last = nullptr;
    bool last_kernel = false;      // whether `last` is a kernel node
    bool pdl = false;              // launch_pdl() may overlap (else a plain launch)
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
        if (err == cudaSuccess) {
            last = n;
            last_kernel = true;
        }
    }

    // Launch that may start while the previous kernel (of this sink) is still
    // running: a programmatic edge in a graph, programmatic stream serialisation
    // when launching directly.  The kernel must call griddep_wait() before it
    // reads what the previous kernel writes.  After a non-kernel node it is an
    // ordinary launch.
    template <typename... P, typename... A>
    void launch_pdl(void (*f)(P...), dim3 grid, dim3 block, size_t smem, A... args) {
        if (err != cudaSuccess) return;
        if (grid.x == 0 || grid.y == 0 || grid.z == 0) return;
        if (!pdl) {
            launch(f, grid, block, smem, args...);
            return;
        }
        pdl_typed<P...>(f, grid, block, smem, static_cast<P>(args)...);
    }

    template <typename... P>
    void pdl_typed(void (*f)(P...), dim3 grid, dim3 block, size_t smem, P... args) {
        void* ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1] = {(void*)&args...};
        if (!graph) {
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            attr[0].val.programmaticStreamSerializationAllowed = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = block;
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            err = cudaLaunchKernelExC(&cfg, (const void*)f, ptrs);
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
        if (!last || !last_kernel) {
            err = cudaGraphAddKernelNode(&n, graph, last ? &last : nullptr, last ? 1 : 0, &p);
        } else {
            err = cudaGraphAddKernelNode(&n, graph, nullptr, 0, &p);
            if (err == cudaSuccess) {
                cudaGraphEdgeData e = {};
                e.from_port = cudaGraphKernelNodePortProgrammatic;
                e.to_port = 0;
                e.type = cudaGraphDependencyTypeProgrammatic;
                err = cudaGraphAddDependencies(graph, &last, &n, &e, 1);
            }
        }
        if (err == cudaSuccess) {
            last = n;
            last_kernel = true;
        }
    }

    // Cooperative launch (all CTAs co-resident; the kernel may wait on other CTAs).
    template <typename... P, typename... A>
    void launch_cooperative(void (*f)(P...), dim3 grid, dim3 block, size_t smem, A... args) {
        if (err != cudaSuccess) return;
        coop_typed<P...>(f, grid, block, smem, static_cast<P>(args)...);
    }

    template <typename... P>
    void coop_typed(void (*f)(P...), dim3 grid, dim3 block, size_t smem, P... args) {
        void* ptrs[sizeof...(P) > 0 ? sizeof...(P) : 1] = {(void*)&args...};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        if (!graph) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = block;
            cfg.dynamicSmemBytes = smem;
            cfg.stream = stream;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            err = cudaLaunchKernelExC(&cfg, (const void*)f, ptrs);
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
        if (err != cudaSuccess) return;
        err = cudaGraphKernelNodeSetAttribute(n, cudaLaunchAttributeCooperative, &attr[0].val);
        if (err == cudaSuccess) {
            last = n;
            last_kernel = true;
        }
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
        body.pdl = pdl;
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
        last_kernel = false;
        body.graph = np.conditional.phGraph_out[0];
        return body;
    }
};

// Sets a graph conditional from one device thread (no-op for a zero handle,
// used in the direct-launch mode).
// Programmatic dependent launch: a kernel launched with a programmatic edge
// may start before its predecessor finishes; griddep_wait() blocks until the
// predecessor has completed and its writes are visible (no-op otherwise), and
// griddep_launch() lets this kernel's own dependents start early.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int v) {
    if (h) cudaGraphSetConditional(h, v ? 1u : 0u);
}

// CG step u is a residual-replacement step (Alg. 2 with replacement every
// rr_period steps): the update's decision, read again by the kernels of the
// step that a fit graph defers until after the replacement.
__device__ __forceinline__ bool rr_step(const DevCtl* ctl) {
    return ctl->rr_period > 0 && ctl->u % ctl->rr_period == 0;
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
    void* tc = nullptr;              // tensor-core operator plan (kernels_tc.cu)
    bool use_tc = false;             // dense dictionary applied on the tensor cores
    float* h = nullptr;              // Toeplitz filter, L floats
    bool use_fftconv = false;        // convolution applied through FFTs (kernels_fftconv.cu)
    float2* fc_H = nullptr;          // FFT convolution: DFT of h (8192 points)
    float2* fc_tw = nullptr;         // FFT convolution: twiddles (4096)
    int* dct_rows = nullptr;         // DCT dictionary: the N kept rows of Omega^-1
    float* dct_mask = nullptr;       // DCT dictionary: 1 at the kept rows, Dp floats
    float2* dct_tw = nullptr;        // DCT dictionary: FFT twiddles e^{-2 pi i m / (D/2)}, D/4 of them
    float* theta = nullptr;          // Dp

    // fit workspace (sized for Qcap columns)
    int Qcap = 0;
    int QP = 0;                      // padded column count of the dense intermediate T
    float *X = nullptr, *R = nullptr, *P = nullptr;   // Qcap x Dp each
    float *U = nullptr;              // operator output partials, S2 x Qcap x Dp
    float *alpha = nullptr, *minv = nullptr;          // Dp
    float *b = nullptr, *yv = nullptr;                // Lcap x Dp (yv: Lcap x Np): one per task
    float *mu_out = nullptr, *s_out = nullptr;        // Lcap x Dp
    int Lcap = 1;                                     // tasks the per-task buffers hold
    int graph_L = -1;                                 // tasks of the cached fit graph
    float *T = nullptr;              // dense: Np x QP
    float *Tpart = nullptr;          // dense: S1 x Np x QP
    double* part = nullptr;          // vector-kernel partials: 3 x Qcap x nch
    double* tt_part = nullptr;       // operator partials of ||Phi p||^2
    unsigned* counters = nullptr;    // last-block counters
    unsigned* check_flag = nullptr;  // one word for input finiteness checks
    uint8_t* phi8 = nullptr;         // FP8 E4M3 codes (Np x Dp), FP8 form
    float* scale8 = nullptr;         // per-row scales (Np), FP8 form
    // precision form (rr_period > 0 or check_residual): X = X + Xlo as an FP32
    // pair, the accurate residual's buffers, per-E-step true residuals
    float* Xlo = nullptr;            // Qcap x Dp
    float* Rt = nullptr;             // Qcap x Dp: the last checked true residual
    double* df_T = nullptr;          // k-split partials of Phi~ X
    float *df_thi = nullptr, *df_tlo = nullptr;   // Phi~ X as an FP32 pair
    double* df_U = nullptr;          // k-split partials of Phi~^T t: [s][q][j]
    double* res_dev = nullptr;       // iters_cap x COFEM_QMAX relative true residuals
    int df_QP = 0, df_S1 = 1, df_S2 = 1;
    int last_T = 0, last_Q = 0;      // EM iterations and columns of the last fit
    int last_rr = 0, last_check = 0; // residual replacements and checks of the last fit
    long long df_k1 = 0, df_k2 = 0;
    void* sl = nullptr;              // tensor-core form of the accurate residual (kernels_sliced.cu)
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
    bool graph_pdl = false;   // the fit graph has programmatic edges

    long long bytes = 0;
    std::unordered_map<void*, size_t> alloc_bytes;   // size of every live device allocation
};

// ---------------------------------------------------------------------------
// Kernel launchers (defined in the .cu files).
// ---------------------------------------------------------------------------
// kernels_vec.cu
void launch_fit_setup(Sink& s, cofem_ctx* c, int Q);                 // alpha -> minv, ctl t = 1
void launch_cg_init(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg);
void launch_cg_update(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_rr,
                      cudaGraphConditionalHandle h_cg);
void launch_cg_direction(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg, bool defer_rr = false);
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

// kernels_accurate.cu (precision form)
struct DfSizes {
    int QP, S1, S2;
    long long k1, k2;
    size_t t, T, U;   // elements of df_thi / df_tlo, df_T, df_U
};
DfSizes df_configure(cofem_ctx* c, int Q);
void launch_true_residual(Sink& s, cofem_ctx* c, int Q, int mode);
int true_residual_kernels(cofem_ctx* c);
cudaError_t df_kernel_attributes();
void launch_df_first_product(Sink& s, cofem_ctx* c, int Q);   // dense only
void launch_df_check(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_vf);
void launch_cg_gate(Sink& s, cofem_ctx* c, cudaGraphConditionalHandle h_set, cudaGraphConditionalHandle h_clear = 0);
void launch_df_gram(Sink& s, cofem_ctx* c, int Q, double* out);   // Phi~^T Phi~ (X + Xlo), dense

// Packed serving (kernels_tc.cu, kernels_vec.cu, cofem_api.cu)
#define PK_SEGK 16   // k tiles per segment of the packed GEMM
struct PackedFit {   // what serve.cu needs of one fit's tensor-core plan
    TcSlot g1, g2;                      // the two products
    std::vector<TcSeg> s1, s2;          // their fixed segments (slot field 0)
    std::vector<double> c1, c2;         // bytes of the dictionary image each segment reads
    bool tf;                            // 3xTF32 products (else BF16)
};
cudaError_t tc_pack_setup(cofem_ctx* c);                       // fixed segments and their partials
void tc_pack_describe(cofem_ctx* c, PackedFit* out);
void tc_pack_vslot(cofem_ctx* c, VSlot* out);
size_t tc_packed_smem(bool tf, int QSmax);
void launch_gemm_packed(Sink& s, bool tf, const TcBatch& b, int nCTA, size_t smem);
// grids are sized for a capacity (nblocks); blocks at or beyond *count return
void launch_reduce_T_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks);
void launch_update_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks);
void launch_direction_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks);
void launch_mstep_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks);
void launch_init_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks);
void launch_packed_status(Sink& s, const VSlot* vs, const int* nfits, int* status, const volatile int* pending,
                          unsigned* steps, unsigned max_steps, cudaGraphConditionalHandle h_loop);
// fit prologue up to the first E-step's initialisation, and the epilogue
cofem_status packed_prepare(cofem_ctx* c, const cofem_request& r);
cofem_status packed_finish(cofem_ctx* c, const cofem_request& r, unsigned* flags);

// kernels_sliced.cu (precision form, BF16 dictionary: the accurate residual
// from exact integer slices on the tensor cores)
bool sl_applies(const cofem_ctx* c, int Q);
cudaError_t sl_setup(cofem_ctx* c, int Q);
void sl_release(cofem_ctx* c);
cudaError_t sl_kernel_attributes(int max_smem);
int sl_kernels();
void launch_sl_first_product(Sink& s, cofem_ctx* c, int Q);
void launch_sl_residual(Sink& s, cofem_ctx* c, int Q, int mode);
void launch_sl_gram(Sink& s, cofem_ctx* c, int Q, double* out);

// kernels_dense.cu
void dense_configure(cofem_ctx* c, int Q);
void launch_dense_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
void launch_dense_colreduce(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out);

// kernels_tc.cu (BF16 dictionary on tcgen05 tensor cores)
cudaError_t tc_setup(cofem_ctx* c, int Q);
cudaError_t tc_kernel_attributes(int max_smem);
void tc_release(cofem_ctx* c);
void launch_tc_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
// the operator of the CG loop split in two: the first product alone, and the
// T reduction with the second product (two-pass tensor-core forms)
bool tc_rotatable(cofem_ctx* c);
void launch_tc_first_product(Sink& s, cofem_ctx* c, bool defer_rr = false);
void launch_tc_rest(Sink& s, cofem_ctx* c, int Q, int mode);
// Split image of the CG direction block (written by k_cg_init / k_cg_direction)
// and the description of the operator output (null / dense slices otherwise).
SplitOut tc_direction_split(cofem_ctx* c);
OpOut op_output(cofem_ctx* c);

// kernels_toeplitz.cu
size_t toeplitz_smem_bytes(int L);
cudaError_t toeplitz_prepare(int L);
cudaError_t toeplitz_kernel_attributes();
void launch_toeplitz_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
void launch_toeplitz_theta(cudaStream_t st, cofem_ctx* c);
void launch_toeplitz_phit_y(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out);

// kernels_dct.cu
size_t dct_smem_bytes(long long D);
cudaError_t dct_kernel_attributes();
void launch_dct_setup(cudaStream_t st, cofem_ctx* c);
void launch_dct_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);
void launch_dct_phit_y(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out, float* tmp);

// kernels_fftconv.cu
size_t fftconv_smem_bytes();
cudaError_t fftconv_kernel_attributes();
int fftconv_bout(int L);
void launch_fftconv_setup(cudaStream_t st, cofem_ctx* c);
void launch_fftconv_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode);

// dispatch
inline void launch_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    if (c->kind == COFEM_OP_DENSE) launch_dense_operator(s, c, Q, V, mode);
    else if (c->kind == COFEM_OP_DCT) launch_dct_operator(s, c, Q, V, mode);
    else if (c->use_fftconv) launch_fftconv_operator(s, c, Q, V, mode);
    else launch_toeplitz_operator(s, c, Q, V, mode);
}

// End of an operator application that left per-block partials of
// ||Phi p_q||^2 (layout [q][nparts]).  Outside the CG loop one block (the
// last to arrive) reduces them into ctl->tt (op_finalize_block).  In the CG
// loop (OP_CG) nothing is reduced here: the update kernel's blocks form
// pi_q = p^T A p = beta ||Phi p_q||^2 + p^T diag(alpha) p and
// gamma_q = rho_q / pi_q (Alg. 2, "pi" and "gamma") from the partials
// themselves; one thread of the operator records where the partials are and
// counts the CG iteration (op_cg_begin).  Writing pi through Phi p instead of
// sum_j P_jq Psi_jq is the same number in exact arithmetic and is a sum of
// non-negative terms.
__device__ __forceinline__ void op_cg_begin(DevCtl* ctl, const double* tt_part, int nparts) {
    ctl->tt_part = tt_part;
    ctl->tt_n = nparts;
    ctl->u += 1;
}

__device__ __forceinline__ void op_finalize_block(DevCtl* ctl, const double* tt_part, int nparts, int Q) {
    __shared__ double s_tt[COFEM_QMAX];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = w; q < Q; q += nw) {
        double v = 0.0;
        for (int i = lane; i < nparts; i += 32) v += __ldcg(&tt_part[(size_t)q * nparts + i]);
        v = warp_sum(v);
        if (lane == 0) s_tt[q] = v;
    }
    __syncthreads();
    if (threadIdx.x < Q) ctl->tt[threadIdx.x] = s_tt[threadIdx.x];
}

void tc_operator_info(cofem_ctx* c, int* path, int* k_cg, int* k_rr);

// FP8 E4M3 dictionary storage (kernels_fp8.cu).
void launch_quantize_fp8(cudaStream_t st, const float* src, long long ld, long long N, long long D, long long Np,
                         long long Dp, uint8_t* codes, float* scales);
void launch_colreduce_fp8(cudaStream_t st, const uint8_t* codes, const float* scales, long long Dp, long long N,
                          long long D, const float* y, double scale, float* out);
void launch_dequant_fp8(cudaStream_t st, const uint8_t* codes, const float* scales, long long N, long long D,
                        long long Dp, float* out);
void launch_bf16_to_f32(cudaStream_t st, const __nv_bfloat16* src, long long N, long long D, long long ld,
                        float* out);

// Single-pass BF16 dense operator (kernels_fused.cu).
struct FusedPlan;
size_t fused_smem_bytes(int QS);
bool fused_supported(int num_sms, long long Dp, int QS, bool coop, int max_smem);
cudaError_t fused_create(FusedPlan** out, int num_sms, long long Np, long long Dp, int Q, int QS,
                         const void* A_image, const void* Bv, void* Bt, float* U, DevCtl* ctl, cudaStream_t st,
                         long long* bytes);
void fused_destroy(FusedPlan* f, cudaStream_t st);
void launch_fused(Sink& s, const FusedPlan* f, int mode);
cudaError_t fused_kernel_attributes(int max_smem);

// Records a failure message for cofem_last_error() (cofem_api.cu) and returns st.
cofem_status cofem_set_error(cofem_status st, const char* msg);

// Vector-kernel geometry
inline int vec_chunks(long long Dp) { return (int)((Dp + COFEM_VEC_CHUNK - 1) / COFEM_VEC_CHUNK); }
