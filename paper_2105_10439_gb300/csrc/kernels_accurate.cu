// Accurate residual R = B - A X of the precision form: residual replacement
// inside the CG loop and the true-residual check at the end of each E-step.
//
// Why a separate path.  The CG state is FP32 and the operator of the CG loop
// accumulates in FP32, so its error is about 2^-24 ||A| |x||.  On the
// underdetermined dictionaries of the dense workloads most of a probe
// solution lies in the null space of Phi, where beta Phi^T (Phi x) is a
// cancellation of terms 10^3-10^4 times larger than the right-hand side: an
// FP32 product then cannot tell whether ||b - A x|| <= 1e-5 ||b||.  Here X is
// held as an unevaluated pair of FP32 numbers (X + Xlo, updated exactly by the
// CG kernels) and A X is formed with error-free transformations in FP32 pairs
// (TwoProduct through the FMA, Knuth's TwoSum: the compensated dot product of
// Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput.
// 2005), which carries about 2^-48 relative error; partial sums across
// threads and blocks and the residual itself are FP64.  The GB300's FP64 rate
// is a small fraction of its FP32 rate, so the inner products stay in FP32
// pairs on the CUDA cores.
//
// Dense dictionary (row-major Phi~, FP32 / BF16 / FP8 codes with row scales):
//   k_df_gemm<E, false, false>  T_s = Phi~ X over a k range s, every product
//                               and sum error-free (FP64 partials)
//   k_df_combine_t              t = sum_s T_s (times s_i^2 for FP8) as an FP32 pair
//   k_df_gemm<E, true, true>    U_s = Phi~^T t over an i range s: plain FP32
//                               sums of 32 terms, folded into FP32 pairs
//   k_df_residual               R = B - beta sum_s U_s - alpha X (FP64), norms
// The cancellation is in T = Phi~ X (X mostly in Phi's null space); U is not
// a cancellation of that kind, and FP32 sums of 32 terms, combined exactly,
// leave an error near 1e-7 ||b|| in the residual (measured in an FP32
// emulation at 1024 x 4096), so the second product takes two FMAs per term
// instead of the eleven instructions of the error-free form.
// Convolution dictionary:
//   k_df_conv, k_df_conv_t (direct sums over the L taps), k_df_residual.
#include <algorithm>

#include <cuda_fp8.h>

#include "cofem_internal.cuh"

namespace {

constexpr int NT = COFEM_VEC_THREADS;
constexpr int CH = COFEM_VEC_CHUNK;

// ---------------------------------------------------------------------------
// FP32-pair arithmetic.  The _rn intrinsics are never contracted into FMAs,
// which the error-free transformations rely on.
// ---------------------------------------------------------------------------
// (S, C) += a * (xh + xl): p + e = a * xh exactly (FMA), a * xl is below the
// pair's precision in its own rounding; S + p = s + t exactly (TwoSum).
__device__ __forceinline__ void df_mac(float& S, float& C, float a, float xh, float xl) {
    const float p = __fmul_rn(a, xh);
    float e = __fmaf_rn(a, xh, -p);
    e = __fmaf_rn(a, xl, e);
    const float s = __fadd_rn(S, p);
    const float z = __fsub_rn(s, S);
    const float t = __fadd_rn(__fsub_rn(S, __fsub_rn(s, z)), __fsub_rn(p, z));
    S = s;
    C = __fadd_rn(C, __fadd_rn(t, e));
}

// x = hi + lo with hi = fl(x), |lo| <= ulp(hi) / 2 (split of an FP64 value).
__device__ __forceinline__ void df_split(double x, float& hi, float& lo) {
    hi = (float)x;
    lo = (float)(x - (double)hi);
}

template <typename E> __device__ __forceinline__ float elem(E v);
template <> __device__ __forceinline__ float elem<float>(float v) { return v; }
template <> __device__ __forceinline__ float elem<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
// an E4M3 code as its value (exact: every E4M3 value is an FP16 value)
template <> __device__ __forceinline__ float elem<uint8_t>(uint8_t v) {
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)v, __NV_E4M3)));
}

// ---------------------------------------------------------------------------
// Dense product in FP32 pairs.  out[s][m][q] = sum over k in chunk s of
// A(m, k) (Xh + Xl)(k, q), with A(m, k) = A[m lda + k] (TRANS false: Phi~ X)
// or A[k lda + m] (TRANS true: Phi~^T t), X(k, q) = X[k xk + q xq].  M and K
// are the padded extents (the padding of Phi~, X and t is zero), so every
// tile is whole.  A block owns DF_BM rows of the output and all (padded) QP
// columns for one k chunk; thread (tm, tq) keeps the rows tm + 16 a (a < 4)
// and the columns 4 tq .. 4 tq + 3 as FP32 pairs.  Tiles of DF_KC k values
// arrive by cp.async through a three-stage ring, so the copies of the next
// tiles overlap the arithmetic on tile t; the dictionary tile stays in its storage type (FP32,
// BF16 or E4M3 codes) in shared memory and is widened when read.
// ---------------------------------------------------------------------------
constexpr int DF_BM = 64, DF_KC = 32, DF_TM = 4, DF_TQ = 4, DF_NBUF = 3;

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename E> struct DfTile {
    // elements per 4-byte copy; row stride of the shared tile in elements
    static constexpr int PER = 4 / (int)sizeof(E);
    // [m][k] (TRANS false): DF_KC + pad elements per row, an odd number of
    // 4-byte words so that 16 consecutive rows fall in 16 banks
    static constexpr int ROWK = sizeof(E) == 4 ? DF_KC + 1 : (sizeof(E) == 2 ? DF_KC + 2 : DF_KC + 4);
    static constexpr int ELEMS_N = DF_BM * ROWK;     // TRANS false
    static constexpr int ELEMS_T = DF_KC * DF_BM;    // TRANS true: [k][m]
    static constexpr int ELEMS = ELEMS_N > ELEMS_T ? ELEMS_N : ELEMS_T;
};

template <typename E, bool TRANS, bool BLOCKED>
__global__ __launch_bounds__(256) void k_df_gemm(const E* __restrict__ A, long long lda, long long M, long long K,
                                                 long long kchunk, const float* __restrict__ Xh,
                                                 const float* __restrict__ Xl, long long xk, long long xq, int Q,
                                                 int QP, double* __restrict__ out, long long osS, long long osM,
                                                 long long osQ) {
    using TT = DfTile<E>;
    extern __shared__ __align__(16) unsigned char df_smem[];
    E* As = reinterpret_cast<E*>(df_smem);                                  // [DF_NBUF][TT::ELEMS]
    const int QS = QP + 4;                                                  // row of the X tiles
    float* Hs = reinterpret_cast<float*>(df_smem + ((DF_NBUF * TT::ELEMS * sizeof(E) + 15) / 16) * 16);
    float* Ls = Hs + DF_NBUF * DF_KC * QS;                                  // [DF_NBUF][KC][QS] each
    const int nthr = blockDim.x;
    const int tm = threadIdx.x % (DF_BM / DF_TM), tq = threadIdx.x / (DF_BM / DF_TM);
    const long long m0 = (long long)blockIdx.x * DF_BM;
    const long long kb = (long long)blockIdx.y * kchunk;
    const long long ke = kb + kchunk < K ? kb + kchunk : K;
    const int ntiles = (int)((ke - kb + DF_KC - 1) / DF_KC);

    auto issue = [&](int tile, int buf) {
        const long long k0 = kb + (long long)tile * DF_KC;
        E* a = As + buf * TT::ELEMS;
        constexpr int CPR = DF_KC / TT::PER;    // 4-byte copies per tile row
        if (TRANS) {   // rows k, DF_BM contiguous elements of m
            for (int e = threadIdx.x; e < DF_KC * (DF_BM / TT::PER); e += nthr) {
                const int kk = e / (DF_BM / TT::PER), c = e % (DF_BM / TT::PER);
                const long long k = k0 + kk;
                const bool v = k < ke && m0 + c * TT::PER < M;
                cp_async4(a + kk * DF_BM + c * TT::PER, v ? (const void*)(A + k * lda + m0 + c * TT::PER) : (const void*)A, v);
            }
        } else {       // rows m, DF_KC contiguous elements of k
            for (int e = threadIdx.x; e < DF_BM * CPR; e += nthr) {
                const int mm = e / CPR, c = e % CPR;
                const long long m = m0 + mm;
                const bool v = m < M && k0 + c * TT::PER < ke;
                cp_async4(a + mm * TT::ROWK + c * TT::PER, v ? (const void*)(A + m * lda + k0 + c * TT::PER) : (const void*)A, v);
            }
        }
        float* h = Hs + buf * DF_KC * QS;
        float* l = Ls + buf * DF_KC * QS;
        for (int e = threadIdx.x; e < DF_KC * QP; e += nthr) {
            int kk, q;
            if (xq == 1) { kk = e / QP; q = e % QP; }   // contiguous in q
            else { q = e / DF_KC; kk = e % DF_KC; }      // contiguous in k
            const long long k = k0 + kk;
            const bool v = q < Q && k < ke;
            const long long idx = v ? k * xk + (long long)q * xq : 0;
            cp_async4(h + kk * QS + q, Xh + idx, v);
            cp_async4(l + kk * QS + q, Xl + idx, v);
        }
        cp_async_commit();
    };

    float S[DF_TM][DF_TQ], C[DF_TM][DF_TQ];
#pragma unroll
    for (int a = 0; a < DF_TM; ++a)
#pragma unroll
        for (int b = 0; b < DF_TQ; ++b) S[a][b] = C[a][b] = 0.0f;
    // three buffers: tile t + 2 is issued after the barrier of iteration t,
    // into the buffer every thread finished reading in iteration t - 1, so one
    // barrier per tile suffices
    if (ntiles > 0) issue(0, 0);
    if (ntiles > 1) issue(1, 1);
    for (int t = 0; t < ntiles; ++t) {
        const int buf = t % DF_NBUF;
        if (t + 1 < ntiles) cp_async_wait1();
        else cp_async_wait0();
        __syncthreads();   // tile t has landed for every thread; tile t - 1 is done
        if (t + 2 < ntiles) issue(t + 2, (t + 2) % DF_NBUF);
        const E* a = As + buf * TT::ELEMS;
        const float* h = Hs + buf * DF_KC * QS;
        const float* l = Ls + buf * DF_KC * QS;
        float B_[DF_TM][DF_TQ];   // BLOCKED: this tile's plain FP32 sums
        if (BLOCKED) {
#pragma unroll
            for (int r = 0; r < DF_TM; ++r)
#pragma unroll
                for (int c = 0; c < DF_TQ; ++c) B_[r][c] = 0.0f;
        }
#pragma unroll 2
        for (int kk = 0; kk < DF_KC; ++kk) {
            float av[DF_TM];
#pragma unroll
            for (int r = 0; r < DF_TM; ++r)
                av[r] = elem<E>(TRANS ? a[kk * DF_BM + tm + 16 * r] : a[(tm + 16 * r) * TT::ROWK + kk]);
            const float4 h4 = *reinterpret_cast<const float4*>(h + kk * QS + tq * DF_TQ);
            const float4 l4 = *reinterpret_cast<const float4*>(l + kk * QS + tq * DF_TQ);
            const float hv[4] = {h4.x, h4.y, h4.z, h4.w};
            const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
            for (int r = 0; r < DF_TM; ++r)
#pragma unroll
                for (int c = 0; c < DF_TQ; ++c) {
                    if (BLOCKED) B_[r][c] = fmaf(av[r], lv[c], fmaf(av[r], hv[c], B_[r][c]));
                    else df_mac(S[r][c], C[r][c], av[r], hv[c], lv[c]);
                }
        }
        if (BLOCKED) {   // fold the tile's sums into the FP32 pairs exactly (TwoSum)
#pragma unroll
            for (int r = 0; r < DF_TM; ++r)
#pragma unroll
                for (int c = 0; c < DF_TQ; ++c) df_mac(S[r][c], C[r][c], 1.0f, B_[r][c], 0.0f);
        }
    }
#pragma unroll
    for (int r = 0; r < DF_TM; ++r) {
        const long long m = m0 + tm + 16 * r;
        if (m >= M) continue;
#pragma unroll
        for (int c = 0; c < DF_TQ; ++c) {
            const int q = tq * DF_TQ + c;
            if (q < Q) out[blockIdx.y * osS + m * osM + q * osQ] = (double)S[r][c] + (double)C[r][c];
        }
    }
}

template <typename E> size_t df_gemm_smem(int QP) {
    return ((DF_NBUF * DfTile<E>::ELEMS * sizeof(E) + 15) / 16) * 16 + 2 * DF_NBUF * DF_KC * (QP + 4) * sizeof(float);
}

// t[i][q] = sum_s Tpart[s][i][q] (times scale[i]^2: Phi~ = diag(scale) C for
// the FP8 form, so Phi~^T Phi~ x = C^T diag(scale^2) C x), as an FP32 pair in
// the [i][QP] layout the transposed product reads; zero for i >= N, q >= Q.
__global__ void k_df_combine_t(const double* __restrict__ Tpart, int S, long long N, long long Np, int Q, int QP,
                               const float* __restrict__ scale, float* __restrict__ thi, float* __restrict__ tlo) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Np * QP) return;
    const long long i = e / QP;
    const int q = (int)(e % QP);
    double v = 0.0;
    if (i < N && q < Q) {
        for (int s = 0; s < S; ++s) v += Tpart[(size_t)s * Np * QP + e];
        if (scale) {
            const double sc = scale[i];
            v *= sc * sc;
        }
    }
    float h, l;
    df_split(v, h, l);
    thi[e] = h;
    tlo[e] = l;
}

// Convolution dictionary, (Phi x)_i = sum_{tau < L, tau <= i} h[tau] x[i - tau],
// one thread per (i, q), FP32 pairs; t[q][i] as an FP32 pair (i < Np).
__global__ void k_df_conv(const float* __restrict__ h, int L, long long N, long long Dp,
                          const float* __restrict__ X, const float* __restrict__ Xlo, float* __restrict__ thi,
                          float* __restrict__ tlo) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (i >= Dp) return;
    float S = 0.0f, C = 0.0f;
    if (i < N) {
        const float* x = X + (size_t)q * Dp;
        const float* xl = Xlo + (size_t)q * Dp;
        const int tmax = (long long)L - 1 < i ? L - 1 : (int)i;
        for (int tau = 0; tau <= tmax; ++tau) df_mac(S, C, __ldg(h + tau), x[i - tau], xl[i - tau]);
    }
    float hh, ll;
    df_split((double)S + (double)C, hh, ll);
    thi[(size_t)q * Dp + i] = hh;
    tlo[(size_t)q * Dp + i] = ll;
}

// (Phi^T t)_j = sum_{tau < L, j + tau < N} h[tau] t[j + tau] into U[q][j] (FP64).
__global__ void k_df_conv_t(const float* __restrict__ h, int L, long long N, long long Dp,
                            const float* __restrict__ thi, const float* __restrict__ tlo, double* __restrict__ U) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= Dp) return;
    float S = 0.0f, C = 0.0f;
    if (j < N) {
        const float* th = thi + (size_t)q * Dp;
        const float* tl = tlo + (size_t)q * Dp;
        const long long rem = N - 1 - j;
        const int tmax = (long long)L - 1 < rem ? L - 1 : (int)rem;
        for (int tau = 0; tau <= tmax; ++tau) df_mac(S, C, __ldg(h + tau), th[j + tau], tl[j + tau]);
    }
    U[(size_t)q * Dp + j] = j < N ? (double)S + (double)C : 0.0;
}

// R = B - beta U - alpha (X + Xlo) in FP64 for column q (block (ch, q)), with
// U = sum_s Upart[s][q][j].  mode DF_RR (residual replacement): active columns
// take R, and the partials of ||r||^2 and r^T M^-1 r go where the direction
// kernel reads the update's (slabs 0 and 1).  mode DF_CHECK: every column's
// true residual goes to Rt and the partials of ||r||^2 to slab 0.
__global__ __launch_bounds__(NT) void k_df_residual(DevCtl* ctl, int mode, const float* __restrict__ b,
                                                    const float* __restrict__ X, const float* __restrict__ Xlo,
                                                    const double* __restrict__ Upart, int S, size_t sstride,
                                                    const float* __restrict__ alpha, const float* __restrict__ minv,
                                                    float* __restrict__ Rout, long long D, long long Dp, int nch,
                                                    double* part) {
    __shared__ double sh[NT / 32];
    const int q = blockIdx.y, ch = blockIdx.x, Q = ctl->Q;
    const bool on = mode == DF_CHECK ? ctl->bnorm2[q] > 0.0 : ctl->active[q] != 0;
    const double beta = ctl->beta;
    double rr = 0.0, rz = 0.0;
    if (on) {
        const size_t off = (size_t)q * Dp;
        for (int e = threadIdx.x; e < CH; e += NT) {
            const long long j = (long long)ch * CH + e;
            if (j >= Dp) break;
            double r = 0.0;   // padding beyond D stays zero
            if (j < D) {
                double u = 0.0;
                for (int s = 0; s < S; ++s) u += Upart[(size_t)s * sstride + off + j];
                const double x = (double)X[off + j] + (double)Xlo[off + j];
                r = accurate_rhs(ctl, b, q, j, D, Dp) - beta * u - (double)alpha[j] * x;
            }
            Rout[off + j] = (float)r;
            rr += r * r;
            rz += r * r * (double)minv[j];
        }
    }
    rr = block_sum(rr, sh);
    rz = block_sum(rz, sh);
    if (threadIdx.x == 0) {
        part[(size_t)(0 * Q + q) * nch + ch] = rr;
        if (mode == DF_RR) part[(size_t)(1 * Q + q) * nch + ch] = rz;
    }
}

// out[q][j] = (Phi~^T Phi~ (X + Xlo))_jq = sum_s Upart[s][q][j] in FP64, j < D.
__global__ void k_df_gram_out(const double* __restrict__ Upart, int S, size_t sstride, long long D, long long Dp,
                              double* __restrict__ out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= D) return;
    double u = 0.0;
    for (int s = 0; s < S; ++s) u += Upart[(size_t)s * sstride + (size_t)q * Dp + j];
    out[(size_t)q * D + j] = u;
}

// ---------------------------------------------------------------------------
// True-residual check at the end of the CG loop (block (ch, q)).  Every block
// sums the partials of ||B - A X||^2 of its column (all columns for the
// Frobenius test) in a fixed order, so all blocks of a column take the same
// decision.  Block 0 of the column records ||r_q|| / ||b_q|| for EM iteration
// t.  With fix = 1, a column whose true residual misses the tolerance (not
// broken down, CG budget left) restarts from it: R = R_true, P = M^-1 R,
// and the last block to arrive forms rho = R^T M^-1 R, reactivates those
// columns and keeps the verification loop going.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(NT) void k_df_check(DevCtl* ctl, const float* __restrict__ Rt, float* __restrict__ R,
                                                 float* __restrict__ P, const float* __restrict__ minv,
                                                 const float* __restrict__ alpha, long long Dp, int nch,
                                                 double* part, unsigned* counter, double* res,
                                                 cudaGraphConditionalHandle h_vf, SplitOut so) {
    __shared__ double sh[NT / 32];
    __shared__ double s_rt[COFEM_QMAX];
    __shared__ int s_fail;
    const int q = blockIdx.y, ch = blockIdx.x, Q = ctl->Q;
    const int w = threadIdx.x >> 5;
    const bool frob = ctl->conv == COFEM_CONV_FROBENIUS;
    for (int k = w; k < Q; k += NT / 32) {
        if (!frob && k != q) continue;
        const double v = warp_sum_parts(part + (size_t)k * nch, nch);
        if ((threadIdx.x & 31) == 0) s_rt[k] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const double t2 = ctl->tol * ctl->tol, bn2 = ctl->bnorm2[q], rt2 = s_rt[q];
        bool pass = true;
        if (bn2 > 0.0) {
            if (frob) {
                double num = 0.0, den = 0.0;
                for (int k = 0; k < Q; ++k) {
                    if (ctl->bnorm2[k] > 0.0) num += s_rt[k];
                    den += ctl->bnorm2[k];
                }
                pass = num <= t2 * den;
            } else {
                pass = rt2 <= t2 * bn2;
            }
        }
        const bool can = ctl->fix_residual && !ctl->broken[q] && ctl->u < ctl->maxit;
        const int fail = !pass && can;
        s_fail = fail;
        if (ch == 0) {
            ctl->restart[q] = fail;
            ctl->rt2[q] = rt2;
            if (res) res[(size_t)(ctl->t - 1) * COFEM_QMAX + q] = bn2 > 0.0 ? sqrt(rt2 / bn2) : 0.0;
            if (!pass && ctl->fix_residual && !ctl->broken[q] && !can)
                atomicOr(&ctl->flags, COFEM_FLAG_CG_NOT_CONVERGED);
        }
    }
    __syncthreads();
    float rz = 0.0f, ap = 0.0f;
    if (s_fail) {
        const size_t off = (size_t)q * Dp;
        for (int e = threadIdx.x * 4; e < CH; e += NT * 4) {
            const long long j = (long long)ch * CH + e;
            if (j >= Dp) break;
            const float4 r = *reinterpret_cast<const float4*>(Rt + off + j);
            const float4 m = *reinterpret_cast<const float4*>(minv + j);
            const float4 a = *reinterpret_cast<const float4*>(alpha + j);
            const float4 p = make_float4(r.x * m.x, r.y * m.y, r.z * m.z, r.w * m.w);
            *reinterpret_cast<float4*>(R + off + j) = r;
            *reinterpret_cast<float4*>(P + off + j) = p;
            store_split(so, q, j, p);
            rz += r.x * p.x + r.y * p.y + r.z * p.z + r.w * p.w;
            ap += a.x * p.x * p.x + a.y * p.y * p.y + a.z * p.z * p.z + a.w * p.w * p.w;
        }
    }
    const double rzd = block_sum_f(rz, sh);
    const double apd = block_sum_f(ap, sh);
    if (threadIdx.x == 0 && s_fail) {   // slab 0 (the true residuals) is still read by other blocks
        part[(size_t)(1 * Q + q) * nch + ch] = rzd;
        part[(size_t)(2 * Q + q) * nch + ch] = apd;
    }
    if (!last_block_arrive(counter, gridDim.x * gridDim.y)) return;
    int any = 0;
    for (int k = threadIdx.x; k < Q; k += blockDim.x) {
        if (!ctl->restart[k]) continue;
        double v = 0.0;
        for (int i = 0; i < nch; ++i) v += __ldcg(part + (size_t)(1 * Q + k) * nch + i);
        ctl->rho[ctl->u & 1][k] = v;   // the next update reads rho of parity u
        ctl->rnorm2[k] = ctl->rt2[k];
        ctl->active[k] = 1;
        any = 1;
    }
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) {
        ctl->n_check += 1;
        ctl->any_active = any;
        ctl->verify_again = any;
        set_cond(h_vf, any);
    }
}

// Loop gate: h_set = (some column is active and the CG budget is not spent),
// the entry condition of a CG loop (or of a run of CG steps up to a residual
// replacement); h_clear = 0.
__global__ void k_cg_gate(DevCtl* ctl, cudaGraphConditionalHandle h_set, cudaGraphConditionalHandle h_clear) {
    if (threadIdx.x == 0) {
        set_cond(h_set, ctl->any_active && ctl->u < ctl->maxit);
        set_cond(h_clear, 0);
    }
}

int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// k split of a product with M output rows and K terms (K a multiple of
// DF_KC, so every chunk is whole tiles): the split whose grid fills the
// resident block slots (`capacity` = blocks per SM x SMs) in whole waves best,
// among splits that leave at least 16 tiles per block (a partial last wave
// runs a few blocks on an otherwise idle GPU).
void df_split_k(long long M, long long K, long long capacity, int* S, long long* kchunk) {
    const long long mb = ceil_div(M, DF_BM);
    const long long tiles = ceil_div(K, DF_KC);
    const long long smax = std::max(1LL, tiles / 16);
    long long best = 1;
    double best_eff = -1.0;
    for (long long sp = 1; sp <= smax; ++sp) {
        const long long kc = ceil_div(tiles, sp) * DF_KC;          // chunk, whole tiles
        const long long nb = mb * ceil_div(K, kc);                   // blocks launched
        const long long waves = ceil_div(nb, capacity);
        const double eff = (double)nb / (double)(waves * capacity);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = sp;
        }
    }
    const long long kc = ceil_div(tiles, best) * DF_KC;
    *kchunk = kc;
    *S = (int)ceil_div(K, kc);
}

// Resident blocks per SM of the products for QP columns (the occupancy the
// k split is chosen for).
template <typename E, bool TRANS>
int df_blocks_per_sm(int QP) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_df_gemm<E, TRANS, TRANS>, 16 * (QP / DF_TQ),
                                                      df_gemm_smem<E>(QP)) != cudaSuccess) {
        (void)cudaGetLastError();
        nb = 1;
    }
    return nb > 0 ? nb : 1;
}

template <bool TRANS>
int df_blocks_per_sm_of(const cofem_ctx* c, int QP) {
    if (c->phi16) return df_blocks_per_sm<__nv_bfloat16, TRANS>(QP);
    if (c->phi8) return df_blocks_per_sm<uint8_t, TRANS>(QP);
    return df_blocks_per_sm<float, TRANS>(QP);
}

template <typename E>
void launch_df_dense(Sink& s, cofem_ctx* c, int Q, const E* phi) {
    const int QP = c->df_QP;
    const dim3 blk(16 * (QP / DF_TQ));
    const size_t smem = df_gemm_smem<E>(QP);
    // padded extents: Phi~ is Np x Dp, X is Q x Dp and t is Np x QP, all zero padded
    s.launch(k_df_gemm<E, false, false>, dim3(ceil_div(c->Np, DF_BM), c->df_S1), blk, smem, phi, c->Dp, c->Np, c->Dp,
             c->df_k1, c->X, c->Xlo, 1LL, c->Dp, Q, QP, c->df_T, c->Np * QP, (long long)QP, 1LL);
    s.launch(k_df_combine_t, dim3(ceil_div(c->Np * QP, 256)), dim3(256), 0, c->df_T, c->df_S1, c->N, c->Np, Q, QP,
             c->phi8 ? (const float*)c->scale8 : (const float*)nullptr, c->df_thi, c->df_tlo);
    s.launch(k_df_gemm<E, true, true>, dim3(ceil_div(c->Dp, DF_BM), c->df_S2), blk, smem, phi, c->Dp, c->Dp, c->Np,
             c->df_k2, c->df_thi, c->df_tlo, (long long)QP, 1LL, Q, QP, c->df_U, (long long)QP * c->Dp, 1LL, c->Dp);
}

}  // namespace

// Sizes of the accurate-residual workspace for Q columns (kernels_accurate.cu
// owns the layout): the k splits and the element counts of each buffer.
DfSizes df_configure(cofem_ctx* c, int Q) {
    DfSizes z{};
    z.QP = (Q + DF_TQ - 1) / DF_TQ * DF_TQ;
    if (c->kind == COFEM_OP_DENSE) {
        df_split_k(c->Np, c->Dp, (long long)df_blocks_per_sm_of<false>(c, z.QP) * c->num_sms, &z.S1, &z.k1);
        df_split_k(c->Dp, c->Np, (long long)df_blocks_per_sm_of<true>(c, z.QP) * c->num_sms, &z.S2, &z.k2);
        z.t = (size_t)c->Np * z.QP;
        z.T = (size_t)z.S1 * c->Np * z.QP;
        z.U = (size_t)z.S2 * z.QP * c->Dp;
    } else {
        z.S1 = z.S2 = 1;
        z.t = (size_t)z.QP * c->Dp;
        z.T = 0;
        z.U = (size_t)z.QP * c->Dp;
    }
    return z;
}

// The first product alone (Phi~ X in FP32 pairs; the dominant kernel of the
// accurate residual), for timing.
void launch_df_first_product(Sink& s, cofem_ctx* c, int Q) {
    if (c->sl) {
        launch_sl_first_product(s, c, Q);
        return;
    }
    const int QP = c->df_QP;
    const dim3 blk(16 * (QP / DF_TQ));
#define DF_FIRST(E, ptr)                                                                                         \
    s.launch(k_df_gemm<E, false, false>, dim3(ceil_div(c->Np, DF_BM), c->df_S1), blk, df_gemm_smem<E>(QP), ptr, \
             c->Dp, c->Np, c->Dp, c->df_k1, c->X, c->Xlo, 1LL, c->Dp, Q, QP, c->df_T, c->Np * QP, (long long)QP, 1LL)
    if (c->phi16) DF_FIRST(__nv_bfloat16, c->phi16);
    else if (c->phi8) DF_FIRST(uint8_t, c->phi8);
    else DF_FIRST(float, c->phi32);
#undef DF_FIRST
}

// R_out = B - A (X + Xlo) for the active columns (DF_RR, into R) or for every
// column (DF_CHECK, into Rt), with the norm partials the next kernel reads.
void launch_true_residual(Sink& s, cofem_ctx* c, int Q, int mode) {
    if (c->sl) {
        launch_sl_residual(s, c, Q, mode);
        return;
    }
    if (c->kind == COFEM_OP_DENSE) {
        if (c->phi16) launch_df_dense<__nv_bfloat16>(s, c, Q, c->phi16);
        else if (c->phi8) launch_df_dense<uint8_t>(s, c, Q, c->phi8);
        else launch_df_dense<float>(s, c, Q, c->phi32);
    } else {
        const dim3 g((unsigned)ceil_div(c->Dp, 256), Q);
        s.launch(k_df_conv, g, dim3(256), 0, c->h, c->L, c->N, c->Dp, c->X, c->Xlo, c->df_thi, c->df_tlo);
        s.launch(k_df_conv_t, g, dim3(256), 0, c->h, c->L, c->N, c->Dp, c->df_thi, c->df_tlo, c->df_U);
    }
    const size_t sstride = (size_t)c->df_QP * c->Dp;
    s.launch(k_df_residual, dim3(c->nch, Q), dim3(NT), 0, c->ctl, mode, c->b, c->X, c->Xlo, c->df_U, c->df_S2,
             sstride, c->alpha, c->minv, mode == DF_RR ? c->R : c->Rt, c->D, c->Dp, c->nch, c->part);
}

// The accurate product alone (dense dictionary): out = Phi~^T Phi~ (X + Xlo)
// in FP64, Q x D, by the handle's accurate-residual form.
void launch_df_gram(Sink& s, cofem_ctx* c, int Q, double* out) {
    if (c->sl) {
        launch_sl_gram(s, c, Q, out);
        return;
    }
    if (c->phi16) launch_df_dense<__nv_bfloat16>(s, c, Q, c->phi16);
    else if (c->phi8) launch_df_dense<uint8_t>(s, c, Q, c->phi8);
    else launch_df_dense<float>(s, c, Q, c->phi32);
    s.launch(k_df_gram_out, dim3((unsigned)ceil_div(c->D, 256), Q), dim3(256), 0, c->df_U, c->df_S2,
             (size_t)c->df_QP * c->Dp, c->D, c->Dp, out);
}

cudaError_t df_kernel_attributes() {
    const int QPmax = COFEM_QMAX;
    cudaError_t e;
#define DF_ATTR(E, TR)                                                                                       \
    if ((e = cudaFuncSetAttribute(k_df_gemm<E, TR, TR>, cudaFuncAttributeMaxDynamicSharedMemorySize,         \
                                  (int)df_gemm_smem<E>(QPmax))) != cudaSuccess)                             \
        return e;
    DF_ATTR(float, false) DF_ATTR(float, true) DF_ATTR(__nv_bfloat16, false) DF_ATTR(__nv_bfloat16, true)
    DF_ATTR(uint8_t, false) DF_ATTR(uint8_t, true)
#undef DF_ATTR
    return cudaSuccess;
}

int true_residual_kernels(cofem_ctx* c) {
    if (c->sl) return sl_kernels();
    return c->kind == COFEM_OP_DENSE ? 4 : (c->kind == COFEM_OP_TOEPLITZ ? 3 : 0);   // not built for the DCT
}

void launch_df_check(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_vf) {
    s.launch(k_df_check, dim3(c->nch, Q), dim3(NT), 0, c->ctl, c->Rt, c->R, c->P, c->minv, c->alpha, c->Dp, c->nch,
             c->part, c->counters + 12, c->res_dev, h_vf, tc_direction_split(c));
}

void launch_cg_gate(Sink& s, cofem_ctx* c, cudaGraphConditionalHandle h_set, cudaGraphConditionalHandle h_clear) {
    s.launch(k_cg_gate, dim3(1), dim3(32), 0, c->ctl, h_set, h_clear);
}
