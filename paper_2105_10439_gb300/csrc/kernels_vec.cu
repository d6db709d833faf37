// Vector kernels of the CoFEM hot path: PCG initialisation, the fused CG
// update (with pi and gamma; X as an exact FP32 pair in the precision form),
// the per-column stopping test with the direction update, and the fused
// diagonal-estimate + M-step.  (The accurate residual of the precision form is
// in kernels_accurate.cu.)
//
// Layout: each of X, R, P is Q columns of Dp floats ("column q" of Alg. 2 is
// the contiguous run [q*Dp, q*Dp + D)); padding entries are kept at zero.
// Vector kernels run on a (chunk, q) grid: block (ch, q) owns elements
// [ch*CH, ch*CH + CH) of column q, so the per-column reductions of Alg. 2 are
// one partial per block, summed in block order either by the last block to
// arrive (initialisation, M-step) or, inside the CG loop, by every block of
// the next kernel for its own column.
#include "cofem_internal.cuh"

namespace {

constexpr int CH = COFEM_VEC_CHUNK;
constexpr int NT = COFEM_VEC_THREADS;
constexpr int IT = CH / (NT * 4);   // float4 positions per thread in a chunk
static_assert(CH % (NT * 4) == 0, "a chunk is a whole number of float4 sweeps of the block");

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// x + lo += d with x = fl(x + d) and the rounding error of that sum added to lo
// (Knuth's TwoSum; the _rn intrinsics keep the compiler from fusing it).
__device__ __forceinline__ void two_sum_acc(float& x, float& lo, float d) {
    const float s = __fadd_rn(x, d);
    const float z = __fsub_rn(s, x);
    const float e = __fadd_rn(__fsub_rn(x, __fsub_rn(s, z)), __fsub_rn(d, z));
    x = s;
    lo = __fadd_rn(lo, e);
}

// Sum the per-block partials part[(k*Q + q)*nch + ch] over ch for k < nk,
// into out[k*COFEM_QMAX + q] (shared).  One warp per (k, q).
__device__ void reduce_parts(const double* part, int nk, int Q, int nch, double* out) {
    // one (slab, column) per thread: its nch partials are independent loads,
    // issued together, then added in order (one L2 round trip, fixed order)
    for (int kq = threadIdx.x; kq < nk * Q; kq += blockDim.x) {
        const int k = kq / Q, q = kq % Q;
        const double* src = part + (size_t)(k * Q + q) * nch;
        double v = 0.0;
        int i = 0;
        for (; i + 8 <= nch; i += 8) {
            double x[8];
#pragma unroll
            for (int t = 0; t < 8; ++t) x[t] = __ldcg(src + i + t);
#pragma unroll
            for (int t = 0; t < 8; ++t) v += x[t];
        }
        for (; i < nch; ++i) v += __ldcg(src + i);
        out[k * COFEM_QMAX + q] = v;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Fit set-up: M^-1 = 1 / (beta theta + alpha); t = 1.
// ---------------------------------------------------------------------------
__global__ void k_fit_setup(DevCtl* ctl, const float* __restrict__ theta, const float* __restrict__ alpha,
                            float* __restrict__ minv, long long D, long long Dp) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float beta = (float)ctl->beta;
    if (j < Dp) minv[j] = j < D ? (ctl->precond_none ? 1.0f : 1.0f / (beta * theta[j] + alpha[j])) : 0.0f;
    if (j == 0) {
        ctl->t = 1;
        ctl->u = 0;
        ctl->flags = 0u;
        ctl->n_rr = 0;
        ctl->n_check = 0;
    }
}

// ---------------------------------------------------------------------------
// PCG initialisation (Alg. 2 "Initialize", PCG reading: P_0 = W_0 = M^-1 B):
// B column 0 = b = beta Phi^T y, columns q >= 1 = probe p_q of EM iteration t
// (multi-task: the columns of task l are b_l and its probes).
// X = 0, R = B, P = M^-1 B; rho_q = B^T M^-1 B, ||b_q||^2, p^T diag(alpha) p.
// h_cg is the condition of the loop that follows: the CG loop, or in the
// precision form the verification loop around it.
// ---------------------------------------------------------------------------
// Block (ch, q) of one handle's grid; `total` = blocks of that grid (the
// last-block reduction).  The last block also records the phase a packed
// serving step reads (PH_CG: the CG loop runs; PH_START: it is not entered).
__device__ __forceinline__ void cg_init_body(DevCtl* ctl, const float* __restrict__ b,
                                             const float* __restrict__ minv, const float* __restrict__ alpha,
                                             float* __restrict__ X, float* __restrict__ R, float* __restrict__ P,
                                             float* __restrict__ Xlo, long long D, long long Dp, int nch,
                                             double* part, unsigned* counter, cudaGraphConditionalHandle h_cg,
                                             const SplitOut& so, const OpOut& uo, int q, int ch, unsigned total) {
    __shared__ double sh[NT / 32];
    __shared__ double red[3 * COFEM_QMAX];
    const int Q = ctl->Q, t = ctl->t;
    const int tp = ctl->warm ? 1 : t;           // probe reuse draws the probes of t = 1
    const bool warm = ctl->warm && t > 1;       // start from the previous E-step's X
    const float beta = (float)ctl->beta;
    const unsigned long long seed = ctl->seed;
    float bb = 0.0f, rz = 0.0f, ap = 0.0f;
    const size_t off = (size_t)q * Dp;
    for (int e = threadIdx.x * 4; e < CH; e += NT * 4) {
        const long long j = (long long)ch * CH + e;
        if (j >= Dp) break;
        float4 bv;
        int task, k;
        column_task(ctl, q, task, k);
        if (k == 0) {
            bv = ld4(b + (size_t)task * Dp + j);
        } else {
            const uint64_t w = probe_word(seed, tp, k, j, task);   // j..j+3 share one 64-bit word
            bv.x = j + 0 < D ? probe_sign_from_word(w, j + 0) : 0.0f;
            bv.y = j + 1 < D ? probe_sign_from_word(w, j + 1) : 0.0f;
            bv.z = j + 2 < D ? probe_sign_from_word(w, j + 2) : 0.0f;
            bv.w = j + 3 < D ? probe_sign_from_word(w, j + 3) : 0.0f;
        }
        const float4 mv = ld4(minv + j), av = ld4(alpha + j);
        float4 rv = bv;
        if (warm) {   // R = B - A X with A X = beta Phi^T Phi X + alpha X from the operator
            int s0, ns;
            op_range(uo, j, s0, ns);
            const float4 u = op_sum4(uo, Q, q, Dp, j, s0, ns);
            const float4 xv = ld4(X + off + j);
            const float bu = beta * uo.uscale;
            rv = make_float4(bv.x - (bu * u.x + av.x * xv.x), bv.y - (bu * u.y + av.y * xv.y),
                             bv.z - (bu * u.z + av.z * xv.z), bv.w - (bu * u.w + av.w * xv.w));
        } else {
            st4(X + off + j, make_float4(0.f, 0.f, 0.f, 0.f));
            if (Xlo) st4(Xlo + off + j, make_float4(0.f, 0.f, 0.f, 0.f));
        }
        const float4 wv = make_float4(rv.x * mv.x, rv.y * mv.y, rv.z * mv.z, rv.w * mv.w);
        st4(R + off + j, rv);
        st4(P + off + j, wv);
        store_split(so, q, j, wv);
        bb += bv.x * bv.x + bv.y * bv.y + bv.z * bv.z + bv.w * bv.w;
        rz += rv.x * wv.x + rv.y * wv.y + rv.z * wv.z + rv.w * wv.w;
        ap += av.x * wv.x * wv.x + av.y * wv.y * wv.y + av.z * wv.z * wv.z + av.w * wv.w * wv.w;
    }
    const double bbd = block_sum_f(bb, sh);
    const double rzd = block_sum_f(rz, sh);
    const double apd = block_sum_f(ap, sh);
    if (threadIdx.x == 0) {
        part[(size_t)(0 * Q + q) * nch + ch] = bbd;
        part[(size_t)(1 * Q + q) * nch + ch] = rzd;
        part[(size_t)(2 * Q + q) * nch + ch] = apd;
    }
    if (!last_block_arrive(counter, total)) return;
    reduce_parts(part, 3, Q, nch, red);
    const int qq = threadIdx.x;
    int act = 0;
    if (qq < Q) {
        ctl->bnorm2[qq] = red[qq];
        ctl->rho[0][qq] = red[COFEM_QMAX + qq];
        ctl->ap[qq] = red[2 * COFEM_QMAX + qq];
        ctl->rnorm2[qq] = red[qq];   // (the warm start's first stopping test reads the update's)
        act = red[qq] > 0.0;   // a zero right-hand side starts converged (x = 0)
        ctl->active[qq] = act;
        ctl->broken[qq] = 0;
    }
    act = __syncthreads_or(act);
    if (threadIdx.x == 0) {
        ctl->u = 0;
        ctl->any_active = act;
        ctl->phase = act && ctl->maxit > 0 ? PH_CG : PH_START;
        set_cond(h_cg, act && ctl->maxit > 0);
    }
}

__global__ __launch_bounds__(NT) void k_cg_init(DevCtl* ctl, const float* __restrict__ b,
                                                const float* __restrict__ minv, const float* __restrict__ alpha,
                                                float* __restrict__ X, float* __restrict__ R, float* __restrict__ P,
                                                float* __restrict__ Xlo, long long D, long long Dp, int nch,
                                                double* part, unsigned* counter, cudaGraphConditionalHandle h_cg,
                                                SplitOut so, OpOut uo) {
    cg_init_body(ctl, b, minv, alpha, X, R, P, Xlo, D, Dp, nch, part, counter, h_cg, so, uo, blockIdx.y, blockIdx.x,
                 gridDim.x * gridDim.y);
}

// ---------------------------------------------------------------------------
// Fused CG update (Alg. 2: X += P Gamma, R -= Psi Gamma, and the per-block
// partials of ||r||^2 and r^T M^-1 r), for the active columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cg_update_body(DevCtl* ctl, const float* __restrict__ P, const OpOut& uo,
                                               const float* __restrict__ alpha, const float* __restrict__ minv,
                                               float* __restrict__ X, float* __restrict__ R,
                                               float* __restrict__ Xlo, long long Dp, int nch, double* part,
                                               cudaGraphConditionalHandle h_rr, cudaGraphConditionalHandle h_cg,
                                               int q, int ch) {
    __shared__ double sh[NT / 32];
    __shared__ double s_sum[2];
    __shared__ int s_act;
    __shared__ float s_gamma;
    const int Q = ctl->Q;
    const int u = ctl->u;   // this CG iteration (counted by the operator)
    if (ch == 0 && q == 0 && threadIdx.x == 0) {
        // the stopping test and the loop condition are the direction kernel's
        // (it reads this kernel's partials)
        ctl->any_active = 0;
        const bool rr = ctl->rr_period > 0 && u % ctl->rr_period == 0;
        ctl->n_rr += rr;
        set_cond(h_rr, rr);
        set_cond(h_cg, 0);
    }
    // all loads of the thread's IT float4 positions first (the kernel is bound
    // by memory round trips, not bandwidth); then the partial sums of the
    // operator, then the arithmetic in element order
    const size_t off = (size_t)q * Dp;
    float4 pv[IT], av[IT], mv[IT], xv[IT], rv[IT], uv[IT];
    int s0[IT], ns[IT];
    if (ctl->active[q]) {
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
            if (j < Dp) {
                pv[it] = ld4(P + off + j);
                av[it] = ld4(alpha + j);
                mv[it] = ld4(minv + j);
                xv[it] = ld4(X + off + j);
                rv[it] = ld4(R + off + j);
                op_range(uo, j, s0[it], ns[it]);
            }
        }
    }
    // pi_q = beta ||Phi p_q||^2 + p^T diag(alpha) p and gamma_q = rho_q / pi_q
    // (Alg. 2) from the operator's and the direction kernel's partials (warps 0
    // and 1, in a fixed order): every block of the column gets the same value;
    // block 0 records it.  pi_q <= 0 or non-finite freezes the column (breakdown).
    if (threadIdx.x < 64) {
        const double v = threadIdx.x < 32 ? warp_sum_parts(ctl->tt_part + (size_t)q * ctl->tt_n, ctl->tt_n)
                                          : warp_sum_parts(ctl->ap_part + (size_t)q * ctl->ap_n, ctl->ap_n);
        if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int act = ctl->active[q];
        float gamma = 0.0f;
        if (act) {
            const double tt = s_sum[0], ap = s_sum[1];
            const double pi = ctl->beta * tt + ap;
            const bool ok = pi > 0.0 && isfinite(pi);
            const double g = ok ? ctl->rho[(u - 1) & 1][q] / pi : 0.0;
            act = ok;
            gamma = (float)g;
            if (ch == 0) {
                ctl->tt[q] = tt;
                ctl->ap[q] = ap;
                ctl->pi[q] = pi;
                ctl->gamma[q] = g;
                if (!ok) {
                    atomicOr(&ctl->flags, COFEM_FLAG_BREAKDOWN);
                    ctl->active[q] = 0;
                    ctl->broken[q] = 1;
                }
            }
        }
        s_act = act;
        s_gamma = gamma;
    }
    __syncthreads();
    float rr = 0.0f, rz = 0.0f;
    if (s_act) {   // (implies the loads above were issued)
        const float gamma = s_gamma;
        const float beta = (float)ctl->beta;
        if (Xlo) {   // precision form: X + Xlo += gamma p, the rounding error of X kept in Xlo (TwoSum)
#pragma unroll
            for (int it = 0; it < IT; ++it) {
                const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
                if (j < Dp) {
                    float4 x4 = xv[it], l4 = ld4(Xlo + off + j);
                    const float4 p4 = pv[it];
                    two_sum_acc(x4.x, l4.x, __fmul_rn(gamma, p4.x));
                    two_sum_acc(x4.y, l4.y, __fmul_rn(gamma, p4.y));
                    two_sum_acc(x4.z, l4.z, __fmul_rn(gamma, p4.z));
                    two_sum_acc(x4.w, l4.w, __fmul_rn(gamma, p4.w));
                    st4(X + off + j, x4);
                    st4(Xlo + off + j, l4);
                }
            }
        } else {
#pragma unroll
            for (int it = 0; it < IT; ++it) {   // X needs no operator output: store it now
                const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
                if (j < Dp) {
                    float4 x4 = xv[it];
                    const float4 p4 = pv[it];
                    x4.x += gamma * p4.x; x4.y += gamma * p4.y; x4.z += gamma * p4.z; x4.w += gamma * p4.w;
                    st4(X + off + j, x4);
                }
            }
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
            if (j < Dp) uv[it] = op_sum4(uo, Q, q, Dp, j, s0[it], ns[it]);
        }
        const float bu = beta * uo.uscale;
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
            if (j >= Dp) break;
            const float4 p4 = pv[it], a4 = av[it], m4 = mv[it], u4 = uv[it];
            const float4 psi = make_float4(bu * u4.x + a4.x * p4.x, bu * u4.y + a4.y * p4.y,
                                           bu * u4.z + a4.z * p4.z, bu * u4.w + a4.w * p4.w);
            float4 r4 = rv[it];
            r4.x -= gamma * psi.x; r4.y -= gamma * psi.y; r4.z -= gamma * psi.z; r4.w -= gamma * psi.w;
            st4(R + off + j, r4);
            rr += r4.x * r4.x + r4.y * r4.y + r4.z * r4.z + r4.w * r4.w;
            rz += r4.x * (r4.x * m4.x) + r4.y * (r4.y * m4.y) + r4.z * (r4.z * m4.z) + r4.w * (r4.w * m4.w);
        }
    }
    const double rrd = block_sum_f(rr, sh);
    const double rzd = block_sum_f(rz, sh);
    if (threadIdx.x == 0) {
        part[(size_t)(0 * Q + q) * nch + ch] = rrd;
        part[(size_t)(1 * Q + q) * nch + ch] = rzd;
    }
}

__global__ __launch_bounds__(NT, 2) void k_cg_update(DevCtl* ctl, const float* __restrict__ P, OpOut uo,
                                                  const float* __restrict__ alpha,
                                                  const float* __restrict__ minv, float* __restrict__ X,
                                                  float* __restrict__ R, float* __restrict__ Xlo, long long Dp,
                                                  int nch, double* part, cudaGraphConditionalHandle h_rr,
                                                  cudaGraphConditionalHandle h_cg) {
    griddep_launch();
    griddep_wait();   // the operator's output and partials come from the previous kernels
    cg_update_body(ctl, P, uo, alpha, minv, X, R, Xlo, Dp, nch, part, h_rr, h_cg, blockIdx.y, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Stopping test and direction update (Alg. 2, PCG reading: W = M^-1 R,
// P = W + P H) for the active columns, plus the partials of p^T diag(alpha) p
// for the next pi, and the CG loop condition.  Every block sums the update's
// (or the residual replacement's) partials of its column itself, in block
// order, so all blocks of a column take the same decision without a grid-wide
// hand-off; block 0 of each column records it.  Per column:
// ||r_q||^2 <= tol^2 ||b_q||^2 ends column q (per-column test), or
// sum_q ||r_q||^2 <= tol^2 sum_q ||b_q||^2 ends all of them (Frobenius test);
// otherwise eta_q = rho_new / rho_old.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cg_direction_body(DevCtl* ctl, const float* __restrict__ R,
                                                  const float* __restrict__ alpha, const float* __restrict__ minv,
                                                  float* __restrict__ P, long long Dp, int nch, double* part,
                                                  cudaGraphConditionalHandle h_cg, const SplitOut& so, int q,
                                                  int ch, int defer_rr) {
    // deferred (a fit graph's CG loop): at a replacement step the loop ends
    // here and the direction runs after the replacement, outside the loop
    if (defer_rr && rr_step(ctl)) return;
    __shared__ double sh[NT / 32];
    __shared__ double s_rr[COFEM_QMAX];
    __shared__ double s_sum[2];
    __shared__ int s_act;
    __shared__ float s_eta;
    const int Q = ctl->Q;
    const int u = ctl->u;
    // a column that left the loop stays out; block 0 of this column may already
    // have recorded this iteration's decision, which gives the same result
    const int prev = ctl->active[q];
    const double t2 = ctl->tol * ctl->tol;
    const bool frob = ctl->conv == COFEM_CONV_FROBENIUS;
    // the update's (or replacement's) partials of column q, one warp each, in a
    // fixed order (every block of the column gets the same bits); the Frobenius
    // test needs ||r_k||^2 of every column
    const int w = threadIdx.x >> 5;
    if (frob) {
        for (int k = w; k < Q; k += NT / 32) {
            const double v = warp_sum_parts(part + (size_t)k * nch, nch);
            if ((threadIdx.x & 31) == 0) s_rr[k] = v;
        }
        if (w == NT / 32 - 1) {
            const double v = warp_sum_parts(part + (size_t)(Q + q) * nch, nch);
            if ((threadIdx.x & 31) == 0) s_sum[1] = v;
        }
    } else if (w < 2) {
        const double v = warp_sum_parts(part + (size_t)(w * Q + q) * nch, nch);
        if ((threadIdx.x & 31) == 0) s_sum[w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int act = 0;
        float eta = 0.0f;
        double rr = 0.0, rz = 0.0;
        if (prev) {
            rr = frob ? s_rr[q] : s_sum[0];
            rz = s_sum[1];
            bool stop;
            if (frob) {
                double num = 0.0, den = 0.0;
                for (int k = 0; k < Q; ++k) {
                    if (ctl->active[k]) num += s_rr[k];
                    den += ctl->bnorm2[k];
                }
                stop = num <= t2 * den;
            } else {
                stop = rr <= t2 * ctl->bnorm2[q];
            }
            act = !stop;
            if (act) eta = (float)(rz / ctl->rho[(u - 1) & 1][q]);
        }
        s_act = act;
        s_eta = eta;
        if (ch == 0 && prev) {
            ctl->rnorm2[q] = rr;
            ctl->active[q] = act;
            if (act) {
                ctl->eta[q] = rz / ctl->rho[(u - 1) & 1][q];
                ctl->rho[u & 1][q] = rz;
                ctl->any_active = 1;
                if (u < ctl->maxit) set_cond(h_cg, 1);
                else atomicOr(&ctl->flags, COFEM_FLAG_CG_NOT_CONVERGED);
            }
        }
    }
    __syncthreads();
    const int act = s_act;
    const size_t off = (size_t)q * Dp;
    float ap = 0.0f;
    if (act) {
        const float eta = s_eta;
        float4 rv[IT], mv[IT], av[IT], pv[IT];   // loads first (see k_cg_update)
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
            if (j < Dp) {
                rv[it] = ld4(R + off + j);
                mv[it] = ld4(minv + j);
                av[it] = ld4(alpha + j);
                pv[it] = ld4(P + off + j);
            }
        }
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const long long j = (long long)ch * CH + (long long)(threadIdx.x + it * NT) * 4;
            if (j >= Dp) break;
            float4 p4 = pv[it];
            const float4 r4 = rv[it], m4 = mv[it], a4 = av[it];
            p4.x = r4.x * m4.x + eta * p4.x;
            p4.y = r4.y * m4.y + eta * p4.y;
            p4.z = r4.z * m4.z + eta * p4.z;
            p4.w = r4.w * m4.w + eta * p4.w;
            st4(P + off + j, p4);
            store_split(so, q, j, p4);
            ap += a4.x * p4.x * p4.x + a4.y * p4.y * p4.y + a4.z * p4.z * p4.z + a4.w * p4.w * p4.w;
        }
    }
    const double apd = block_sum_f(ap, sh);
    if (threadIdx.x == 0) part[(size_t)(2 * Q + q) * nch + ch] = apd;   // reduced by the operator's finish
}

__global__ __launch_bounds__(NT) void k_cg_direction(DevCtl* ctl, const float* __restrict__ R,
                                                     const float* __restrict__ alpha,
                                                     const float* __restrict__ minv, float* __restrict__ P,
                                                     long long Dp, int nch, double* part,
                                                     cudaGraphConditionalHandle h_cg, SplitOut so, int defer_rr) {
    griddep_launch();
    griddep_wait();   // R and the partials come from the previous kernel
    cg_direction_body(ctl, R, alpha, minv, P, Dp, nch, part, h_cg, so, blockIdx.y, blockIdx.x, defer_rr);
}

// ---------------------------------------------------------------------------
// Fused diagonal estimate + M-step (Alg. 1: s_j = (1/K) sum_k p_kj x_kj; if t < T,
// alpha_j = 1 / max(E[z_j^2], 1/alpha_max) with E[z_j^2] = mu_j^2 + s_j, or under
// the rectified Gaussian prior the second moment of N(mu_j, s_j) restricted to
// z_j >= 0 (non-negativity subsection of Sec. III); then M^-1 for the next
// E-step), probes regenerated from Philox, plus EM loop bookkeeping.
// ---------------------------------------------------------------------------
// Block jb of one handle's grid of `total` blocks (blockDim.x elements each);
// the last block also records the phase of a packed serving step (PH_INIT:
// another E-step follows; PH_DONE: the fit is complete).
__device__ __forceinline__ void mstep_body(DevCtl* ctl, const float* __restrict__ X, const float* __restrict__ theta,
                                           float* __restrict__ alpha, float* __restrict__ minv,
                                           float* __restrict__ mu_out, float* __restrict__ s_out,
                                           int* __restrict__ iters, const float* __restrict__ Xlo, long long D,
                                           long long Dp, unsigned* counter, cudaGraphConditionalHandle h_em,
                                           int jb, unsigned total) {
    const int t = ctl->t, T = ctl->T, K = ctl->K, L = ctl->L;
    const long long j = (long long)jb * blockDim.x + threadIdx.x;
    int clamped = 0;
    if (j < Dp) {
        // per task l: mu_l = x_{l(K+1)}, s_l = (1/K) sum_k p_{l,k} x_{l(K+1)+k}; the
        // second moment is mu^2 + s (one task) or its mean over the tasks
        // (multi-task M-step alpha_j = L / sum_l (mu_lj^2 + s_lj))
        float m2 = 0.0f, mu = 0.0f, s = 0.0f;
        for (int l = 0; l < L; ++l) {
            const size_t c0 = (size_t)l * (K + 1) * Dp + j;
            mu = Xlo ? X[c0] + Xlo[c0] : X[c0];   // the FP32 pair X + Xlo of the precision form
            s = 0.0f;
            if (j < D) {
                const unsigned long long seed = ctl->seed;
                for (int k = 1; k <= K; ++k) {
                    const uint64_t w = probe_word(seed, ctl->warm ? 1 : t, k, j, l);
                    const size_t e = c0 + (size_t)k * Dp;
                    s = fmaf(probe_sign_from_word(w, j), Xlo ? X[e] + Xlo[e] : X[e], s);
                }
                s /= (float)K;
            }
            mu_out[(size_t)l * Dp + j] = mu;
            s_out[(size_t)l * Dp + j] = s;
            m2 += fmaf(mu, mu, s);
        }
        if (L > 1) m2 /= (float)L;
        if (t < T && j < D) {
            if (L == 1 && ctl->prior == COFEM_PRIOR_RECTIFIED && s > 0.0f) {
                // mu^2 + s + mu sqrt(2 s / pi) exp(-xi^2) / erfc(-xi), xi = mu / sqrt(2 s);
                // exp(-xi^2) / erfc(-xi) = 1 / erfcx(-xi).  FP64: for mu << -sqrt(s)
                // the moment is a small difference of large terms.
                const double md = mu, sd = s;
                const double xi = md / sqrt(2.0 * sd);
                const double pi_ = 3.14159265358979323846;
                m2 = (float)(md * md + sd + md * sqrt(2.0 * sd / pi_) / erfcx(-xi));
            }
            const float floor_ = (float)(1.0 / ctl->alpha_max);
            clamped = m2 < floor_;
            const float a = 1.0f / (m2 > floor_ ? m2 : floor_);
            alpha[j] = a;
            minv[j] = ctl->precond_none ? 1.0f : 1.0f / ((float)ctl->beta * theta[j] + a);
        }
    }
    if (__syncthreads_or(clamped) && threadIdx.x == 0) atomicOr(&ctl->flags, COFEM_FLAG_ALPHA_CLAMPED);
    if (!last_block_arrive(counter, total)) return;
    if (threadIdx.x == 0) {
        iters[t - 1] = ctl->u;
        ctl->t = t + 1;
        ctl->phase = t + 1 <= T ? PH_INIT : PH_DONE;
        set_cond(h_em, t + 1 <= T);
    }
}

__global__ __launch_bounds__(NT) void k_mstep(DevCtl* ctl, const float* __restrict__ X,
                                              const float* __restrict__ theta, float* __restrict__ alpha,
                                              float* __restrict__ minv, float* __restrict__ mu_out,
                                              float* __restrict__ s_out, int* __restrict__ iters,
                                              const float* __restrict__ Xlo, long long D, long long Dp,
                                              unsigned* counter, cudaGraphConditionalHandle h_em) {
    mstep_body(ctl, X, theta, alpha, minv, mu_out, s_out, iters, Xlo, D, Dp, counter, h_em, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// Packed serving: the same kernels over the fits of one step, block b of a
// launch being map[b] = (fit, column, chunk) or (fit, element block, blocks
// of that fit's grid).  A fit takes part only in the phase its kernel is for.
// ---------------------------------------------------------------------------
__global__ __launch_bounds__(NT, 2) void k_cg_update_packed(const VSlot* __restrict__ vs, const int4* __restrict__ map,
                                                            const int* __restrict__ count) {
    griddep_launch();
    if ((int)blockIdx.x >= *count) return;   // the grid is sized for the server's capacity
    griddep_wait();
    const int4 m = map[blockIdx.x];
    const VSlot& f = vs[m.x];
    DevCtl* ctl = f.ctl;
    if (ctl->phase != PH_CG) return;
    const OpOut uo = f.uo;
    cg_update_body(ctl, f.P, uo, f.alpha, f.minv, f.X, f.R, nullptr, f.Dp, f.nch, f.part, 0, 0, m.y, m.z);
}

__global__ __launch_bounds__(NT) void k_cg_direction_packed(const VSlot* __restrict__ vs, const int4* __restrict__ map,
                                                            const int* __restrict__ count) {
    griddep_launch();
    if ((int)blockIdx.x >= *count) return;   // the grid is sized for the server's capacity
    griddep_wait();
    const int4 m = map[blockIdx.x];
    const VSlot& f = vs[m.x];
    DevCtl* ctl = f.ctl;
    if (ctl->phase != PH_CG) return;
    const SplitOut so = f.so;
    cg_direction_body(ctl, f.R, f.alpha, f.minv, f.P, f.Dp, f.nch, f.part, 0, so, m.y, m.z, 0);
}

// The M-step of the fits whose CG loop ended in this step (the direction
// kernel continued no column, or the budget is spent) or was never entered.
__global__ __launch_bounds__(NT) void k_mstep_packed(const VSlot* __restrict__ vs, const int4* __restrict__ map,
                                                     const int* __restrict__ count) {
    if ((int)blockIdx.x >= *count) return;
    const int4 m = map[blockIdx.x];
    const VSlot& f = vs[m.x];
    DevCtl* ctl = f.ctl;
    const int ph = ctl->phase;
    const bool go = ph == PH_START || (ph == PH_CG && !(ctl->any_active && ctl->u < ctl->maxit));
    if (!go) return;
    mstep_body(ctl, f.X, f.theta, f.alpha, f.minv, f.mu_out, f.s_out, f.iters, nullptr, f.D, f.Dp, f.counters + 4,
               0, m.y, (unsigned)m.z);
}

// The initialisation of the next E-step of the fits the M-step left in PH_INIT.
__global__ __launch_bounds__(NT) void k_cg_init_packed(const VSlot* __restrict__ vs, const int4* __restrict__ map,
                                                       const int* __restrict__ count) {
    if ((int)blockIdx.x >= *count) return;
    const int4 m = map[blockIdx.x];
    const VSlot& f = vs[m.x];
    DevCtl* ctl = f.ctl;
    if (ctl->phase != PH_INIT) return;
    const SplitOut so = f.so;
    const OpOut uo = f.uo;
    cg_init_body(ctl, f.b, f.minv, f.alpha, f.X, f.R, f.P, nullptr, f.D, f.Dp, f.nch, f.part, f.counters + 0, 0, so,
                 uo, m.y, m.z, (unsigned)m.w);
}

// End of a packed step: status[i] = phase of fit i; the step loop goes on
// (h_loop) unless a fit reached PH_DONE in this step, the host flagged new
// fits to admit (*pending), or max_steps steps have run in this launch.
__global__ void k_packed_status(const VSlot* __restrict__ vs, const int* __restrict__ nfits, int* status,
                                const volatile int* pending, unsigned* steps, unsigned max_steps,
                                cudaGraphConditionalHandle h_loop) {
    __shared__ int s_done;
    if (threadIdx.x == 0) s_done = 0;
    __syncthreads();
    const int n = *nfits;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ph = vs[i].ctl->phase;
        if (ph == PH_DONE && status[i] != PH_DONE) s_done = 1;
        status[i] = ph;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned k = *steps + 1;
        *steps = k;
        set_cond(h_loop, !s_done && *pending == 0 && k < max_steps);
    }
}

// Probe block for the step-level entry point: out[k-1][j] = p_{t,k,j}.
__global__ void k_probe_fill(unsigned long long seed, int t, int K, long long D, long long ld, float* out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y + 1;
    if (j >= D || k > K) return;
    out[(size_t)(k - 1) * ld + j] = probe_sign_from_word(probe_word(seed, t, k, j), j);
}

// Psi = beta U + alpha V for the step-level operator entry point.
__global__ void k_plain_psi(const float* __restrict__ U, int S2, size_t sstride, const float* __restrict__ V,
                            const float* __restrict__ alpha, float beta, float* __restrict__ Psi, long long D,
                            long long Dp) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= D) return;
    float u = 0.0f;
    for (int s = 0; s < S2; ++s) u += U[(size_t)s * sstride + (size_t)q * Dp + j];
    Psi[(size_t)q * D + j] = beta * u + alpha[j] * V[(size_t)q * Dp + j];
}

// dst (rows_dst x ld_dst, bf16) = round-to-nearest-even(src) inside rows x cols, zero outside.
__global__ void k_quantize_bf16(const float* __restrict__ src, long long rows, long long cols, long long ld_src,
                                __nv_bfloat16* __restrict__ dst, long long rows_dst, long long ld_dst) {
    const long long n = rows_dst * ld_dst;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / ld_dst, j = e % ld_dst;
        dst[e] = __float2bfloat16_rn(j < cols && i < rows ? src[i * ld_src + j] : 0.0f);
    }
}

// out[r] = sum_j a[r*lda + j] * b[r*ldb + j] in FP64, one block per row.
__global__ void k_dot_rows(const float* __restrict__ a, long long lda, const float* __restrict__ b, long long ldb,
                           long long n, double* out) {
    __shared__ double sh[NT / 32];
    const int r = blockIdx.x;
    double acc = 0.0;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) acc += (double)a[r * lda + j] * (double)b[r * ldb + j];
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) out[r] = acc;
}

__global__ void k_check_finite(const float* __restrict__ x, long long n, unsigned* bad) {
    int b = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        b |= !isfinite(x[i]);
    if (__syncthreads_or(b) && threadIdx.x == 0) atomicOr(bad, 1u);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
void launch_fit_setup(Sink& s, cofem_ctx* c, int /*Q*/) {
    s.launch(k_fit_setup, dim3((unsigned)((c->Dp + 255) / 256)), dim3(256), 0, c->ctl, c->theta, c->alpha, c->minv,
             c->D, c->Dp);
}

void launch_cg_init(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg) {
    s.launch(k_cg_init, dim3(c->nch, Q), dim3(NT), 0, c->ctl, c->b, c->minv, c->alpha, c->X, c->R, c->P, c->Xlo,
             c->D, c->Dp, c->nch, c->part, c->counters + 0, h_cg, tc_direction_split(c), op_output(c));
}

void launch_cg_update(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_rr,
                      cudaGraphConditionalHandle h_cg) {
    s.launch_pdl(k_cg_update, dim3(c->nch, Q), dim3(NT), 0, c->ctl, c->P, op_output(c), c->alpha, c->minv, c->X, c->R,
                 c->Xlo, c->Dp, c->nch, c->part, h_rr, h_cg);
}

void launch_cg_direction(Sink& s, cofem_ctx* c, int Q, cudaGraphConditionalHandle h_cg, bool defer_rr) {
    s.launch_pdl(k_cg_direction, dim3(c->nch, Q), dim3(NT), 0, c->ctl, c->R, c->alpha, c->minv, c->P, c->Dp, c->nch,
                 c->part, h_cg, tc_direction_split(c), defer_rr ? 1 : 0);
}

void launch_mstep(Sink& s, cofem_ctx* c, int /*Q*/, cudaGraphConditionalHandle h_em) {
    s.launch(k_mstep, dim3((unsigned)((c->Dp + NT - 1) / NT)), dim3(NT), 0, c->ctl, c->X, c->theta, c->alpha, c->minv,
             c->mu_out, c->s_out, c->iters_dev, c->Xlo, c->D, c->Dp, c->counters + 4, h_em);
}

void launch_probe_fill(cudaStream_t st, unsigned long long seed, int t, int K, long long D, long long ld,
                       float* out) {
    k_probe_fill<<<dim3((unsigned)((D + 255) / 256), K), 256, 0, st>>>(seed, t, K, D, ld, out);
}

void launch_plain_psi(cudaStream_t st, cofem_ctx* c, int Q, const float* V, const float* alpha, double beta,
                      float* Psi) {
    const int S2 = c->kind == COFEM_OP_DENSE ? c->S2 : 1;
    k_plain_psi<<<dim3((unsigned)((c->D + 255) / 256), Q), 256, 0, st>>>(
        c->U, S2, (size_t)c->Qcap * c->Dp, V, alpha, (float)beta, Psi, c->D, c->Dp);
}

void launch_quantize_bf16(cudaStream_t st, const float* src, long long rows, long long cols, long long ld_src,
                          __nv_bfloat16* dst, long long rows_dst, long long ld_dst) {
    k_quantize_bf16<<<4096, 256, 0, st>>>(src, rows, cols, ld_src, dst, rows_dst, ld_dst);
}

void launch_dot_rows(cudaStream_t st, const float* a, long long lda, const float* b, long long ldb, long long n,
                     int rows, double* out) {
    k_dot_rows<<<rows, NT, 0, st>>>(a, lda, b, ldb, n, out);
}

void launch_check_finite(cudaStream_t st, const float* x, long long n, unsigned* bad) {
    if (n <= 0) return;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    k_check_finite<<<(unsigned)blocks, 256, 0, st>>>(x, n, bad);
}

void launch_update_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks) {
    s.launch_pdl(k_cg_update_packed, dim3(nblocks), dim3(NT), 0, vs, map, count);
}

void launch_direction_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks) {
    s.launch_pdl(k_cg_direction_packed, dim3(nblocks), dim3(NT), 0, vs, map, count);
}

void launch_mstep_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks) {
    s.launch(k_mstep_packed, dim3(nblocks), dim3(NT), 0, vs, map, count);
}

void launch_init_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks) {
    s.launch(k_cg_init_packed, dim3(nblocks), dim3(NT), 0, vs, map, count);
}

void launch_packed_status(Sink& s, const VSlot* vs, const int* nfits, int* status, const volatile int* pending,
                          unsigned* steps, unsigned max_steps, cudaGraphConditionalHandle h_loop) {
    s.launch(k_packed_status, dim3(1), dim3(256), 0, vs, nfits, status, pending, steps, max_steps, h_loop);
}
