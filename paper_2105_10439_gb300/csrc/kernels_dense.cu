// Dense operator A V = beta Phi^T (Phi V) + diag(alpha) V (Alg. 2 "Apply matrix",
// Sec. III-B) for an explicit N x D dictionary, FP32 CUDA-core version.
//
//   gemm1: T = Phi V        split over D (S1 slices); the last slice of each
//                            64-row block sums the slice partials into T and the
//                            per-column ||T||^2 partials; the last row block forms
//                            pi and gamma (op_finalize_block).
//   gemm2: U_s = Phi^T T    split over N (S2 slices); U_s are the partial sums
//                            consumed by the CG update (Psi = beta sum_s U_s + alpha V).
//
// Phi is Np x Dp row-major, zero padded; V, U are column blocks of Dp floats.
#include "cofem_internal.cuh"

namespace {

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float4 ld4(const __nv_bfloat16* p) {
    const uint2 r = *reinterpret_cast<const uint2*>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ld1(const __nv_bfloat16* p) { return __bfloat162float(*p); }

constexpr int G1_BM = 64, G1_BK = 32, G1_LD = G1_BK + 4;
constexpr int G2_BI = 32;

template <int QG, typename TPhi>
__global__ __launch_bounds__(256) void k_gemm1_simt(const TPhi* __restrict__ phi, long long ldp,
                                                   const float* __restrict__ V, long long Dp, int Q,
                                                   long long chunk1, int S1, float* __restrict__ Tpart,
                                                   float* __restrict__ T, long long Np, double* tt_part, int nrb,
                                                   unsigned* cnt_rb, unsigned* cnt_all, DevCtl* ctl, int mode) {
    constexpr int QP = QG * 8;
    __shared__ __align__(16) float sA[G1_BM][G1_LD];
    __shared__ __align__(16) float sB[QP][G1_LD];
    const int rb = blockIdx.x, s = blockIdx.y, tid = threadIdx.x;
    const int rp = tid & 31, g = tid >> 5;
    const long long row0 = (long long)rb * G1_BM;
    const long long k0 = (long long)s * chunk1;
    const long long k1 = k0 + chunk1 < Dp ? k0 + chunk1 : Dp;
    float acc0[QG], acc1[QG];
#pragma unroll
    for (int i = 0; i < QG; ++i) acc0[i] = acc1[i] = 0.0f;

    for (long long kb = k0; kb < k1; kb += G1_BK) {
        for (int idx = tid; idx < G1_BM * G1_BK / 4; idx += 256) {
            const int r = idx >> 3, c4 = (idx & 7) * 4;
            *reinterpret_cast<float4*>(&sA[r][c4]) = ld4(phi + (row0 + r) * ldp + kb + c4);
        }
        for (int idx = tid; idx < QP * G1_BK / 4; idx += 256) {
            const int qq = idx >> 3, c4 = (idx & 7) * 4;
            const float4 v = qq < Q ? ld4(V + (size_t)qq * Dp + kb + c4) : make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4*>(&sB[qq][c4]) = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < G1_BK; kk += 4) {
            const float4 a0 = *reinterpret_cast<const float4*>(&sA[rp][kk]);
            const float4 a1 = *reinterpret_cast<const float4*>(&sA[rp + 32][kk]);
#pragma unroll
            for (int i = 0; i < QG; ++i) {
                const float4 bv = *reinterpret_cast<const float4*>(&sB[g * QG + i][kk]);
                acc0[i] = fmaf(a0.x, bv.x, fmaf(a0.y, bv.y, fmaf(a0.z, bv.z, fmaf(a0.w, bv.w, acc0[i]))));
                acc1[i] = fmaf(a1.x, bv.x, fmaf(a1.y, bv.y, fmaf(a1.z, bv.z, fmaf(a1.w, bv.w, acc1[i]))));
            }
        }
        __syncthreads();
    }
    float* Tp = Tpart + (size_t)s * Np * QP;
#pragma unroll
    for (int i = 0; i < QG; ++i) {
        Tp[(row0 + rp) * QP + g * QG + i] = acc0[i];
        Tp[(row0 + rp + 32) * QP + g * QG + i] = acc1[i];
    }
    if (!last_block_arrive(&cnt_rb[rb], (unsigned)S1)) return;

    // this row block's T = sum of the S1 slice partials (fixed order)
    __shared__ float sT[G1_BM][QP + 1];
    for (int e = tid; e < G1_BM * QP; e += 256) {
        const int r = e / QP, qq = e % QP;
        float v = 0.0f;
        for (int ss = 0; ss < S1; ++ss) v += __ldcg(Tpart + (size_t)ss * Np * QP + (row0 + r) * QP + qq);
        T[(row0 + r) * QP + qq] = v;
        sT[r][qq] = v;
    }
    __syncthreads();
    if (tid < Q) {   // ||T_q||^2 over this row block: FP32 runs of 8 rows, FP64 across them
        double a = 0.0;
        for (int r0 = 0; r0 < G1_BM; r0 += 8) {
            float f = 0.0f;
#pragma unroll
            for (int r = 0; r < 8; ++r) f = fmaf(sT[r0 + r][tid], sT[r0 + r][tid], f);
            a += (double)f;
        }
        tt_part[(size_t)tid * nrb + rb] = a;
    }
    if (mode == OP_CG) {   // the update kernel reduces the partials (op_cg_begin)
        if (rb == 0 && tid == 0) op_cg_begin(ctl, tt_part, nrb);
        return;
    }
    if (!last_block_arrive(cnt_all, (unsigned)nrb)) return;
    op_finalize_block(ctl, tt_part, nrb, Q);
}

template <int QG, typename TPhi>
__global__ __launch_bounds__(128) void k_gemm2_simt(const TPhi* __restrict__ phi, long long ldp,
                                                   const float* __restrict__ T, long long Np, long long rchunk2,
                                                   float* __restrict__ U, long long Dp, int Q, size_t sstride) {
    constexpr int QP = QG * 8;
    __shared__ __align__(16) float sT[G2_BI][QP];
    const long long j = (long long)blockIdx.x * 128 + threadIdx.x;
    const int s = blockIdx.y;
    const long long i0 = (long long)s * rchunk2;
    const long long i1 = i0 + rchunk2 < Np ? i0 + rchunk2 : Np;
    float acc[QP];
#pragma unroll
    for (int q = 0; q < QP; ++q) acc[q] = 0.0f;
    for (long long ib = i0; ib < i1; ib += G2_BI) {
        for (int idx = threadIdx.x; idx < G2_BI * QP / 4; idx += 128) {
            const int r = idx / (QP / 4), c4 = (idx % (QP / 4)) * 4;
            *reinterpret_cast<float4*>(&sT[r][c4]) = ld4(T + (ib + r) * QP + c4);
        }
        __syncthreads();
#pragma unroll 1
        for (int r8 = 0; r8 < G2_BI; r8 += 8) {
            float a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) a[u] = ld1(phi + (ib + r8 + u) * ldp + j);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
#pragma unroll
                for (int c4 = 0; c4 < QP; c4 += 4) {
                    const float4 tv = *reinterpret_cast<const float4*>(&sT[r8 + u][c4]);
                    acc[c4 + 0] = fmaf(a[u], tv.x, acc[c4 + 0]);
                    acc[c4 + 1] = fmaf(a[u], tv.y, acc[c4 + 1]);
                    acc[c4 + 2] = fmaf(a[u], tv.z, acc[c4 + 2]);
                    acc[c4 + 3] = fmaf(a[u], tv.w, acc[c4 + 3]);
                }
            }
        }
        __syncthreads();
    }
    float* Us = U + (size_t)s * sstride;
#pragma unroll
    for (int q = 0; q < QP; ++q)
        if (q < Q) Us[(size_t)q * Dp + j] = acc[q];
}

// theta_j = sum_i Phi_ij^2 (y == null) or b_j = scale * sum_i Phi_ij y_i, FP64 accumulation
template <typename TPhi>
__global__ __launch_bounds__(128) void k_colreduce(const TPhi* __restrict__ phi, long long ldp, long long N,
                                                   long long D, const float* __restrict__ y, double scale,
                                                   float* __restrict__ out) {
    const long long j = (long long)blockIdx.x * 128 + threadIdx.x;
    double acc = 0.0;
    long long i = 0;
    for (; i + 8 <= N; i += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = (float)phi[(i + u) * ldp + j];
        float p = 0.0f;
#pragma unroll
        for (int u = 0; u < 8; ++u) p = fmaf(v[u], y ? __ldg(y + i + u) : v[u], p);
        acc += (double)p;
    }
    for (; i < N; ++i) {
        const float v = (float)phi[i * ldp + j];
        acc += (double)v * (double)(y ? y[i] : v);
    }
    out[j] = j < D ? (float)(scale * acc) : 0.0f;
}

template <int QG, typename TPhi>
void launch_pair_t(Sink& s, cofem_ctx* c, const TPhi* phi, int Q, const float* V, int mode) {
    const int nrb = (int)(c->Np / G1_BM);
    s.launch(k_gemm1_simt<QG, TPhi>, dim3(nrb, c->S1), dim3(256), 0, phi, c->Dp, V, c->Dp, Q, c->chunk1, c->S1,
             c->Tpart, c->T, c->Np, c->tt_part, nrb, c->counters + 16, c->counters + 8, c->ctl, mode);
    s.launch(k_gemm2_simt<QG, TPhi>, dim3((unsigned)(c->Dp / 128), c->S2), dim3(128), 0, phi, c->Dp, c->T, c->Np,
             c->rchunk2, c->U, c->Dp, Q, (size_t)c->Qcap * c->Dp);
}

template <int QG>
void launch_pair(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    if (c->phi16) launch_pair_t<QG, __nv_bfloat16>(s, c, c->phi16, Q, V, mode);
    else launch_pair_t<QG, float>(s, c, c->phi32, Q, V, mode);
}

}  // namespace

// Split factors for a block of Q columns.
void dense_configure(cofem_ctx* c, int Q) {
    c->QP = ((Q + 7) / 8) * 8;
    if (c->use_tc) {   // tensor-core path: T and the partial sums live in the plan
        c->S1 = 1;
        c->S2 = 1;
        c->chunk1 = c->Dp;
        c->rchunk2 = c->Np;
        return;
    }
    // split factors: enough blocks to cover the SMs twice, but no more than 8
    // slices and no slice shorter than 512 columns / 128 rows (the slice
    // partials are summed by a dependent chain in the last block)
    const long long nrb = c->Np / G1_BM;
    long long S1 = (2LL * c->num_sms + nrb - 1) / nrb;
    if (S1 < 1) S1 = 1;
    if (S1 > 8) S1 = 8;
    long long chunk1 = ((c->Dp + S1 - 1) / S1 + G1_BK - 1) / G1_BK * G1_BK;
    if (chunk1 < 512) chunk1 = 512;
    c->chunk1 = chunk1;
    c->S1 = (int)((c->Dp + chunk1 - 1) / chunk1);
    const long long ncb = c->Dp / 128;
    long long S2 = (2LL * c->num_sms + ncb - 1) / ncb;
    if (S2 < 1) S2 = 1;
    if (S2 > 8) S2 = 8;
    long long r2 = ((c->Np + S2 - 1) / S2 + G2_BI - 1) / G2_BI * G2_BI;
    if (r2 < 128) r2 = 128;
    c->rchunk2 = r2;
    c->S2 = (int)((c->Np + r2 - 1) / r2);
}

void launch_dense_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    if (c->use_tc) {
        launch_tc_operator(s, c, Q, V, mode);
        return;
    }
    switch (c->QP / 8) {
        case 1: launch_pair<1>(s, c, Q, V, mode); break;
        case 2: launch_pair<2>(s, c, Q, V, mode); break;
        case 3: launch_pair<3>(s, c, Q, V, mode); break;
        case 4: launch_pair<4>(s, c, Q, V, mode); break;
        case 5: launch_pair<5>(s, c, Q, V, mode); break;
        case 6: launch_pair<6>(s, c, Q, V, mode); break;
        case 7: launch_pair<7>(s, c, Q, V, mode); break;
        default: launch_pair<8>(s, c, Q, V, mode); break;
    }
}

void launch_dense_colreduce(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out) {
    const dim3 grid((unsigned)(c->Dp / 128));
    if (c->phi8)
        launch_colreduce_fp8(st, c->phi8, c->scale8, c->Dp, c->N, c->D, y, scale, out);
    else if (c->phi16)
        k_colreduce<__nv_bfloat16><<<grid, 128, 0, st>>>(c->phi16, c->Dp, c->N, c->D, y, scale, out);
    else
        k_colreduce<float><<<grid, 128, 0, st>>>(c->phi32, c->Dp, c->N, c->D, y, scale, out);
}
