// Convolutional dictionary (Sec. V-A "Convolutional", Sec. VI-A): N = D and
//   (Phi v)_i   = sum_{tau<L} h[tau] v[i - tau]      (zero for i - tau < 0)
//   (Phi^T u)_j = sum_{tau<L} h[tau] u[j + tau]      (zero for j + tau >= N)
// Phi is never formed.  One block computes, for one column q and an output tile
// [j0, j0 + B) with B = 2048 - (L - 1), the intermediate T = Phi v on
// [j0, j0 + 2048) from a shared-memory window of v with an L - 1 halo, keeps T in
// shared memory, and writes U = Phi^T T on the tile.  (The paper applies the
// convolution through FFTs; this is the direct form, tiled on chip.)
#include "cofem_internal.cuh"

namespace {

constexpr int TZ_THREADS = 256, TZ_R = 8, TZ_NT = TZ_THREADS * TZ_R;   // 2048 T values per block

__device__ __forceinline__ void ld8(const float* p, float* w) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w; w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

// out[m] = sum_{tau < Lp} coef[tau] * src[base + m + tau], m < 8 (coef zero-padded to Lp).
__device__ __forceinline__ void slide_corr8(const float* coef, const float* src, int base, int Lp, float* out) {
    float acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = 0.0f;
    float w[16];
    ld8(src + base, w);
#pragma unroll 1
    for (int tb = 0; tb < Lp; tb += 8) {
        ld8(src + base + tb + 8, w + 8);
        float c[8];
        ld8(coef + tb, c);
#pragma unroll
        for (int d = 0; d < 8; ++d)
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] = fmaf(c[d], w[m + d], acc[m]);
#pragma unroll
        for (int m = 0; m < 8; ++m) w[m] = w[m + 8];
    }
#pragma unroll
    for (int m = 0; m < 8; ++m) out[m] = acc[m];
}

__global__ __launch_bounds__(TZ_THREADS) void k_toeplitz(const float* __restrict__ h, int L, int Lp,
                                                          const float* __restrict__ V, long long N, long long Dp,
                                                          float* __restrict__ U, int Bout, double* tt_part, int nblk,
                                                          unsigned* counter, DevCtl* ctl, int mode, int Q) {
    extern __shared__ __align__(16) float sm[];
    float* sh = sm;                   // h[tau], zero-padded to Lp
    float* shr = sh + Lp;             // h[L-1-tau'], zero-padded to Lp
    float* sV = shr + Lp;             // v[j0 - (L-1) + idx], idx < TZ_NT + Lp
    float* sT = sV + TZ_NT + Lp;      // T[j0 + idx], idx < TZ_NT + Lp (zero beyond TZ_NT)
    __shared__ double red[TZ_THREADS / 32];
    const int q = blockIdx.y, blk = blockIdx.x, th = threadIdx.x;
    const long long j0 = (long long)blk * Bout;
    const float* Vq = V + (size_t)q * Dp;
    for (int i = th; i < Lp; i += TZ_THREADS) {
        sh[i] = i < L ? h[i] : 0.0f;
        shr[i] = i < L ? h[L - 1 - i] : 0.0f;
    }
    for (int idx = th; idx < TZ_NT + Lp; idx += TZ_THREADS) {
        const long long g = j0 - (L - 1) + idx;
        sV[idx] = (g >= 0 && g < N) ? __ldg(Vq + g) : 0.0f;
        sT[idx] = 0.0f;
    }
    __syncthreads();
    // T_i = sum_tau h[tau] v[i - tau] for i = j0 + 8 th + m
    float tv[8];
    slide_corr8(shr, sV, th * TZ_R, Lp, tv);
    float tt = 0.0f;
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        const int idx = th * TZ_R + m;
        const long long i = j0 + idx;
        const float v = i < N ? tv[m] : 0.0f;
        sT[idx] = v;
        if (idx < Bout) tt = fmaf(v, v, tt);   // T_i owned by this tile
    }
    __syncthreads();
    // U_j = sum_tau h[tau] T[j + tau] for j = j0 + 8 th + m < j0 + Bout
    float* Uq = U + (size_t)q * Dp;
    if (th * TZ_R < Bout) {
        float uv[8];
        slide_corr8(sh, sT, th * TZ_R, Lp, uv);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int idx = th * TZ_R + m;
            const long long j = j0 + idx;
            if (idx < Bout && j < Dp) Uq[j] = j < N ? uv[m] : 0.0f;
        }
    }
    const double ttd = block_sum_f(tt, red);
    if (th == 0) tt_part[(size_t)q * nblk + blk] = ttd;
    if (mode == OP_CG) {   // the update kernel reduces the partials (op_cg_begin)
        if (blk == 0 && q == 0 && th == 0) op_cg_begin(ctl, tt_part, nblk);
        return;
    }
    if (!last_block_arrive(counter, gridDim.x * gridDim.y)) return;
    op_finalize_block(ctl, tt_part, nblk, Q);
}

__global__ void k_toeplitz_theta(const float* __restrict__ h, int L, long long N, long long Dp,
                                 float* __restrict__ theta) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Dp) return;
    double a = 0.0;   // FP32 runs of 8 taps, FP64 across runs
    if (j < N) {
        const long long m = (N - j) < L ? (N - j) : L;
        for (long long t0 = 0; t0 < m; t0 += 8) {
            float f = 0.0f;
            for (long long tau = t0; tau < t0 + 8 && tau < m; ++tau) f = fmaf(h[tau], h[tau], f);
            a += (double)f;
        }
    }
    theta[j] = (float)a;
}

__global__ void k_toeplitz_phit_y(const float* __restrict__ h, int L, long long N, long long Dp,
                                  const float* __restrict__ y, double scale, float* __restrict__ out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Dp) return;
    double a = 0.0;   // FP32 runs of 8 taps, FP64 across runs
    if (j < N) {
        const long long m = (N - j) < L ? (N - j) : L;
        for (long long t0 = 0; t0 < m; t0 += 8) {
            float f = 0.0f;
            for (long long tau = t0; tau < t0 + 8 && tau < m; ++tau) f = fmaf(__ldg(h + tau), __ldg(y + j + tau), f);
            a += (double)f;
        }
    }
    out[j] = (float)(scale * a);
}

}  // namespace

static int toeplitz_lp(int L) { return ((L + 7) / 8) * 8; }

void launch_toeplitz_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    const int Lp = toeplitz_lp(c->L);
    const int Bout = TZ_NT - (c->L - 1);
    const int nblk = (int)((c->Dp + Bout - 1) / Bout);
    const size_t smem = (size_t)(2 * Lp + 2 * (TZ_NT + Lp)) * sizeof(float);
    s.launch(k_toeplitz, dim3(nblk, Q), dim3(TZ_THREADS), smem, c->h, c->L, Lp, V, c->N, c->Dp, c->U, Bout,
             c->tt_part, nblk, c->counters + 8, c->ctl, mode, Q);
}

void launch_toeplitz_theta(cudaStream_t st, cofem_ctx* c) {
    k_toeplitz_theta<<<(unsigned)((c->Dp + 255) / 256), 256, 0, st>>>(c->h, c->L, c->N, c->Dp, c->theta);
}

void launch_toeplitz_phit_y(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out) {
    k_toeplitz_phit_y<<<(unsigned)((c->Dp + 255) / 256), 256, 0, st>>>(c->h, c->L, c->N, c->Dp, y, scale, out);
}

// Shared memory the operator kernel needs (the caller raises the limit once).
size_t toeplitz_smem_bytes(int L) {
    const int Lp = toeplitz_lp(L);
    return (size_t)(2 * Lp + 2 * (TZ_NT + Lp)) * sizeof(float);
}

cudaError_t toeplitz_prepare(int L) {
    // all supported L (<= 1024) stay within the default 48 KiB; raising the limit
    // per handle would race with concurrent handles, so it is set once for the
    // largest L in cofem_kernel_attributes
    (void)L;
    return cudaSuccess;
}

cudaError_t toeplitz_kernel_attributes() {
    return cudaFuncSetAttribute(k_toeplitz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)toeplitz_smem_bytes(1024));
}
