// Convolution dictionary (Sec. V-A "Convolutional", Sec. VI-A) applied through
// FFTs, the paper's own choice for this dictionary: O(log F) per output
// instead of O(L) for the direct form (kernels_toeplitz.cu).  Same operator:
//   (Phi v)_i   = sum_{tau<L} h[tau] v[i - tau]      (zero for i - tau < 0)
//   (Phi^T u)_j = sum_{tau<L} h[tau] u[j + tau]      (zero for j + tau >= N)
// One block computes U = Phi^T (Phi v) on an output tile [j0, j0 + B) with
// B = F - 2 (L - 1), by overlap-save in shared memory (F = 8192 points):
//   1. the window v[j0 - (L-1) .. j0 - (L-1) + F) -> FFT -> times H -> inverse
//      FFT: its entries L-1 .. F-1 are T = Phi v on [j0, j0 + F - L + 1);
//   2. T on [j0, j0 + F - L + 1) (zero beyond, and at rows >= N) -> FFT ->
//      times conj(H) -> inverse FFT: entries 0 .. B-1 are U on the tile
//      (cross-correlation with h, no wrap-around for these outputs);
// with H = DFT_F(h) made once per handle (FP64 direct DFT).  h is real, so two
// columns share one complex FFT (real and imaginary parts), and each block
// takes a pair of columns.  T never leaves shared memory; the partials of
// ||Phi v||^2 over the tile's rows are written for pi.
#include "cofem_internal.cuh"
#include "fft_smem.cuh"

namespace {

constexpr int FC_LOGF = COFEM_FFTCONV_LOGF, FC_F = 1 << FC_LOGF, FC_THREADS = 1024;
constexpr int FC_PT = FC_F / FC_THREADS;   // points a thread gathers

// H[m] = sum_tau h[tau] e^{-2 pi i m tau / F} in FP64 (angle reduced exactly).
__global__ void k_fc_spectrum(const float* __restrict__ h, int L, float2* __restrict__ H) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= FC_F) return;
    double re = 0.0, im = 0.0;
    for (int tau = 0; tau < L; ++tau) {
        const long long k = ((long long)m * tau) % FC_F;
        double sn, cs;
        sincospi(-2.0 * (double)k / (double)FC_F, &sn, &cs);
        re += (double)h[tau] * cs;
        im += (double)h[tau] * sn;
    }
    H[m] = make_float2((float)re, (float)im);
}

// tw[m] = e^{-2 pi i m / F}, m < F/2.
__global__ void k_fc_twiddles(float2* __restrict__ tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= FC_F / 2) return;
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)FC_F, &sn, &cs);
    tw[m] = make_float2((float)cs, (float)sn);
}

__global__ __launch_bounds__(FC_THREADS) void k_toeplitz_fft(const float* __restrict__ V, long long N, long long Dp,
                                                              int L, int Bout, const float2* __restrict__ H,
                                                              const float2* __restrict__ tw, float* __restrict__ U,
                                                              double* tt_part, int nblk, unsigned* counter,
                                                              DevCtl* ctl, int mode, int Q) {
    extern __shared__ __align__(16) float2 s[];   // F complex points
    __shared__ double red[FC_THREADS / 32];
    const int tile = blockIdx.x, q1 = 2 * blockIdx.y, q2 = q1 + 1;
    const bool two = q2 < Q;
    const long long j0 = (long long)tile * Bout;
    const float* v1 = V + (size_t)q1 * Dp;
    const float* v2 = two ? V + (size_t)q2 * Dp : nullptr;
    const float invF = 1.0f / (float)FC_F;
    // 1. T = Phi v on the tile's rows (and the L - 1 after them)
    for (int m = threadIdx.x; m < FC_F; m += FC_THREADS) {
        const long long g = j0 - (L - 1) + m;
        const bool in = g >= 0 && g < N;
        s[brev(m, FC_LOGF)] = make_float2(in ? __ldg(v1 + g) : 0.0f, in && two ? __ldg(v2 + g) : 0.0f);
    }
    __syncthreads();
    fft_smem(s, FC_LOGF, tw, false);
    for (int m = threadIdx.x; m < FC_F; m += FC_THREADS) s[m] = cmul(s[m], __ldg(H + m));
    __syncthreads();
    bitrev_smem(s, FC_LOGF);
    fft_smem(s, FC_LOGF, tw, true);
    // 2. the window of T for the correlation, shifted by L - 1 and bit-reversed
    // (gathered into registers before shared memory is overwritten)
    float2 gv[FC_PT];
    float tt1 = 0.0f, tt2 = 0.0f;
#pragma unroll
    for (int k = 0; k < FC_PT; ++k) {
        const int mp = threadIdx.x + k * FC_THREADS;
        const int idx = mp + L - 1;
        const long long i = j0 + mp;
        float2 t = make_float2(0.0f, 0.0f);
        if (idx < FC_F && i < N) t = make_float2(s[idx].x * invF, s[idx].y * invF);
        if (mp < Bout) {   // rows owned by this tile
            tt1 = fmaf(t.x, t.x, tt1);
            tt2 = fmaf(t.y, t.y, tt2);
        }
        gv[k] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < FC_PT; ++k) s[brev(threadIdx.x + k * FC_THREADS, FC_LOGF)] = gv[k];
    __syncthreads();
    fft_smem(s, FC_LOGF, tw, false);
    for (int m = threadIdx.x; m < FC_F; m += FC_THREADS) s[m] = cmul(s[m], conjf2(__ldg(H + m)));
    __syncthreads();
    bitrev_smem(s, FC_LOGF);
    fft_smem(s, FC_LOGF, tw, true);
    // U = Phi^T T on the tile
    float* U1 = U + (size_t)q1 * Dp;
    float* U2 = U + (size_t)q2 * Dp;
    for (int jp = threadIdx.x; jp < Bout; jp += FC_THREADS) {
        const long long j = j0 + jp;
        if (j >= Dp) break;
        const float2 u = s[jp];
        U1[j] = j < N ? u.x * invF : 0.0f;
        if (two) U2[j] = j < N ? u.y * invF : 0.0f;
    }
    const double d1 = block_sum_f(tt1, red);
    const double d2 = block_sum_f(tt2, red);
    if (threadIdx.x == 0) {
        tt_part[(size_t)q1 * nblk + tile] = d1;
        if (two) tt_part[(size_t)q2 * nblk + tile] = d2;
    }
    if (mode == OP_CG) {   // the update kernel reduces the partials (op_cg_begin)
        if (tile == 0 && blockIdx.y == 0 && threadIdx.x == 0) op_cg_begin(ctl, tt_part, nblk);
        return;
    }
    if (!last_block_arrive(counter, gridDim.x * gridDim.y)) return;
    op_finalize_block(ctl, tt_part, nblk, Q);
}

}  // namespace

size_t fftconv_smem_bytes() { return (size_t)FC_F * sizeof(float2); }

cudaError_t fftconv_kernel_attributes() {
    return cudaFuncSetAttribute(k_toeplitz_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)fftconv_smem_bytes());
}

// Output rows per tile for filter length L (the overlap-save block).
int fftconv_bout(int L) { return FC_F - 2 * (L - 1); }

// Once per handle: H = DFT_F(h) and the FFT twiddles.
void launch_fftconv_setup(cudaStream_t st, cofem_ctx* c) {
    k_fc_spectrum<<<FC_F / 256, 256, 0, st>>>(c->h, c->L, c->fc_H);
    k_fc_twiddles<<<FC_F / 2 / 256, 256, 0, st>>>(c->fc_tw);
}

void launch_fftconv_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    const int Bout = fftconv_bout(c->L);
    const int nblk = (int)((c->Dp + Bout - 1) / Bout);
    s.launch(k_toeplitz_fft, dim3(nblk, (Q + 1) / 2), dim3(FC_THREADS), fftconv_smem_bytes(), V, c->N, c->Dp, c->L,
             Bout, (const float2*)c->fc_H, (const float2*)c->fc_tw, c->U, c->tt_part, nblk, c->counters + 8, c->ctl,
             mode, Q);
}
