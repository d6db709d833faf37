// DCT dictionary (Sec. V-A "DCT"): Phi = M Omega^-1 with Omega the orthonormal
// DCT-II of size D (Omega_kn = c_k cos(pi k (2n + 1) / (2D)), c_0 = sqrt(1/D),
// c_k = sqrt(2/D)), Omega^-1 = Omega^T, and M the selection of N rows.  So
//   Phi v   = (Omega^T v)[rows]                 (a DCT-III, then a gather)
//   Phi^T u = Omega (u scattered to rows)       (a scatter, then a DCT-II)
// and Phi^T Phi p = Omega (mask . Omega^T p): one block per column q applies
// both transforms in shared memory, O(D log D) per column, Phi never formed.
//
// Each real transform of length D (a power of two, 16 <= D <= 32768) is a
// complex FFT of length H = D/2 in shared memory (Makhoul, "A fast cosine
// transform in one and two dimensions", IEEE TASSP 1980: the even-odd
// reordering u_n = v_2n, u_{D-1-n} = v_{2n+1} turns the DCT-II into a length-D
// real DFT with a quarter-sample twiddle; the real DFT is a length-D/2
// complex DFT of z_m = u_2m + i u_{2m+1} and a split step; the DCT-III runs
// the same steps backwards).  The FFT is radix-2, decimation in time, in
// place, with the input in bit-reversed order and the e^{-2 pi i m / H}
// twiddles from a table made once per handle.
#include "cofem_internal.cuh"
#include "fft_smem.cuh"

namespace {

constexpr int DCT_THREADS = 1024;
constexpr int DCT_MAXPT = (COFEM_DCT_MAX_D / 2) / DCT_THREADS;   // FFT points a thread gathers (16)

// y_n of the DCT-III result left in s by dct3_to_smem (natural-order z):
// y_2a = u_a, y_{2a+1} = u_{D-1-a}, u_2m = Re z_m, u_{2m+1} = Im z_m.
__device__ __forceinline__ float y_at(const float2* s, int n, int D) {
    const int j = (n & 1) ? D - 1 - (n >> 1) : (n >> 1);
    const float2 z = s[j >> 1];
    return (j & 1) ? z.y : z.x;
}

// Orthonormal DCT-III (y = Omega^T w) of the column w (global, D floats) into
// shared memory: X_0 = sqrt(D) w_0, X_k = sqrt(D/2) w_k (so that the plain
// inverse DCT-II recurrence applies), U_k = e^{i pi k / 2D} (X_k - i X_{D-k}),
// Z_k = E_k + i O_k with E_k = (U_k + U_{k+H}) / 2 and O_k = (U_k - U_{k+H})
// e^{2 pi i k / D} / 2, then z = IFFT_H(Z) / H.
__device__ void dct3_to_smem(const float* __restrict__ w, int D, int logH, float2* s,
                             const float2* __restrict__ tw) {
    const int H = D / 2;
    const float sD = sqrtf((float)D), sD2 = sqrtf(0.5f * (float)D);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        const float xk = k == 0 ? sD * w[0] : sD2 * w[k];
        const float xdk = k == 0 ? 0.0f : sD2 * w[D - k];           // X_{D-k}, X_D = 0
        const float xkh = sD2 * w[k + H];                             // X_{k+H}
        const float xdkh = sD2 * w[H - k];                            // X_{D-k-H} = X_{H-k}
        const float2 uk = cmul(expi_pi(k, 2LL * D), make_float2(xk, -xdk));
        const float2 ukh = cmul(expi_pi(k + H, 2LL * D), make_float2(xkh, -xdkh));
        const float2 e = make_float2(0.5f * (uk.x + ukh.x), 0.5f * (uk.y + ukh.y));
        const float2 o = cmul(make_float2(0.5f * (uk.x - ukh.x), 0.5f * (uk.y - ukh.y)), expi_pi(2LL * k, (long long)D));
        s[brev(k, logH)] = make_float2(e.x - o.y, e.y + o.x);        // E + i O
    }
    __syncthreads();
    fft_smem(s, logH, tw, true);
    const float inv = 1.0f / (float)H;
    for (int m = threadIdx.x; m < H; m += blockDim.x) s[m] = make_float2(s[m].x * inv, s[m].y * inv);
    __syncthreads();
}

// Orthonormal DCT-II of the real vector whose reordered FFT input z already
// sits in s (bit-reversed): FFT, then U_k = E_k + e^{-2 pi i k / D} O_k with
// E_k = (Z_k + conj Z_{H-k}) / 2, O_k = (Z_k - conj Z_{H-k}) / 2i, and
// X_k = Re(e^{-i pi k / 2D} U_k), X_{D-k} = Re(e^{-i pi (D-k) / 2D} conj U_k);
// out[k] = scale c_k X_k.
__device__ void dct2_from_smem(float2* s, int D, int logH, const float2* __restrict__ tw, float scale,
                               float* __restrict__ out) {
    const int H = D / 2;
    fft_smem(s, logH, tw, false);
    const float c0 = scale * sqrtf(1.0f / (float)D), c1 = scale * sqrtf(2.0f / (float)D);
    for (int k = threadIdx.x; k <= H; k += blockDim.x) {
        const float2 zk = s[k & (H - 1)], zc = conjf2(s[(H - k) & (H - 1)]);
        const float2 e = make_float2(0.5f * (zk.x + zc.x), 0.5f * (zk.y + zc.y));
        const float2 d = make_float2(0.5f * (zk.x - zc.x), 0.5f * (zk.y - zc.y));
        const float2 o = make_float2(d.y, -d.x);                      // d / i
        const float2 t = cmul(expi_pi(2LL * D - 2LL * k, (long long)D), o);   // e^{-2 pi i k / D} O_k
        const float2 U = make_float2(e.x + t.x, e.y + t.y);
        out[k] = (k == 0 ? c0 : c1) * cmul(expi_pi(4LL * D - k, 2LL * D), U).x;
        if (k > 0 && k < H) out[D - k] = c1 * cmul(expi_pi(4LL * D - (D - k), 2LL * D), conjf2(U)).x;
    }
}

// The operator on column q of V: T = Phi v = (Omega^T v)[rows] (kept as the
// masked DCT-III in shared memory), U = Phi^T T = Omega (mask . Omega^T v)
// into U[q], and the partial of ||Phi v||^2 (one per column).
__global__ __launch_bounds__(DCT_THREADS) void k_dct_apply(const float* __restrict__ V, int D, int logH, long long Dp,
                                                           const float* __restrict__ mask,
                                                           const float2* __restrict__ tw, float* __restrict__ U,
                                                           double* tt_part, unsigned* counter, DevCtl* ctl, int mode,
                                                           int Q) {
    extern __shared__ __align__(16) float2 sz[];
    __shared__ double red[DCT_THREADS / 32];
    const int q = blockIdx.x, H = D / 2;
    dct3_to_smem(V + (size_t)q * Dp, D, logH, sz, tw);
    // masked y, reordered for the DCT-II: z'_m = u'_2m + i u'_{2m+1} with
    // u'_j = y'_{2j} (j < H), y'_{2(D-1-j)+1} (j >= H); gathered into registers
    // before shared memory is overwritten
    float2 g[DCT_MAXPT];
    float tt = 0.0f;
#pragma unroll
    for (int it = 0; it < DCT_MAXPT; ++it) {
        const int m = threadIdx.x + it * DCT_THREADS;
        if (m < H) {
            float v2[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = 2 * m + h;
                const int n = j < H ? 2 * j : 2 * (D - 1 - j) + 1;
                const float y = y_at(sz, n, D) * __ldg(mask + n);
                v2[h] = y;
                tt = fmaf(y, y, tt);   // every n appears once over all (m, h)
            }
            g[it] = make_float2(v2[0], v2[1]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < DCT_MAXPT; ++it) {
        const int m = threadIdx.x + it * DCT_THREADS;
        if (m < H) sz[brev(m, logH)] = g[it];
    }
    __syncthreads();
    float* Uq = U + (size_t)q * Dp;
    dct2_from_smem(sz, D, logH, tw, 1.0f, Uq);
    for (long long j = D + threadIdx.x; j < Dp; j += DCT_THREADS) Uq[j] = 0.0f;
    const double ttd = block_sum_f(tt, red);
    if (threadIdx.x == 0) tt_part[q] = ttd;
    if (mode == OP_CG) {   // the update kernel reduces the partials (op_cg_begin)
        if (q == 0 && threadIdx.x == 0) op_cg_begin(ctl, tt_part, 1);
        return;
    }
    if (!last_block_arrive(counter, gridDim.x)) return;
    op_finalize_block(ctl, tt_part, 1, Q);
}

// out = scale * Omega v for one real vector v (global, D floats): b = beta Phi^T y
// after y has been scattered to its rows.
__global__ __launch_bounds__(DCT_THREADS) void k_dct_forward(const float* __restrict__ v, int D, int logH,
                                                             long long Dp, const float2* __restrict__ tw,
                                                             float scale, float* __restrict__ out) {
    extern __shared__ __align__(16) float2 sz[];
    const int H = D / 2;
    for (int m = threadIdx.x; m < H; m += DCT_THREADS) {
        float v2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = 2 * m + h;
            v2[h] = v[j < H ? 2 * j : 2 * (D - 1 - j) + 1];
        }
        sz[brev(m, logH)] = make_float2(v2[0], v2[1]);
    }
    __syncthreads();
    dct2_from_smem(sz, D, logH, tw, scale, out);
    for (long long j = D + threadIdx.x; j < Dp; j += DCT_THREADS) out[j] = 0.0f;
}

// full[rows[i]] = y[i], zero elsewhere (D floats).
__global__ void k_dct_scatter(const int* __restrict__ rows, long long N, const float* __restrict__ y,
                              float* __restrict__ full) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) full[rows[i]] = y[i];
}

__global__ void k_dct_mask(const int* __restrict__ rows, long long N, float* __restrict__ mask) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) mask[rows[i]] = 1.0f;
}

// theta_j = sum_i Phi_ij^2 = c_j^2 sum_i cos^2(pi j (2 r_i + 1) / 2D), the angle
// reduced exactly modulo 2 pi in integers.
__global__ void k_dct_theta(const int* __restrict__ rows, long long N, int D, long long Dp, float* __restrict__ theta) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Dp) return;
    double a = 0.0;
    if (j < D) {
        for (long long i = 0; i < N; ++i) {
            const long long m = (j * (2LL * rows[i] + 1)) % (4LL * D);
            const float c = cospif((float)m / (float)(2LL * D));
            a += (double)(c * c);
        }
        a *= j == 0 ? 1.0 / D : 2.0 / D;
    }
    theta[j] = (float)a;
}

// tw[m] = e^{-2 pi i m / H}, m < H/2 (FP64 sincospi, rounded to FP32).
__global__ void k_dct_twiddles(int H, float2* __restrict__ tw) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= H / 2) return;
    double sn, cs;
    sincospi(-2.0 * (double)m / (double)H, &sn, &cs);
    tw[m] = make_float2((float)cs, (float)sn);
}

}  // namespace

static int log2i(long long v) {
    int l = 0;
    while ((1LL << l) < v) ++l;
    return l;
}

size_t dct_smem_bytes(long long D) { return (size_t)(D / 2) * sizeof(float2); }

cudaError_t dct_kernel_attributes() {
    cudaError_t e = cudaFuncSetAttribute(k_dct_apply, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dct_smem_bytes(COFEM_DCT_MAX_D));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dct_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dct_smem_bytes(COFEM_DCT_MAX_D));
}

// Handle set-up: the row mask (D floats), the FFT twiddles and theta.
void launch_dct_setup(cudaStream_t st, cofem_ctx* c) {
    const long long H = c->D / 2;
    cudaMemsetAsync(c->dct_mask, 0, c->Dp * sizeof(float), st);
    k_dct_mask<<<(unsigned)((c->N + 255) / 256), 256, 0, st>>>(c->dct_rows, c->N, c->dct_mask);
    k_dct_twiddles<<<(unsigned)((H / 2 + 255) / 256), 256, 0, st>>>((int)H, c->dct_tw);
    k_dct_theta<<<(unsigned)((c->Dp + 127) / 128), 128, 0, st>>>(c->dct_rows, c->N, (int)c->D, c->Dp, c->theta);
}

void launch_dct_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    s.launch(k_dct_apply, dim3(Q), dim3(DCT_THREADS), dct_smem_bytes(c->D), V, (int)c->D, log2i(c->D / 2), c->Dp,
             c->dct_mask, c->dct_tw, c->U, c->tt_part, c->counters + 8, c->ctl, mode, Q);
}

// out = scale Phi^T y: y scattered to its rows in `tmp` (Dp floats), then Omega.
void launch_dct_phit_y(cudaStream_t st, cofem_ctx* c, const float* y, double scale, float* out, float* tmp) {
    cudaMemsetAsync(tmp, 0, c->Dp * sizeof(float), st);
    k_dct_scatter<<<(unsigned)((c->N + 255) / 256), 256, 0, st>>>(c->dct_rows, c->N, y, tmp);
    k_dct_forward<<<1, DCT_THREADS, dct_smem_bytes(c->D), st>>>(tmp, (int)c->D, log2i(c->D / 2), c->Dp, c->dct_tw,
                                                                 (float)scale, out);
}
