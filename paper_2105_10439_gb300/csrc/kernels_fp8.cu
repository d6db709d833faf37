// FP8 E4M3 storage of a dense dictionary with per-row FP32 scales:
//   Phi~_ij = s_i * e4m3(Phi_ij / s_i),  s_i = max_j |Phi_ij| / 448
// (448 = the largest E4M3 magnitude; the codes are round-to-nearest-even with
// saturation).  The method then runs on Phi~ (theta, b and the operator).
// Rows with max |Phi_ij| = 0, and the padding rows, get s_i = 0 and zero codes;
// padding columns get zero codes.
#include <cuda_fp8.h>

#include "cofem_internal.cuh"

namespace {

__device__ __forceinline__ float e4m3_to_float(uint8_t b) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
    return __half2float(__half(h));
}

// One block per row: row max, scale, codes.
__global__ __launch_bounds__(256) void k_quantize_fp8(const float* __restrict__ src, long long ld, long long N,
                                                      long long D, long long Dp, uint8_t* __restrict__ codes,
                                                      float* __restrict__ scales) {
    __shared__ float red[8];
    const long long i = blockIdx.x;
    uint8_t* out = codes + (size_t)i * Dp;
    float m = 0.0f;
    if (i < N)
        for (long long j = threadIdx.x; j < D; j += blockDim.x) m = fmaxf(m, fabsf(src[(size_t)i * ld + j]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    const float s = m / 448.0f;
    if (threadIdx.x == 0) scales[i] = i < N ? s : 0.0f;
    for (long long j = 2 * threadIdx.x; j < Dp; j += 2 * blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (i < N && s > 0.0f) {
            if (j < D) v.x = src[(size_t)i * ld + j] / s;
            if (j + 1 < D) v.y = src[(size_t)i * ld + j + 1] / s;
        }
        const __nv_fp8x2_storage_t q = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
        *reinterpret_cast<__nv_fp8x2_storage_t*>(out + j) = q;
    }
}

// theta_j = sum_i Phi~_ij^2 (y == null) or b_j = scale * sum_i Phi~_ij y_i:
// FP32 runs of 8 rows, FP64 across runs.
__global__ __launch_bounds__(128) void k_colreduce_fp8(const uint8_t* __restrict__ codes, const float* __restrict__ s,
                                                       long long Dp, long long N, long long D,
                                                       const float* __restrict__ y, double scale,
                                                       float* __restrict__ out) {
    const long long j = (long long)blockIdx.x * 128 + threadIdx.x;
    double acc = 0.0;
    for (long long i0 = 0; i0 < N; i0 += 8) {
        float p = 0.0f;
        for (long long i = i0; i < i0 + 8 && i < N; ++i) {
            const float v = s[i] * e4m3_to_float(codes[(size_t)i * Dp + j]);
            p = fmaf(v, y ? __ldg(y + i) : v, p);
        }
        acc += (double)p;
    }
    out[j] = j < D ? (float)(scale * acc) : 0.0f;
}

// out (N x D, row stride D) = Phi~ in FP32.
__global__ void k_dequant_fp8(const uint8_t* __restrict__ codes, const float* __restrict__ s, long long N,
                              long long D, long long Dp, float* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * D) return;
    const long long i = idx / D, j = idx % D;
    out[idx] = s[i] * e4m3_to_float(codes[(size_t)i * Dp + j]);
}

// out (N x D, row stride D) = bf16 dictionary in FP32.
__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ src, long long N, long long D, long long ld,
                              float* __restrict__ out) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * D) return;
    out[idx] = __bfloat162float(src[(size_t)(idx / D) * ld + idx % D]);
}

}  // namespace

void launch_bf16_to_f32(cudaStream_t st, const __nv_bfloat16* src, long long N, long long D, long long ld,
                        float* out) {
    const long long n = N * D;
    k_bf16_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, N, D, ld, out);
}

void launch_quantize_fp8(cudaStream_t st, const float* src, long long ld, long long N, long long D, long long Np,
                         long long Dp, uint8_t* codes, float* scales) {
    k_quantize_fp8<<<(unsigned)Np, 256, 0, st>>>(src, ld, N, D, Dp, codes, scales);
}

void launch_colreduce_fp8(cudaStream_t st, const uint8_t* codes, const float* scales, long long Dp, long long N,
                          long long D, const float* y, double scale, float* out) {
    k_colreduce_fp8<<<(unsigned)(Dp / 128), 128, 0, st>>>(codes, scales, Dp, N, D, y, scale, out);
}

void launch_dequant_fp8(cudaStream_t st, const uint8_t* codes, const float* scales, long long N, long long D,
                        long long Dp, float* out) {
    const long long n = N * D;
    k_dequant_fp8<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(codes, scales, N, D, Dp, out);
}
