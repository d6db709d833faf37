// Accurate residual R = B - A X of the precision form on the tensor cores:
// both products of A X = beta Phi~^T (Phi~ X) + alpha X formed from exact
// integer slices, for a BF16 dictionary or the FP8 form's codes.  The splitting idea is the
// error-free matrix product of Ozaki, Ogita, Oishi and Rump ("Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012), here with
// fixed-point slices whose digit products the tensor core sums exactly.
//
// Slices.  Each row i of the dictionary (product 1: Phi~; product 2: Phi~^T,
// i.e. each column of Phi~) gets a power of two 2^E_i >= 2 max |row|, and each
// entry v becomes three signed base-256 digits,
//     v = 2^(E_i - 24) (a0 2^16 + a1 2^8 + a2) (+ a remainder below 2^(E_i - 25)),
// with a0, a1, a2 integers in [-128, 128]: exact for every entry within 2^-15
// of the row's largest one (a bfloat16 has 8 significant bits).  Each column q
// of the right-hand block (the FP32 pair X = Xh + Xl, or t = Phi~ X in FP64)
// gets 2^F_q >= 4 max |column| and each entry x the integer
//     I = rn(x 2^(40 - F_q)) = b0 2^32 + b1 2^24 + b2 2^16 + b3 2^8 + b4,
// b_k in [-128, 128] (|I| <= 2^38).  Digits are exact in bfloat16 and a digit
// product is an integer of magnitude <= 2^14, exact in the FP32 accumulator of
// tcgen05.mma kind::f16.  The products with a + b = d share the accumulator
// block d (d <= 4; the dropped d = 5, 6 terms are below 2^-40 of the sum), and
// the accumulator is read every 128 values of k, when its sums are at most
// 3 x 128 x 2^14 < 2^23: integers that FP32 holds exactly.  The epilogue adds
// them into 32-bit integers (exact for k <= 40960) and ends a segment with the
// 64-bit integer Z = sum_d acc_d 2^(8 (4 - d)), so that
//     (Phi~ X)_iq = 2^(E_i + F_q - 48) Z_iq,
// with a relative error of about 2^-38 of sum_k |Phi~_ik| |x_kq| in all.
//
// Why: on the underdetermined dense workloads, B - A X is a cancellation of
// terms up to 10^4 times ||b||, and the precision form needs it to about
// 1e-6 ||b||, i.e. about 2^-33 relative to those terms.  The CUDA-core form
// (kernels_accurate.cu: FP32 pairs with error-free transformations) takes
// eleven FP32 instructions per multiply-add; here the tensor cores do the
// arithmetic (12 digit products per multiply-add) and the kernel streams six
// bytes per dictionary entry (the three slice images).
//
// Kernels of one accurate residual (Q columns, QO = Q rounded up to 16 <= 48):
//   k_sl_colexp     F_q from max |Xh_q|
//   k_sl_digits     digit image of X (the B operand of product 1)
//   k_sl_gemm       product 1: segment partials Z of Phi~ X
//   k_sl_finish_t   t = Phi~ X in FP64 and G_q from max |t_q|
//   k_sl_digits     digit image of t
//   k_sl_gemm       product 2: segment partials of Phi~^T t
//   k_sl_residual   R = B - beta U - alpha X (FP64) and its norms
//
// The GEMM (k_sl_gemm) is persistent and stream-K, like the CG operator's:
// work units are (row tile of 128, chunk of two 64-wide k tiles), split into
// equal contiguous ranges, one per CTA.  Warp 0 lane 0 fetches, per k tile,
// the three 16 KiB slice tiles of the dictionary (one 48 KiB bulk copy,
// L2 evict-first) and the digit tile of the vector block (5 QO rows of 128
// bytes, from L2); warp 1 lane 0 issues, per k tile, four K = 16 steps of
// three MMAs (slice a into accumulator blocks a..4, N = (5 - a) QO, the B
// operand being the first 5 - a digit blocks); sixteen epilogue warps read the
// two alternating accumulators (2 x 5 QO <= 480 TMEM columns) and keep the
// 32-bit sums of their row (TMEM lane) and QO / 4 columns.  Every wait is
// bounded: on timeout the kernel sets COFEM_FLAG_DEVICE_TIMEOUT, lets its
// copies and MMAs finish, frees TMEM and returns.
#include <algorithm>
#include <vector>

#include <cuda_fp8.h>

#include "cofem_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int SL_BM = 128, SL_BK = 64;     // tile: 128 rows x 64 bf16 (128-byte rows, 128-byte swizzle)
constexpr int SL_NA = 3;                   // digits of a dictionary entry
constexpr int SL_NB = 5;                   // digits of a vector entry
constexpr int SL_DMAX = 4;                 // digit products a + b <= SL_DMAX are kept
constexpr int SL_CHUNK = 2;                // k tiles between accumulator reads (128 values of k)
constexpr int SL_RA = 3, SL_RB = 2;        // ring stages (dictionary, vector digits)
constexpr int SL_EPI = 16;                 // epilogue warps (four per TMEM sub-partition)
constexpr int SL_THREADS = 64 + 32 * SL_EPI;
constexpr uint32_t SL_TILE = SL_BM * SL_BK * 2;     // 16 KiB
constexpr uint32_t SL_ABYTES = SL_NA * SL_TILE;     // the three slice tiles of one (row tile, k tile)
constexpr int SL_QOMAX = 48;               // 5 QO <= 240 columns per accumulator, two in 512
constexpr long long SL_KMAX = 40960;       // 3 x 2^14 x k < 2^31: the 32-bit sums of a segment
constexpr uint32_t SL_TMEM_COLS = 512;
constexpr uint32_t SL_BUF_COLS = 256;
constexpr int SL_NT = COFEM_VEC_THREADS;
constexpr int SL_CH = COFEM_VEC_CHUNK;

struct SlParams {
    const uint8_t* A;       // slice image: (row tile m, k tile kt) at ((m KT + kt) SL_ABYTES), slice a at + a SL_TILE
    const uint8_t* B;       // digit image: k tile kt at kt 5 QO 128 bytes, row b QO + q = digit b of column q
    long long W;            // work units MT x CPR
    int MT, KT, CPR;        // row tiles, k tiles, chunks per row tile
    int QO;                 // columns per digit block (multiple of 16, <= SL_QOMAX)
    uint32_t idesc[SL_NA];  // MMA of slice a: M = 128, N = (SL_NB - a) QO
    const int* seg_base;    // first segment of each CTA
    long long* part;        // [segment][QO][128] 64-bit integer sums
    unsigned* flags;        // error flag word (DevCtl::flags)
};

constexpr uint32_t sl_idesc(int M, int N) {   // kind::f16: FP32 accumulator, BF16 A and B, both K-major
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}
template <int N>
__device__ __forceinline__ void tmem_wait4(uint32_t* r) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < N; i += 4) asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]));
}

// Exponent of a row (dictionary: 2^e >= 2 max) or of a column (vector block:
// 2^e >= 4 max); 0 for an all-zero row or column.
__device__ __forceinline__ int exp_of(float m, int margin) { return m > 0.0f ? ilogbf(m) + margin : 0; }
__device__ __forceinline__ int exp_of(double m, int margin) { return m > 0.0 ? ilogb(m) + margin : 0; }

// The three digits of a dictionary entry v with row exponent e (|v| <= 2^(e-1)):
// w = v 2^(8 - e) in [-128, 128]; a0 = rn(w), a1 = rn(256 (w - a0)), a2 =
// rn(256 (256 (w - a0) - a1)).  Every step is exact in FP32 (w has at most the
// 8 significant bits of a bfloat16).
__device__ __forceinline__ void dict_digits(float v, int e, float d[SL_NA]) {
    float w = ldexpf(v, 8 - e);
#pragma unroll
    for (int a = 0; a < SL_NA; ++a) {
        d[a] = rintf(w);
        w = __fmul_rn(__fsub_rn(w, d[a]), 256.0f);
    }
}

// The five digits of the integer I (|I| <= 2^38), lowest first: b4 = the
// signed residue of I mod 256 in [-128, 127], I <- (I - b4) / 256, ...;
// b0 = what is left (|b0| <= 64).
__device__ __forceinline__ void vec_digits(long long I, int d[SL_NB]) {
#pragma unroll
    for (int b = SL_NB - 1; b > 0; --b) {
        const int r = (int)((I + 128) & 255) - 128;
        d[b] = r;
        I = (I - r) >> 8;
    }
    d[0] = (int)I;
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

// ---------------------------------------------------------------------------
// Dictionary slice images (once per handle).  The dictionary is the BF16
// copy, or the FP8 form's E4M3 codes C (Phi~ = diag(s) C: the slices are
// those of C, exact with three digits since a code has 4 significant bits
// and spans 2^-9 .. 448, and the row scales enter t = s^2 (C X)).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dict_value(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float dict_value(uint8_t v) {   // an E4M3 code's value (exact in FP16)
    return __half2float(__half(__nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)v, __NV_E4M3)));
}

// E[i] for each row i of the row-major Np x Dp dictionary (one block per row).
template <typename TE>
__global__ __launch_bounds__(256) void k_sl_row_exp(const TE* __restrict__ phi, long long Dp, int* __restrict__ E) {
    __shared__ float sh[8];
    const long long i = blockIdx.x;
    float m = 0.0f;
    for (long long j = threadIdx.x; j < Dp; j += blockDim.x) m = fmaxf(m, fabsf(dict_value(phi[i * Dp + j])));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
        E[i] = exp_of(fmaxf(m, sh[0]), 2);
    }
}

// Column maxima of the dictionary as FP32 bit patterns (non-negative floats
// order like their bit patterns): rows split over blockIdx.y, atomicMax.
template <typename TE>
__global__ __launch_bounds__(256) void k_sl_col_max(const TE* __restrict__ phi, long long Np, long long Dp,
                                                    int rows_per_block, unsigned* __restrict__ cmax) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Dp) return;
    const long long i0 = (long long)blockIdx.y * rows_per_block;
    const long long i1 = std::min(Np, i0 + rows_per_block);
    float m = 0.0f;
    for (long long i = i0; i < i1; ++i) m = fmaxf(m, fabsf(dict_value(phi[i * Dp + j])));
    atomicMax(cmax + j, __float_as_uint(m));
}

__global__ void k_sl_col_exp(const unsigned* __restrict__ cmax, long long Dp, int* __restrict__ E) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < Dp) E[j] = exp_of(__uint_as_float(cmax[j]), 2);
}

// Slice image of product 1: tile (m, kt, a) holds digit a of rows m 128 ..
// m 128 + 127 and columns kt 64 .. kt 64 + 63 of the dictionary, rows of 128
// bytes, 16-byte chunk c of row r at chunk c ^ (r & 7).  Grid (KT, MT), one
// thread per row.
template <typename TE>
__global__ __launch_bounds__(128) void k_sl_tile_rows(const TE* __restrict__ phi, long long Dp, int KT,
                                                      const int* __restrict__ E, uint8_t* __restrict__ img) {
    const int kt = blockIdx.x, m = blockIdx.y, rr = threadIdx.x;
    const long long i = (long long)m * SL_BM + rr;
    const int e = E[i];
    const TE* src = phi + i * Dp + (long long)kt * SL_BK;
    uint8_t* tile = img + ((size_t)m * KT + kt) * SL_ABYTES;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t out[SL_NA][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float d0[SL_NA], d1[SL_NA];
            dict_digits(dict_value(src[c * 8 + 2 * h]), e, d0);
            dict_digits(dict_value(src[c * 8 + 2 * h + 1]), e, d1);
#pragma unroll
            for (int a = 0; a < SL_NA; ++a) out[a][h] = pack_bf16(d0[a], d1[a]);
        }
#pragma unroll
        for (int a = 0; a < SL_NA; ++a)
            *reinterpret_cast<uint4*>(tile + a * SL_TILE + rr * 128 + ((c ^ (rr & 7)) << 4)) =
                make_uint4(out[a][0], out[a][1], out[a][2], out[a][3]);
    }
}

// Slice image of product 2 (rows = columns of the dictionary): tile (m, kt, a)
// holds digit a of element (rr, cc) = phi[kt 64 + cc][m 128 + rr] with the
// exponent of dictionary column m 128 + rr.  Grid (KT, MT).
template <typename TE>
__global__ __launch_bounds__(128) void k_sl_tile_cols(const TE* __restrict__ phi, long long Dp, int KT,
                                                      const int* __restrict__ E, uint8_t* __restrict__ img) {
    __shared__ float sm[SL_BK][SL_BM + 1];
    const int kt = blockIdx.x, m = blockIdx.y, t = threadIdx.x;
    for (int n = 0; n < SL_BK; ++n)
        sm[n][t] = dict_value(phi[((long long)kt * SL_BK + n) * Dp + (long long)m * SL_BM + t]);
    __syncthreads();
    const int e = E[(long long)m * SL_BM + t];
    uint8_t* tile = img + ((size_t)m * KT + kt) * SL_ABYTES;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        uint32_t out[SL_NA][4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float d0[SL_NA], d1[SL_NA];
            dict_digits(sm[c * 8 + 2 * h][t], e, d0);
            dict_digits(sm[c * 8 + 2 * h + 1][t], e, d1);
#pragma unroll
            for (int a = 0; a < SL_NA; ++a) out[a][h] = pack_bf16(d0[a], d1[a]);
        }
#pragma unroll
        for (int a = 0; a < SL_NA; ++a)
            *reinterpret_cast<uint4*>(tile + a * SL_TILE + t * 128 + ((c ^ (t & 7)) << 4)) =
                make_uint4(out[a][0], out[a][1], out[a][2], out[a][3]);
    }
}

// ---------------------------------------------------------------------------
// Digits of the right-hand block.
// ---------------------------------------------------------------------------
// F[q] from max_j |Xh[q][j]| (one block per column of the padded block; 0 for
// q >= Q).  |Xh + Xl| exceeds |Xh| by at most 2^-24 relative, inside the margin.
__global__ __launch_bounds__(1024) void k_sl_colexp(const float* __restrict__ X, long long ld, long long n, int Q,
                                                    int* __restrict__ F) {
    __shared__ float sh[32];
    const int q = blockIdx.x;
    float m = 0.0f;
    if (q < Q)
        for (long long j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, fabsf(X[(size_t)q * ld + j]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, sh[w]);
        F[q] = exp_of(m, 3);
    }
}

// Digit image of QO columns of length Kp (a multiple of 64): thread (g, q)
// turns the 8 values k = 8 g .. 8 g + 7 of column q into five 16-byte chunks,
// one per digit row b QO + q of k tile 8 g / 64.  PAIR: the FP32 pair
// (xh, xl); else the FP64 column xd.  Columns q >= Q are zero.
template <bool PAIR>
__global__ __launch_bounds__(256) void k_sl_digits(const float* __restrict__ xh, const float* __restrict__ xl,
                                                   const double* __restrict__ xd, long long ld, long long Kp, int Q,
                                                   int QO, const int* __restrict__ F, uint8_t* __restrict__ img) {
    griddep_launch();
    griddep_wait();
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    const long long k0 = g * 8;
    if (k0 >= Kp) return;
    int d[8][SL_NB];
    if (q < Q) {
        const int sh = 40 - F[q];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            long long I;
            if (PAIR) {
                const size_t o = (size_t)q * ld + k0 + e;
                I = __float2ll_rn(ldexpf(xh[o], sh)) + __float2ll_rn(ldexpf(xl[o], sh));
            } else {
                I = __double2ll_rn(ldexp(xd[(size_t)q * ld + k0 + e], sh));
            }
            vec_digits(I, d[e]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e)
#pragma unroll
            for (int b = 0; b < SL_NB; ++b) d[e][b] = 0;
    }
    const int c = (int)((k0 & 63) >> 3);
    uint8_t* tile = img + (size_t)(k0 >> 6) * (SL_NB * QO) * 128;
#pragma unroll
    for (int b = 0; b < SL_NB; ++b) {
        const int n = b * QO + q;
        const uint4 v = make_uint4(pack_bf16((float)d[0][b], (float)d[1][b]), pack_bf16((float)d[2][b], (float)d[3][b]),
                                   pack_bf16((float)d[4][b], (float)d[5][b]), pack_bf16((float)d[6][b], (float)d[7][b]));
        *reinterpret_cast<uint4*>(tile + n * 128 + ((c ^ (n & 7)) << 4)) = v;
    }
}

// ---------------------------------------------------------------------------
// The sliced GEMM: part[seg][q][r] = sum over the segment's k of the digit
// products of row r of its row tile and column q, combined into Z.
// ---------------------------------------------------------------------------
template <int QPW>
__global__ void __launch_bounds__(SL_THREADS, 1) k_sl_gemm(SlParams p) {
    griddep_launch();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int QO = p.QO;
    const uint32_t B_BYTES = (uint32_t)(SL_NB * QO) * 128u;   // a multiple of 1024 (QO % 16 == 0)
    uint8_t* ringA = smem;
    uint8_t* ringB = ringA + SL_RA * SL_ABYTES;
    uint64_t* bars = (uint64_t*)(ringB + SL_RB * B_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = a_full + SL_RA;
    uint64_t* b_full = a_empty + SL_RA;
    uint64_t* b_empty = b_full + SL_RB;
    uint64_t* acc_full = b_empty + SL_RB;   // [2]
    uint64_t* acc_empty = acc_full + 2;     // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < SL_RA; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), 1);
        }
        for (int i = 0; i < SL_RB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(acc_full + i), 1);
            mbar_init(smem_u32(acc_empty + i), SL_EPI);
        }
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(SL_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long u0 = (long long)blockIdx.x * p.W / gridDim.x;
    const long long u1 = (long long)(blockIdx.x + 1) * p.W / gridDim.x;
    long long na = 0, nb = 0;   // copies issued into the two rings (producer thread)

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- bulk-copy producer ----------------
            uint64_t evict_first;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
            // the slice image is written once per handle: fill its ring before
            // waiting for the previous kernel, whose output is the B operand
            long long npre = 0;
            for (long long u = u0; u < u1 && npre < SL_RA; ++u) {
                const int m = (int)(u / p.CPR), c = (int)(u % p.CPR);
                const int kt1 = min(p.KT, (c + 1) * SL_CHUNK);
                for (int kt = c * SL_CHUNK; kt < kt1 && npre < SL_RA; ++kt, ++npre) {
                    mbar_expect_tx(smem_u32(a_full + npre), SL_ABYTES);
                    bulk_load_hint(smem_u32(ringA + npre * SL_ABYTES), p.A + ((size_t)m * p.KT + kt) * SL_ABYTES,
                                   SL_ABYTES, smem_u32(a_full + npre), evict_first);
                }
            }
            na = npre;
            griddep_wait();
            long long ea = 0;   // k tiles walked
            bool ok = true;
            for (long long u = u0; u < u1 && ok; ++u) {
                const int m = (int)(u / p.CPR), c = (int)(u % p.CPR);
                const int kt1 = min(p.KT, (c + 1) * SL_CHUNK);
                for (int kt = c * SL_CHUNK; kt < kt1; ++kt, ++ea) {
                    int slot = (int)(nb % SL_RB);
                    long long use = nb / SL_RB;
                    if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(b_full + slot), B_BYTES);
                    bulk_load(smem_u32(ringB + slot * B_BYTES), p.B + (size_t)kt * B_BYTES, B_BYTES,
                              smem_u32(b_full + slot));
                    ++nb;
                    if (ea < npre) continue;   // issued before the wait
                    slot = (int)(ea % SL_RA);
                    use = ea / SL_RA;
                    if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(a_full + slot), SL_ABYTES);
                    bulk_load_hint(smem_u32(ringA + slot * SL_ABYTES), p.A + ((size_t)m * p.KT + kt) * SL_ABYTES,
                                   SL_ABYTES, smem_u32(a_full + slot), evict_first);
                    ++na;
                }
            }
        }
    } else if (warp == 1) {
        griddep_wait();
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long ma = 0, mb = 0, nch = 0;
            bool ok = true;
            for (long long u = u0; u < u1 && ok; ++u) {
                const int c = (int)(u % p.CPR);
                const int kt0 = c * SL_CHUNK, kt1 = min(p.KT, kt0 + SL_CHUNK);
                const int buf = (int)(nch & 1);
                if (nch >= 2 &&
                    !mbar_wait(smem_u32(acc_empty + buf), (uint32_t)(((nch >> 1) - 1) & 1), abort_flag))
                    break;
                tc_fence_after();
                const uint32_t dbuf = tmem + (uint32_t)buf * SL_BUF_COLS;
                for (int kt = kt0; kt < kt1; ++kt) {
                    const int sb = (int)(mb % SL_RB), sa = (int)(ma % SL_RA);
                    if (!mbar_wait(smem_u32(b_full + sb), (uint32_t)((mb / SL_RB) & 1), abort_flag) ||
                        !mbar_wait(smem_u32(a_full + sa), (uint32_t)((ma / SL_RA) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t db = desc_sw128(smem_u32(ringB + sb * B_BYTES));
#pragma unroll
                    for (int a = 0; a < SL_NA; ++a) {
                        const uint64_t da = desc_sw128(smem_u32(ringA + sa * SL_ABYTES + a * SL_TILE));
                        const uint32_t dt = dbuf + (uint32_t)(a * QO);
#pragma unroll
                        for (int kk = 0; kk < SL_BK / 16; ++kk) {
                            // slice 0's first step writes all five blocks; every other MMA adds
                            const uint32_t acc = (kt > kt0 || kk > 0 || a > 0) ? 1u : 0u;
                            mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc[a], acc);
                        }
                    }
                    mma_commit(smem_u32(a_empty + sa));
                    mma_commit(smem_u32(b_empty + sb));
                    ++ma;
                    ++mb;
                }
                if (!ok) break;
                mma_commit(smem_u32(acc_full + buf));
                ++nch;
            }
            // every issued MMA must finish before TMEM is released
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else {
        // ------- epilogue warps: accumulator blocks -> 32-bit sums -> Z -------
        const int ew = warp - 2, sub = warp & 3, w4 = ew >> 2;   // TMEM lanes 32 sub .. + 31
        const int row = 32 * sub + lane, q0 = w4 * QPW;
        griddep_wait();
        int seg = p.seg_base[blockIdx.x];
        int acc[SL_DMAX + 1][QPW];
#pragma unroll
        for (int d = 0; d <= SL_DMAX; ++d)
#pragma unroll
            for (int i = 0; i < QPW; ++i) acc[d][i] = 0;
        long long nch = 0;
        for (long long u = u0; u < u1; ++u) {
            const int buf = (int)(nch & 1);
            if (!mbar_wait(smem_u32(acc_full + buf), (uint32_t)((nch >> 1) & 1), abort_flag)) break;
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)buf * SL_BUF_COLS + (uint32_t)q0;
#pragma unroll
            for (int d = 0; d <= SL_DMAX; ++d) {
                uint32_t v[QPW];
#pragma unroll
                for (int i = 0; i < QPW; i += 4) tmem_ld4(ta + (uint32_t)(d * QO + i), v + i);
                tmem_wait4<QPW>(v);
#pragma unroll
                for (int i = 0; i < QPW; ++i) acc[d][i] += __float2int_rn(__uint_as_float(v[i]));
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty + buf));
            ++nch;
            if (u + 1 == u1 || (u + 1) % p.CPR == 0) {   // end of a segment
                long long* out = p.part + ((size_t)seg * QO + q0) * SL_BM + row;
#pragma unroll
                for (int i = 0; i < QPW; ++i) {
                    long long z = 0;
#pragma unroll
                    for (int d = 0; d <= SL_DMAX; ++d) {
                        z += (long long)acc[d][i] * (1LL << (8 * (SL_DMAX - d)));
                        acc[d][i] = 0;
                    }
                    out[(size_t)i * SL_BM] = z;
                }
                ++seg;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        // some role gave up: the latest copy issued into every ring slot must
        // land before the CTA exits
        for (int s = 0; s < SL_RA; ++s) {
            const long long n_s = na > s ? (na - s + SL_RA - 1) / SL_RA : 0;
            if (n_s > 0) mbar_drain(smem_u32(a_full + s), (uint32_t)((n_s - 1) & 1));
        }
        for (int s = 0; s < SL_RB; ++s) {
            const long long n_s = nb > s ? (nb - s + SL_RB - 1) / SL_RB : 0;
            if (n_s > 0) mbar_drain(smem_u32(b_full + s), (uint32_t)((n_s - 1) & 1));
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SL_TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(p.flags, COFEM_FLAG_DEVICE_TIMEOUT);
}

// The 64-bit sum of the segment partials of element r of row tile m, column q.
__device__ __forceinline__ long long seg_sum(const long long* __restrict__ part, const int* __restrict__ grp_seg,
                                             int QO, int q, long long i) {
    const int m = (int)(i >> 7), r = (int)(i & 127);
    const int s0 = grp_seg[2 * m], ns = grp_seg[2 * m + 1];
    long long z = 0;
    for (int s = 0; s < ns; ++s) z += __ldcg(part + ((size_t)(s0 + s) * QO + q) * SL_BM + r);
    return z;
}

// t[q][i] = (Phi~ X)_iq in FP64 (Np rows, zero for q >= Q; the FP8 form's
// rows times s_i^2) and G[q] with
// 2^G >= 4 max_i |t_iq| (one block per column of the padded block).
__global__ __launch_bounds__(1024) void k_sl_finish_t(const long long* __restrict__ part,
                                                      const int* __restrict__ grp_seg, int QO, int Q, long long Np,
                                                      const int* __restrict__ E, const int* __restrict__ F,
                                                      const float* __restrict__ rscale, double* __restrict__ t,
                                                      int* __restrict__ G) {
    __shared__ double sh[32];
    griddep_launch();
    griddep_wait();
    const int q = blockIdx.x;
    double m = 0.0;
    for (long long i = threadIdx.x; i < Np; i += blockDim.x) {
        double v = 0.0;
        if (q < Q) {
            v = ldexp((double)seg_sum(part, grp_seg, QO, q, i), E[i] + F[q] - 48);
            if (rscale) {   // FP8 form: t = s^2 (C X), Phi~^T Phi~ = C^T diag(s^2) C
                const double sc = rscale[i];
                v *= sc * sc;
            }
        }
        t[(size_t)q * Np + i] = v;
        m = fmax(m, fabs(v));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
        G[q] = exp_of(m, 3);
    }
}

// R = B - beta U - alpha (X + Xlo) in FP64 for column q (block (ch, q)), U from
// the second product's partials.  Modes, outputs and norm partials as the
// CUDA-core form's residual kernel (kernels_accurate.cu).
__global__ __launch_bounds__(SL_NT) void k_sl_residual(DevCtl* ctl, int mode, const float* __restrict__ b,
                                                       const float* __restrict__ X, const float* __restrict__ Xlo,
                                                       const long long* __restrict__ part,
                                                       const int* __restrict__ grp_seg, int QO,
                                                       const int* __restrict__ E, const int* __restrict__ G,
                                                       const float* __restrict__ alpha,
                                                       const float* __restrict__ minv, float* __restrict__ Rout,
                                                       long long D, long long Dp, int nch, double* npart) {
    __shared__ double sh[SL_NT / 32];
    griddep_launch();
    griddep_wait();
    const int q = blockIdx.y, ch = blockIdx.x, Q = ctl->Q;
    const bool on = mode == DF_CHECK ? ctl->bnorm2[q] > 0.0 : ctl->active[q] != 0;
    const double beta = ctl->beta;
    double rr = 0.0, rz = 0.0;
    if (on) {
        const size_t off = (size_t)q * Dp;
        const int gq = G[q];
        for (int e = threadIdx.x; e < SL_CH; e += SL_NT) {
            const long long j = (long long)ch * SL_CH + e;
            if (j >= Dp) break;
            double r = 0.0;   // padding beyond D stays zero
            if (j < D) {
                const double u = ldexp((double)seg_sum(part, grp_seg, QO, q, j), E[j] + gq - 48);
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
        npart[(size_t)(0 * Q + q) * nch + ch] = rr;
        if (mode == DF_RR) npart[(size_t)(1 * Q + q) * nch + ch] = rz;
    }
}

// out[q][j] = (Phi~^T Phi~ (X + Xlo))_jq in FP64, j < D (the accurate product alone).
__global__ void k_sl_gram_out(const long long* __restrict__ part, const int* __restrict__ grp_seg, int QO,
                              const int* __restrict__ E, const int* __restrict__ G, long long D,
                              double* __restrict__ out) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int q = blockIdx.y;
    if (j >= D) return;
    out[(size_t)q * D + j] = ldexp((double)seg_sum(part, grp_seg, QO, q, j), E[j] + G[q] - 48);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct SlGemm {
    SlParams p{};
    int nCTA = 0, nseg = 0;
    int* seg_base = nullptr;   // device, nCTA + 1
    int* grp_seg = nullptr;    // device, 2 MT: first segment and count of each row tile
    long long* part = nullptr;
};

struct SlPlan {
    int Q = 0, QO = 0;
    size_t smem = 0;
    uint8_t *A1 = nullptr, *A2 = nullptr;   // slice images of Phi~ and Phi~^T
    int *E1 = nullptr, *E2 = nullptr;       // exponents of the rows of Phi~ (Np) and of its columns (Dp)
    uint8_t *B1 = nullptr, *B2 = nullptr;   // digit images of X (k = Dp) and of t (k = Np)
    int *F = nullptr, *G = nullptr;         // column exponents of X and t (QO each)
    double* t = nullptr;                    // QO x Np
    SlGemm g1, g2;
    long long bytes = 0;
};

template <typename T>
cudaError_t sl_alloc(SlPlan* s, T** p, size_t count, cudaStream_t st) {
    const size_t bytes = std::max<size_t>(16, count * sizeof(T));
    cudaError_t e = cudaMallocAsync((void**)p, bytes, st);
    if (e == cudaSuccess) s->bytes += (long long)bytes;
    else *p = nullptr;
    return e;
}

template <typename T>
void sl_free(T** p, cudaStream_t st) {
    if (*p) cudaFreeAsync(*p, st);
    *p = nullptr;
}

cudaError_t sl_plan_gemm(SlPlan* s, SlGemm& g, int num_sms, int MT, int KT, int QO, unsigned* flags,
                         cudaStream_t st) {
    SlParams& p = g.p;
    p.MT = MT;
    p.KT = KT;
    p.CPR = (KT + SL_CHUNK - 1) / SL_CHUNK;
    p.W = (long long)MT * p.CPR;
    p.QO = QO;
    for (int a = 0; a < SL_NA; ++a) p.idesc[a] = sl_idesc(SL_BM, (SL_NB - a) * QO);
    p.flags = flags;
    g.nCTA = (int)std::max<long long>(1, std::min<long long>(num_sms, p.W / 8));
    // segments: each CTA's unit range split at row-tile boundaries
    std::vector<int> seg_base(g.nCTA + 1), first(MT, -1), count(MT, 0);
    int nseg = 0;
    for (int c = 0; c < g.nCTA; ++c) {
        seg_base[c] = nseg;
        const long long u0 = (long long)c * p.W / g.nCTA, u1 = (long long)(c + 1) * p.W / g.nCTA;
        for (long long u = u0; u < u1;) {
            const int m = (int)(u / p.CPR);
            if (first[m] < 0) first[m] = nseg;
            ++count[m];
            ++nseg;
            u = std::min(u1, (long long)(m + 1) * p.CPR);
        }
    }
    seg_base[g.nCTA] = nseg;
    g.nseg = nseg;
    std::vector<int> grp(2 * (size_t)MT);
    for (int m = 0; m < MT; ++m) {
        grp[2 * m] = first[m];
        grp[2 * m + 1] = count[m];
    }
    cudaError_t e;
    if ((e = sl_alloc(s, &g.seg_base, seg_base.size(), st))) return e;
    if ((e = sl_alloc(s, &g.grp_seg, grp.size(), st))) return e;
    if ((e = sl_alloc(s, &g.part, (size_t)nseg * QO * SL_BM, st))) return e;
    if ((e = cudaMemcpyAsync(g.seg_base, seg_base.data(), seg_base.size() * sizeof(int), cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(g.grp_seg, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;   // the host tables go out of scope
    p.seg_base = g.seg_base;
    p.part = g.part;
    return cudaSuccess;
}

void sl_free_gemm(SlGemm& g, cudaStream_t st) {
    sl_free(&g.seg_base, st);
    sl_free(&g.grp_seg, st);
    sl_free(&g.part, st);
}

size_t sl_smem(int QO) { return 1024 + (size_t)SL_RA * SL_ABYTES + (size_t)SL_RB * SL_NB * QO * 128 + 256; }

void (*sl_gemm_kernel(int QO))(SlParams) {
    return QO <= 16 ? k_sl_gemm<4> : (QO <= 32 ? k_sl_gemm<8> : k_sl_gemm<12>);
}

int ceil_div_i(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace

bool sl_applies(const cofem_ctx* c, int Q) {
    return c->kind == COFEM_OP_DENSE && (c->phi16 != nullptr || c->phi8 != nullptr) &&
           c->opts.residual_path != COFEM_RESIDUAL_FP32_PAIRS &&
           (Q + 15) / 16 * 16 <= SL_QOMAX && c->Np <= SL_KMAX && c->Dp <= SL_KMAX;
}

void sl_release(cofem_ctx* c) {
    SlPlan* s = (SlPlan*)c->sl;
    if (!s) return;
    cudaStream_t st = c->stream;
    sl_free(&s->A1, st);
    sl_free(&s->A2, st);
    sl_free(&s->E1, st);
    sl_free(&s->E2, st);
    sl_free(&s->B1, st);
    sl_free(&s->B2, st);
    sl_free(&s->F, st);
    sl_free(&s->G, st);
    sl_free(&s->t, st);
    sl_free_gemm(s->g1, st);
    sl_free_gemm(s->g2, st);
    c->bytes -= s->bytes;
    delete s;
    c->sl = nullptr;
}

namespace {

// Builds the plan's buffers; every allocation is counted in s->bytes.
cudaError_t sl_build(cofem_ctx* c, SlPlan* s, int Q) {
    cudaStream_t st = c->stream;
    s->Q = Q;
    s->QO = (Q + 15) / 16 * 16;
    const long long Np = c->Np, Dp = c->Dp;
    const int MT1 = (int)(Np / SL_BM), KT1 = (int)(Dp / SL_BK), MT2 = (int)(Dp / SL_BM), KT2 = (int)(Np / SL_BK);
    cudaError_t e;
    if ((e = sl_alloc(s, &s->A1, (size_t)MT1 * KT1 * SL_ABYTES, st))) return e;
    if ((e = sl_alloc(s, &s->A2, (size_t)MT2 * KT2 * SL_ABYTES, st))) return e;
    if ((e = sl_alloc(s, &s->E1, (size_t)Np, st))) return e;
    if ((e = sl_alloc(s, &s->E2, (size_t)Dp, st))) return e;
    if ((e = sl_alloc(s, &s->B1, (size_t)KT1 * SL_NB * s->QO * 128, st))) return e;
    if ((e = sl_alloc(s, &s->B2, (size_t)KT2 * SL_NB * s->QO * 128, st))) return e;
    if ((e = sl_alloc(s, &s->F, (size_t)s->QO, st))) return e;
    if ((e = sl_alloc(s, &s->G, (size_t)s->QO, st))) return e;
    if ((e = sl_alloc(s, &s->t, (size_t)s->QO * Np, st))) return e;
    unsigned* cmax = nullptr;   // column maxima of the dictionary (set-up scratch)
    if ((e = cudaMallocAsync((void**)&cmax, (size_t)Dp * sizeof(unsigned), st))) return e;
    e = cudaMemsetAsync(cmax, 0, (size_t)Dp * sizeof(unsigned), st);
    if (e == cudaSuccess) {
        const int rpb = 256;   // rows per block of the column maxima
        const dim3 gcm((unsigned)ceil_div_i(Dp, 256), (unsigned)ceil_div_i(Np, rpb));
        if (c->phi16) {
            k_sl_row_exp<<<(unsigned)Np, 256, 0, st>>>(c->phi16, Dp, s->E1);
            k_sl_col_max<<<gcm, 256, 0, st>>>(c->phi16, Np, Dp, rpb, cmax);
        } else {
            k_sl_row_exp<<<(unsigned)Np, 256, 0, st>>>(c->phi8, Dp, s->E1);
            k_sl_col_max<<<gcm, 256, 0, st>>>(c->phi8, Np, Dp, rpb, cmax);
        }
        k_sl_col_exp<<<(unsigned)ceil_div_i(Dp, 256), 256, 0, st>>>(cmax, Dp, s->E2);
        if (c->phi16) {
            k_sl_tile_rows<<<dim3((unsigned)KT1, (unsigned)MT1), 128, 0, st>>>(c->phi16, Dp, KT1, s->E1, s->A1);
            k_sl_tile_cols<<<dim3((unsigned)KT2, (unsigned)MT2), 128, 0, st>>>(c->phi16, Dp, KT2, s->E2, s->A2);
        } else {
            k_sl_tile_rows<<<dim3((unsigned)KT1, (unsigned)MT1), 128, 0, st>>>(c->phi8, Dp, KT1, s->E1, s->A1);
            k_sl_tile_cols<<<dim3((unsigned)KT2, (unsigned)MT2), 128, 0, st>>>(c->phi8, Dp, KT2, s->E2, s->A2);
        }
        e = cudaGetLastError();
    }
    cudaFreeAsync(cmax, st);
    if (e) return e;
    if ((e = sl_plan_gemm(s, s->g1, c->num_sms, MT1, KT1, s->QO, &c->ctl->flags, st))) return e;
    if ((e = sl_plan_gemm(s, s->g2, c->num_sms, MT2, KT2, s->QO, &c->ctl->flags, st))) return e;
    s->g1.p.A = s->A1;
    s->g1.p.B = s->B1;
    s->g2.p.A = s->A2;
    s->g2.p.B = s->B2;
    s->smem = sl_smem(s->QO);
    return cudaStreamSynchronize(st);
}

}  // namespace

// Slice images of the dictionary and its transpose, the digit images and the
// segment tables of both products for Q columns.
cudaError_t sl_setup(cofem_ctx* c, int Q) {
    sl_release(c);
    SlPlan* s = new SlPlan();
    c->sl = s;
    const cudaError_t e = sl_build(c, s, Q);
    c->bytes += s->bytes;   // sl_release takes them off again
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        sl_release(c);
    }
    return e;
}

cudaError_t sl_kernel_attributes(int max_smem) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_sl_gemm<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    if ((e = cudaFuncSetAttribute(k_sl_gemm<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))) return e;
    return cudaFuncSetAttribute(k_sl_gemm<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

int sl_kernels() { return 7; }

// Digits of X and the first product (Phi~ X as segment partials).
void launch_sl_first_product(Sink& s, cofem_ctx* c, int Q) {
    SlPlan* p = (SlPlan*)c->sl;
    const int QO = p->QO;
    s.launch(k_sl_colexp, dim3(QO), dim3(1024), 0, c->X, c->Dp, c->Dp, Q, p->F);
    s.launch_pdl(k_sl_digits<true>, dim3((unsigned)ceil_div_i(c->Dp / 8, 256), QO), dim3(256), 0, c->X, c->Xlo,
                 (const double*)nullptr, c->Dp, c->Dp, Q, QO, p->F, p->B1);
    s.launch_pdl(sl_gemm_kernel(QO), dim3(p->g1.nCTA), dim3(SL_THREADS), p->smem, p->g1.p);
}

// Both products: the second one's partials and G are left for the residual.
void launch_sl_products(Sink& s, cofem_ctx* c, int Q) {
    SlPlan* p = (SlPlan*)c->sl;
    const int QO = p->QO;
    launch_sl_first_product(s, c, Q);
    s.launch_pdl(k_sl_finish_t, dim3(QO), dim3(1024), 0, p->g1.part, p->g1.grp_seg, QO, Q, c->Np, p->E1, p->F,
                 c->phi8 ? (const float*)c->scale8 : (const float*)nullptr, p->t,
                 p->G);
    s.launch_pdl(k_sl_digits<false>, dim3((unsigned)ceil_div_i(c->Np / 8, 256), QO), dim3(256), 0,
                 (const float*)nullptr, (const float*)nullptr, p->t, c->Np, c->Np, Q, QO, p->G, p->B2);
    s.launch_pdl(sl_gemm_kernel(QO), dim3(p->g2.nCTA), dim3(SL_THREADS), p->smem, p->g2.p);
}

void launch_sl_residual(Sink& s, cofem_ctx* c, int Q, int mode) {
    SlPlan* p = (SlPlan*)c->sl;
    // plain launches, not programmatic ones: in the fit graph at 8192 x 32768
    // (K = 32) the residual's kernels took 0.748 ms with programmatic edges
    // between them and 0.641 ms without (same bits)
    const bool pdl = s.pdl;
    s.pdl = false;
    launch_sl_products(s, c, Q);
    s.launch_pdl(k_sl_residual, dim3(c->nch, Q), dim3(SL_NT), 0, c->ctl, mode, c->b, c->X, c->Xlo, p->g2.part,
                 p->g2.grp_seg, p->QO, p->E2, p->G, c->alpha, c->minv, mode == DF_RR ? c->R : c->Rt, c->D, c->Dp,
                 c->nch, c->part);
    s.pdl = pdl;
}

void launch_sl_gram(Sink& s, cofem_ctx* c, int Q, double* out) {
    SlPlan* p = (SlPlan*)c->sl;
    launch_sl_products(s, c, Q);
    s.launch(k_sl_gram_out, dim3((unsigned)ceil_div_i(c->D, 256), Q), dim3(256), 0, p->g2.part, p->g2.grp_seg,
             p->QO, p->E2, p->G, c->D, out);
}
