// Dense operator for a BF16 dictionary on the 5th-generation tensor cores
// (tcgen05.mma, TMA, TMEM): A V = beta Phi~^T (Phi~ V) + diag(alpha) V with
// Phi~ = bf16(Phi) (Alg. 2 "Apply matrix", Sec. III-B).
//
// Both products are the same skinny GEMM, D[rows x Q] = A[rows x K] * B[Q x K]^T:
//   GEMM1: A = Phi~   (Np x Dp),  B = split(V)   -> T  = Phi~ V       (Np x Q)
//   GEMM2: A = Phi~^T (Dp x Np),  B = split(T)   -> U  = Phi~^T T     (Dp x Q)
// Phi~^T is a second copy made once at create time, so that both A operands
// are K-major (contiguous along the reduction).  The FP32 right-hand blocks are
// split into three bfloat16 terms v = hi + mid + lo (24 significant bits);
// bf16 x bf16 products are exact in the FP32 accumulator, so the operator is
// applied to the quantised dictionary at FP32 accuracy.  Term t of column q is
// B row 3q + t; the epilogue adds the three accumulator columns back.
//
// The GEMM kernel is persistent (one CTA per SM) and stream-K: the work units
// (group of G row tiles of 128 rows, one 64-wide k tile) are split into equal
// contiguous ranges, one per CTA; the B tile of a k step is reused by the G A
// tiles of the group (G accumulators = all 512 TMEM columns).  A range crosses
// at most a few group boundaries; each (CTA, group) segment writes a partial
// sum, and a small kernel adds the partials of each group in a fixed order.
//
// Warp roles (192 threads): warp 0 lane 0 issues TMA loads, warp 1 allocates
// TMEM and lane 0 issues the MMAs, warps 2-5 drain TMEM (each its 32-lane
// sub-partition).  Every mbarrier wait is bounded: on timeout the kernel sets
// COFEM_FLAG_DEVICE_TIMEOUT, waits (bounded) for its in-flight copies and MMAs,
// frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "cofem_internal.cuh"

namespace {

constexpr int TC_BM = 128, TC_BK = 64;
constexpr int TC_NA = 8, TC_NB = 3;
constexpr int TC_THREADS = 192;
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcParams {
    long long W;          // work units = groups * K_tiles
    int K_tiles;          // 64-wide k tiles
    int M_tiles;          // 128-row tiles
    int G;                // row tiles per group
    int acc_stride;       // TMEM columns per accumulator
    int QS;               // MMA N (3 Q rounded up to 16)
    int Q;                // output columns
    uint32_t idesc;       // tcgen05 instruction descriptor
    const int* seg_base;  // first segment id of each CTA
    float* part;          // [segment][Q][G * 128]
    unsigned* flags;      // error flag word (DevCtl::flags)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.b32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the completion of the phase with the given parity.  Returns
// false on timeout (and raises the block's abort flag) or when another role
// has already aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
    for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 127) == 127) {
            if (*abort_flag) return false;
            __nanosleep(64);
        }
    }
    *abort_flag = 1;
    return false;
}
// Bounded wait that ignores the abort flag (used to drain in-flight work).
__device__ __noinline__ void mbar_drain(uint32_t bar, uint32_t parity) {
    for (uint32_t i = 0; i < TC_WAIT_LIMIT; ++i) {
        if (mbar_try(bar, parity)) return;
        if ((i & 127) == 127) __nanosleep(64);
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row core-matrix groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
// Registers written by tcgen05.ld are valid only after tcgen05.wait::ld; the
// empty asm statements re-define them after the wait so no use moves above it.
__device__ __forceinline__ void tmem_ld_wait(uint32_t* r, int n) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    for (int i = 0; i < n; i += 8)
        asm volatile("" : "+r"(r[i]), "+r"(r[i + 1]), "+r"(r[i + 2]), "+r"(r[i + 3]), "+r"(r[i + 4]),
                     "+r"(r[i + 5]), "+r"(r[i + 6]), "+r"(r[i + 7]));
}

__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, TcParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)p.QS * 128u;
    uint8_t* ringA = smem;
    uint8_t* ringB = smem + TC_NA * TC_A_BYTES;
    uint64_t* bars = (uint64_t*)(ringB + TC_NB * B_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + TC_NA;
    uint64_t* b_full = bars + 2 * TC_NA;
    uint64_t* b_empty = bars + 2 * TC_NA + TC_NB;
    uint64_t* acc_full = bars + 2 * TC_NA + 2 * TC_NB;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 3);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < TC_NA; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), 1);
        }
        for (int i = 0; i < TC_NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(acc_empty), 4);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    const long long u0 = (long long)blockIdx.x * p.W / gridDim.x;
    const long long u1 = (long long)(blockIdx.x + 1) * p.W / gridDim.x;
    long long na = 0, nb = 0;   // TMA loads issued into the A and B rings (producer thread)

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapA) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&mapB) : "memory");
            for (long long u = u0; u < u1; ++u) {
                const int g = (int)(u / p.K_tiles), k = (int)(u % p.K_tiles);
                const int valid = min(p.G, p.M_tiles - g * p.G);
                int slot = (int)(nb % TC_NB);
                long long use = nb / TC_NB;
                if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) break;
                mbar_expect_tx(smem_u32(b_full + slot), B_BYTES);
                tma_load_2d(smem_u32(ringB + slot * B_BYTES), &mapB, k * TC_BK, 0, smem_u32(b_full + slot));
                ++nb;
                bool ok = true;
                for (int r = 0; r < valid; ++r) {
                    slot = (int)(na % TC_NA);
                    use = na / TC_NA;
                    if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(a_full + slot), TC_A_BYTES);
                    tma_load_2d(smem_u32(ringA + slot * TC_A_BYTES), &mapA, k * TC_BK, (g * p.G + r) * TC_BM,
                                smem_u32(a_full + slot));
                    ++na;
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long ma = 0, mb = 0;   // ring positions consumed
            int nseg = 0;
            long long u = u0;
            bool ok = true;
            while (u < u1 && ok) {
                const int g = (int)(u / p.K_tiles);
                const long long seg_end = min(u1, (long long)(g + 1) * p.K_tiles);
                const int valid = min(p.G, p.M_tiles - g * p.G);
                if (nseg > 0 && !mbar_wait(smem_u32(acc_empty), (uint32_t)((nseg - 1) & 1), abort_flag)) break;
                tc_fence_after();
                const long long seg_start = u;
                for (; u < seg_end; ++u) {
                    const int sb = (int)(mb % TC_NB);
                    if (!mbar_wait(smem_u32(b_full + sb), (uint32_t)((mb / TC_NB) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint64_t db = desc_sw128(smem_u32(ringB + sb * B_BYTES));
                    for (int r = 0; r < valid; ++r) {
                        const int sa = (int)(ma % TC_NA);
                        if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((ma / TC_NA) & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t da = desc_sw128(smem_u32(ringA + sa * TC_A_BYTES));
                        const uint32_t dt = tmem + (uint32_t)(r * p.acc_stride);
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk)
                            mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc,
                                     (u > seg_start || kk > 0) ? 1u : 0u);
                        mma_commit(smem_u32(a_empty + sa));
                        ++ma;
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(b_empty + sb));
                    ++mb;
                }
                if (!ok) break;
                mma_commit(smem_u32(acc_full));
                ++nseg;
            }
            // every issued MMA must finish before TMEM is released
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else {
        // ---------------- epilogue: TMEM -> partial sums ----------------
        const int sub = warp & 3;
        const int GR = p.G * TC_BM;
        const int NC = p.QS / 16;
        int nseg = 0;
        long long u = u0;
        while (u < u1) {
            const int g = (int)(u / p.K_tiles);
            const long long seg_end = min(u1, (long long)(g + 1) * p.K_tiles);
            const int valid = min(p.G, p.M_tiles - g * p.G);
            if (!mbar_wait(smem_u32(acc_full), (uint32_t)(nseg & 1), abort_flag)) break;
            tc_fence_after();
            float* out = p.part + (size_t)(p.seg_base[blockIdx.x] + nseg) * p.Q * GR;
            const int row = 32 * sub + lane;
            for (int r = 0; r < valid; ++r) {
                const uint32_t tbase = tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(r * p.acc_stride);
                for (int qb = 0; qb * 16 < p.Q; ++qb) {
                    uint32_t v[48];
                    const int c0 = 3 * qb;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        if (c0 + c < NC) tmem_ld16(tbase + (uint32_t)((c0 + c) * 16), v + 16 * c);
                    tmem_ld_wait(v, 48);
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int q = 16 * qb + i;
                        if (q < p.Q)
                            out[(size_t)q * GR + r * TC_BM + row] =
                                __uint_as_float(v[3 * i]) + __uint_as_float(v[3 * i + 1]) +
                                __uint_as_float(v[3 * i + 2]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty));
            ++nseg;
            u = seg_end;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        // some role gave up: the latest load issued into every ring slot must
        // land before the CTA exits
        for (int s = 0; s < TC_NA; ++s) {
            const long long n_s = na > s ? (na - s + TC_NA - 1) / TC_NA : 0;
            if (n_s > 0) mbar_drain(smem_u32(a_full + s), (uint32_t)((n_s - 1) & 1));
        }
        for (int s = 0; s < TC_NB; ++s) {
            const long long n_s = nb > s ? (nb - s + TC_NB - 1) / TC_NB : 0;
            if (n_s > 0) mbar_drain(smem_u32(b_full + s), (uint32_t)((n_s - 1) & 1));
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
    if (threadIdx.x == 0 && *abort_flag) atomicOr(p.flags, COFEM_FLAG_DEVICE_TIMEOUT);
}

// v = hi + mid + lo with hi = bf16(v), mid = bf16(v - hi), lo = bf16(v - hi - mid)
__device__ __forceinline__ void split3(float v, __nv_bfloat16& a, __nv_bfloat16& b, __nv_bfloat16& c) {
    a = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(a);
    b = __float2bfloat16_rn(r1);
    c = __float2bfloat16_rn(r1 - __bfloat162float(b));
}

// Vs (QS x ld, bf16), row 3q + t = term t of column q of V (Q x Dp, FP32).
__global__ void k_split3(const float* __restrict__ V, long long Dp, __nv_bfloat16* __restrict__ Vs, long long ld) {
    const int q = blockIdx.y;
    const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j >= Dp) return;
    const float4 v = *reinterpret_cast<const float4*>(V + (size_t)q * Dp + j);
    __nv_bfloat16 t[3][4];
    split3(v.x, t[0][0], t[1][0], t[2][0]);
    split3(v.y, t[0][1], t[1][1], t[2][1]);
    split3(v.z, t[0][2], t[1][2], t[2][2]);
    split3(v.w, t[0][3], t[1][3], t[2][3]);
#pragma unroll
    for (int k = 0; k < 3; ++k)
        *reinterpret_cast<uint2*>(Vs + (size_t)(3 * q + k) * ld + j) = *reinterpret_cast<const uint2*>(t[k]);
}

// GEMM1 epilogue: T = sum of the segment partials of its group (fixed order),
// split into bf16 terms for GEMM2, and ||T_q||^2 partials -> pi, gamma.
__global__ __launch_bounds__(256) void k_tc_reduce_T(const float* __restrict__ part, const int* __restrict__ grp_seg,
                                                     int GR, int Q, long long Np, __nv_bfloat16* __restrict__ Ts,
                                                     double* tt_part, int nblk, unsigned* counter, DevCtl* ctl,
                                                     int mode) {
    __shared__ double sh[8];
    const int q = blockIdx.y;
    const long long i = (long long)blockIdx.x * 1024 + threadIdx.x * 4;
    double tt = 0.0;
    if (i < Np) {
        const int g = (int)(i / GR), r = (int)(i % GR);
        const int s0 = grp_seg[2 * g], ns = grp_seg[2 * g + 1];
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int s = 0; s < ns; ++s) {
            const float4 b = *reinterpret_cast<const float4*>(part + ((size_t)(s0 + s) * Q + q) * GR + r);
            a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
        }
        __nv_bfloat16 t[3][4];
        split3(a.x, t[0][0], t[1][0], t[2][0]);
        split3(a.y, t[0][1], t[1][1], t[2][1]);
        split3(a.z, t[0][2], t[1][2], t[2][2]);
        split3(a.w, t[0][3], t[1][3], t[2][3]);
#pragma unroll
        for (int k = 0; k < 3; ++k)
            *reinterpret_cast<uint2*>(Ts + (size_t)(3 * q + k) * Np + i) = *reinterpret_cast<const uint2*>(t[k]);
        tt = (double)a.x * a.x + (double)a.y * a.y + (double)a.z * a.z + (double)a.w * a.w;
    }
    tt = block_sum(tt, sh);
    if (threadIdx.x == 0) tt_part[(size_t)q * nblk + blockIdx.x] = tt;
    if (!last_block_arrive(counter, gridDim.x * gridDim.y)) return;
    op_finalize_block(ctl, tt_part, nblk, Q, mode);
}

// GEMM2 epilogue: U (Q x Dp) = sum of the segment partials of its group.
__global__ __launch_bounds__(256) void k_tc_reduce_U(const float* __restrict__ part, const int* __restrict__ grp_seg,
                                                     int GR, int Q, long long Dp, float* __restrict__ U) {
    const int q = blockIdx.y;
    const long long j = (long long)blockIdx.x * 1024 + threadIdx.x * 4;
    if (j >= Dp) return;
    const int g = (int)(j / GR), r = (int)(j % GR);
    const int s0 = grp_seg[2 * g], ns = grp_seg[2 * g + 1];
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int s = 0; s < ns; ++s) {
        const float4 b = *reinterpret_cast<const float4*>(part + ((size_t)(s0 + s) * Q + q) * GR + r);
        a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
    }
    *reinterpret_cast<float4*>(U + (size_t)q * Dp + j) = a;
}

// dst (cols x rows) = src^T (rows x cols), bf16, 32 x 32 tiles.
__global__ void k_transpose_bf16(const __nv_bfloat16* __restrict__ src, long long rows, long long cols,
                                 __nv_bfloat16* __restrict__ dst) {
    __shared__ __nv_bfloat16 tile[32][33];
    const long long c0 = (long long)blockIdx.x * 32, r0 = (long long)blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = src[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[c * rows + r] = tile[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encoder() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
    }
    return fn;
}

// 2-D bf16 row-major matrix (rows x cols, leading dimension ld elements),
// box = box_rows x 64 columns, 128-byte swizzle.
bool encode_map(CUtensorMap* m, const void* base, long long rows, long long cols, long long ld, int box_rows) {
    EncodeTiledFn enc = get_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

struct GemmPlan {
    TcParams p{};
    int nCTA = 0;
    int nseg = 0, groups = 0;
    int* seg_base = nullptr;   // device
    int* grp_seg = nullptr;    // device
    float* part = nullptr;     // device
    CUtensorMap mapA, mapB;
};

struct TcPlan {
    int Q = 0, QS = 0, G = 0;
    size_t smem = 0;
    __nv_bfloat16* Vs = nullptr;   // QS x Dp
    __nv_bfloat16* Ts = nullptr;   // QS x Np
    GemmPlan g1, g2;
    long long bytes = 0;
};

constexpr uint32_t make_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

cudaError_t plan_gemm(GemmPlan& gp, int num_sms, long long M_rows, long long K_cols, int G, int acc_stride, int QS,
                      int Q, unsigned* flags, long long* bytes) {
    TcParams& p = gp.p;
    p.M_tiles = (int)((M_rows + TC_BM - 1) / TC_BM);
    p.K_tiles = (int)((K_cols + TC_BK - 1) / TC_BK);
    p.G = G;
    p.acc_stride = acc_stride;
    p.QS = QS;
    p.Q = Q;
    p.idesc = make_idesc(TC_BM, QS);
    p.flags = flags;
    gp.groups = (p.M_tiles + G - 1) / G;
    p.W = (long long)gp.groups * p.K_tiles;
    gp.nCTA = (int)std::min<long long>(num_sms, p.W);
    // segments: each CTA's unit range split at group boundaries
    std::vector<int> seg_base(gp.nCTA + 1), grp_first(gp.groups, -1), grp_count(gp.groups, 0);
    int nseg = 0;
    for (int c = 0; c < gp.nCTA; ++c) {
        seg_base[c] = nseg;
        const long long u0 = (long long)c * p.W / gp.nCTA, u1 = (long long)(c + 1) * p.W / gp.nCTA;
        long long u = u0;
        while (u < u1) {
            const int g = (int)(u / p.K_tiles);
            if (grp_first[g] < 0) grp_first[g] = nseg;
            ++grp_count[g];
            ++nseg;
            u = std::min(u1, (long long)(g + 1) * p.K_tiles);
        }
    }
    seg_base[gp.nCTA] = nseg;
    gp.nseg = nseg;
    std::vector<int> grp(2 * gp.groups);
    for (int g = 0; g < gp.groups; ++g) {
        grp[2 * g] = grp_first[g];
        grp[2 * g + 1] = grp_count[g];
    }
    cudaError_t e;
    if ((e = cudaMalloc(&gp.seg_base, seg_base.size() * sizeof(int)))) return e;
    if ((e = cudaMalloc(&gp.grp_seg, grp.size() * sizeof(int)))) return e;
    const size_t part_elems = (size_t)nseg * Q * G * TC_BM;
    if ((e = cudaMalloc(&gp.part, part_elems * sizeof(float)))) return e;
    *bytes += (long long)(seg_base.size() + grp.size()) * 4 + (long long)part_elems * 4;
    if ((e = cudaMemcpy(gp.seg_base, seg_base.data(), seg_base.size() * sizeof(int), cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(gp.grp_seg, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice))) return e;
    p.seg_base = gp.seg_base;
    p.part = gp.part;
    return cudaSuccess;
}

void free_gemm(GemmPlan& gp) {
    if (gp.seg_base) cudaFree(gp.seg_base);
    if (gp.grp_seg) cudaFree(gp.grp_seg);
    if (gp.part) cudaFree(gp.part);
    gp.seg_base = gp.grp_seg = nullptr;
    gp.part = nullptr;
}

}  // namespace

void tc_release(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    if (!t) return;
    free_gemm(t->g1);
    free_gemm(t->g2);
    if (t->Vs) cudaFree(t->Vs);
    if (t->Ts) cudaFree(t->Ts);
    c->bytes -= t->bytes;
    delete t;
    c->tc = nullptr;
}

cudaError_t tc_setup(cofem_ctx* c, int Q) {
    tc_release(c);
    TcPlan* t = new TcPlan();
    c->tc = t;
    t->Q = Q;
    t->QS = ((3 * Q + 15) / 16) * 16;
    int acc_stride;
    if (t->QS <= 128) {
        t->G = 4;
        acc_stride = 128;
    } else {
        t->G = 2;
        acc_stride = 256;
    }
    cudaError_t e;
    unsigned* flags = &c->ctl->flags;
    if ((e = plan_gemm(t->g1, c->num_sms, c->Np, c->Dp, t->G, acc_stride, t->QS, Q, flags, &t->bytes))) return e;
    if ((e = plan_gemm(t->g2, c->num_sms, c->Dp, c->Np, t->G, acc_stride, t->QS, Q, flags, &t->bytes))) return e;
    if ((e = cudaMalloc(&t->Vs, (size_t)t->QS * c->Dp * 2))) return e;
    if ((e = cudaMalloc(&t->Ts, (size_t)t->QS * c->Np * 2))) return e;
    t->bytes += (long long)t->QS * (c->Dp + c->Np) * 2;
    c->bytes += t->bytes;
    if ((e = cudaMemset(t->Vs, 0, (size_t)t->QS * c->Dp * 2))) return e;
    if ((e = cudaMemset(t->Ts, 0, (size_t)t->QS * c->Np * 2))) return e;
    if (!encode_map(&t->g1.mapA, c->phi16, c->Np, c->Dp, c->Dp, TC_BM) ||
        !encode_map(&t->g1.mapB, t->Vs, t->QS, c->Dp, c->Dp, t->QS) ||
        !encode_map(&t->g2.mapA, c->phiT16, c->Dp, c->Np, c->Np, TC_BM) ||
        !encode_map(&t->g2.mapB, t->Ts, t->QS, c->Np, c->Np, t->QS))
        return cudaErrorInvalidValue;
    t->smem = 1024 + (size_t)TC_NA * TC_A_BYTES + (size_t)TC_NB * t->QS * 128 + 256;
    return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
}

cudaError_t tc_make_transpose(cofem_ctx* c, cudaStream_t st) {
    const dim3 grid((unsigned)(c->Dp / 32), (unsigned)(c->Np / 32));
    k_transpose_bf16<<<grid, dim3(32, 8), 0, st>>>(c->phi16, c->Np, c->Dp, c->phiT16);
    return cudaGetLastError();
}

void launch_tc_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    TcPlan* t = (TcPlan*)c->tc;
    s.launch(k_split3, dim3((unsigned)((c->Dp / 4 + 255) / 256), Q), dim3(256), 0, V, c->Dp, t->Vs, c->Dp);
    s.launch(k_gemm_tc, dim3(t->g1.nCTA), dim3(TC_THREADS), t->smem, t->g1.mapA, t->g1.mapB, t->g1.p);
    const int nblk = (int)((c->Np + 1023) / 1024);
    s.launch(k_tc_reduce_T, dim3(nblk, Q), dim3(256), 0, t->g1.part, t->g1.grp_seg, t->G * TC_BM, Q, c->Np, t->Ts,
             c->tt_part, nblk, c->counters + 8, c->ctl, mode);
    s.launch(k_gemm_tc, dim3(t->g2.nCTA), dim3(TC_THREADS), t->smem, t->g2.mapA, t->g2.mapB, t->g2.p);
    s.launch(k_tc_reduce_U, dim3((unsigned)((c->Dp + 1023) / 1024), Q), dim3(256), 0, t->g2.part, t->g2.grp_seg,
             t->G * TC_BM, Q, c->Dp, c->U);
}
