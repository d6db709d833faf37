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
// Memory layout: the library's copies of Phi~ and Phi~^T are stored pre-tiled,
// each 128 x 64 tile as the exact 128-byte-swizzled shared-memory image the
// MMA reads (16 KiB contiguous), tiles ordered (group, k tile, row tile), so the
// range of work units of one CTA is one contiguous run of HBM, fetched with 1-D
// bulk copies.  The B operands (split vector blocks) are written in the same
// per-k-tile swizzled image by the kernels that produce them.
//
// The GEMM kernel is persistent (one CTA per SM) and stream-K: the work units
// (group of G row tiles of 128 rows, one 64-wide k tile) are split into equal
// contiguous ranges, one per CTA; the B tile of a k step is reused by the G A
// tiles of the group (G accumulators = all 512 TMEM columns).  A range crosses
// at most a few group boundaries; each (CTA, group) segment writes a partial
// sum, and a small kernel adds the partials of each group in a fixed order.
//
// Warp roles: warp 0 lane 0 issues the bulk copies, warp 1 allocates TMEM and
// lane 0 issues the MMAs, and the epilogue warps (16 in the BF16 form, 8 in the
// TF32 form; warp id mod 4 selects the 32-lane TMEM sub-partition) drain the
// accumulators, four of them first splitting the TF32 tiles.  (The FP8 kernel
// further down has its own roles.)  Every mbarrier wait is bounded: on timeout the kernel sets
// COFEM_FLAG_DEVICE_TIMEOUT, waits (bounded) for its in-flight copies and MMAs,
// frees TMEM and returns.
#include <algorithm>
#include <vector>

#include "cofem_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_BM = 128, TC_BK = 64;   // BF16 tile: 128 rows x 64 bf16 (128-byte rows)
constexpr int TC_BK32 = 32;               // TF32 tile: 128 rows x 32 fp32 (128-byte rows)
constexpr int TC_NA = 8, TC_NB = 3;
constexpr int TC_NLO = 3;   // TF32: Phi_lo tiles in a ring of their own
// Epilogue warps: four (one per TMEM sub-partition) convert the TF32 tiles;
// all of them drain the accumulators, the warps of a sub-partition splitting
// the row tiles.  (Eight converter warps instead of four left the 3xTF32
// operator as it was, 0.717 against 0.708 ms at 8192 x 32768: the split is not
// what paces it.)  A lone warp per scheduler drained a 4-tile segment in ~6 us
// (dependent TMEM load -> add -> store chains at one warp's issue rate).
constexpr int tc_epi_warps(bool tf) { return tf ? 8 : 16; }
constexpr int tc_threads(bool tf) { return 64 + 32 * tc_epi_warps(tf); }
constexpr uint32_t TC_A_BYTES = TC_BM * TC_BK * 2;
constexpr uint32_t TC_TMEM_COLS = 512;

struct TcParams {
    const void* A;        // tiled A image: unit u, row tile r at byte (u * G + r) * 16384
    const void* B;        // tiled B image: k tile at byte k * QS * 128
    long long W;          // work units = groups * K_tiles
    int K_tiles;          // 64-wide k tiles
    int M_tiles;          // 128-row tiles
    int G;                // row tiles per group
    int acc_stride;       // TMEM columns per accumulator
    int QS;               // MMA N (3 Q rounded up to 16)
    int Q;                // output columns
    uint32_t idesc;       // tcgen05 instruction descriptor (N = QS)
    uint32_t idesc_lo;    // TF32: descriptor of the Phi_lo product (N = QH)
    int QH;               // TF32: row of the first P_lo term in B
    const int* seg_base;  // first segment id of each CTA
    float* part;          // [segment][Q][G * 128]
    unsigned* flags;      // error flag word (DevCtl::flags)
    const DevCtl* defer;  // the CG step's first product in a fit graph's loop: skipped at replacement steps
};

// The first product of a CG step that a fit graph's loop defers past a
// residual replacement (it runs again after the replacement, outside the
// loop): the launch does nothing.  Read after the programmatic wait.
__device__ __forceinline__ bool gemm_deferred(const TcParams& p) { return p.defer && rr_step(p.defer); }

// TMEM -> segment partials for one epilogue warp: accumulator r (r0 <= r <
// valid, step rstep) holds, in this warp's 32 TMEM lanes (rows), the split
// terms of every output column (BF16: columns 3q..3q+2; TF32: q and QH + q);
// their sum goes to out[q * GR + r * 128 + row].
template <bool TF>
__device__ __forceinline__ void drain_tmem(uint32_t tbase, int r0, int rstep, int valid, int acc_stride, int Q,
                                           int QH, int NC, int GR, float* out, int row) {
    for (int r = r0; r < valid; r += rstep) {
        const uint32_t tb = tbase + (uint32_t)(r * acc_stride);
        for (int qb = 0; qb * 16 < Q; ++qb) {
            uint32_t v[48];
            if (TF) {
                tmem_ld16(tb + (uint32_t)(qb * 16), v);
                tmem_ld16(tb + (uint32_t)(QH + qb * 16), v + 16);
                tmem_ld_wait(v, 32);
            } else {
                const int c0 = 3 * qb;
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (c0 + c < NC) tmem_ld16(tb + (uint32_t)((c0 + c) * 16), v + 16 * c);
                tmem_ld_wait(v, 48);
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int q = 16 * qb + i;
                if (q < Q) {
                    const float val = TF ? __uint_as_float(v[i]) + __uint_as_float(v[16 + i])
                                         : __uint_as_float(v[3 * i]) + __uint_as_float(v[3 * i + 1]) +
                                               __uint_as_float(v[3 * i + 2]);
                    out[(size_t)q * GR + r * TC_BM + row] = val;
                }
            }
        }
    }
}

// Tensor-core skinny GEMM.  TF = false: A, B bf16 (B = 3-term split), one MMA
// chain per tile.  TF = true: A, B fp32 read as TF32 (B = [P_hi | P_lo]); the
// epilogue warps round each A tile to Phi_hi = tf32_rn(A) in place and write
// Phi_lo = tf32_rn(A - Phi_hi) into a ring of its own (TC_NLO tiles, so that
// the A ring holds whole units fetched by one 64 KiB copy, as in the BF16
// form: 0.657 against 0.707 ms per application at 8192 x 32768 with single
// tiles and Phi_lo beside each), and a second MMA chain adds Phi_lo [P_hi |
// P_lo] into the same accumulator columns (all four products).
template <bool TF>
__global__ void __launch_bounds__(tc_threads(TF), 1) k_gemm_tc(TcParams p) {
    constexpr int NA = TC_NA;
    constexpr int KE = TF ? TC_BK32 : TC_BK;    // elements per 128-byte tile row
    // A-ring element: the G row tiles of a unit, fetched as one bulk copy (a
    // copy costs a fixed ~0.3 us of issue time, so fewer, larger copies keep
    // the stream at HBM rate); TF32 converts it tile by tile, Phi_lo into a
    // ring of its own
    const int EPT = p.G;
    const int NE = NA / p.G;                     // ring elements
    const uint32_t E_BYTES = (uint32_t)EPT * TC_A_BYTES;
    constexpr int KM = TF ? 8 : 16;             // K of one MMA instruction
    griddep_launch();   // the next kernel may start its prologue; it waits for this grid's completion
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)p.QS * 128u;
    uint8_t* ringA = smem;
    uint8_t* ringL = smem + NA * TC_A_BYTES;                      // TF32 only: Phi_lo tiles
    uint8_t* ringB = ringL + (TF ? TC_NLO * TC_A_BYTES : 0);
    uint64_t* bars = (uint64_t*)(ringB + TC_NB * B_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + NA;
    uint64_t* lo_full = bars + 2 * NA;                            // TF32 only [TC_NLO]
    uint64_t* lo_empty = lo_full + TC_NLO;                        // TF32 only [TC_NLO]
    uint64_t* b_full = lo_empty + TC_NLO;
    uint64_t* b_empty = b_full + TC_NB;
    uint64_t* acc_full = b_empty + TC_NB;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 3);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), 1);
        }
        for (int i = 0; i < TC_NLO; ++i) {
            mbar_init(smem_u32(lo_full + i), 4);
            mbar_init(smem_u32(lo_empty + i), 1);
        }
        for (int i = 0; i < TC_NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(acc_empty), tc_epi_warps(TF));
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
    long long u1 = (long long)(blockIdx.x + 1) * p.W / gridDim.x;   // u0 when the launch is deferred
    long long na = 0, nb = 0;   // bulk loads issued into the A and B rings (producer thread)
    const char* Ab = (const char*)p.A;
    const char* Bb = (const char*)p.B;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- bulk-copy producer ----------------
            uint64_t evict_first;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
            // The A operand is the dictionary image, which no earlier kernel
            // writes: fill the A ring before waiting for the previous kernel
            // (programmatic launch), whose output is the B operand.
            long long npre = 0;
            for (long long u = u0; u < u1 && npre < NE; ++u, ++npre) {
                mbar_expect_tx(smem_u32(a_full + npre), E_BYTES);
                bulk_load_hint(smem_u32(ringA + npre * E_BYTES), Ab + (size_t)u * p.G * TC_A_BYTES, E_BYTES,
                               smem_u32(a_full + npre), evict_first);
            }
            na = npre;
            griddep_wait();
            if (gemm_deferred(p)) {   // the ring fill issued above lands before the CTA exits
                for (long long s = 0; s < npre; ++s) mbar_drain(smem_u32(a_full + s), 0);
                u1 = u0;
            }
            long long ea = 0;   // A ring elements walked
            for (long long u = u0; u < u1; ++u) {
                const int k = (int)(u % p.K_tiles);
                int slot = (int)(nb % TC_NB);
                long long use = nb / TC_NB;
                if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) break;
                mbar_expect_tx(smem_u32(b_full + slot), B_BYTES);
                bulk_load(smem_u32(ringB + slot * B_BYTES), Bb + (size_t)k * B_BYTES, B_BYTES, smem_u32(b_full + slot));
                ++nb;
                if (ea++ < npre) continue;   // issued before the wait
                slot = (int)((ea - 1) % NE);
                use = (ea - 1) / NE;
                if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) break;
                // all G tiles of the unit (tiles beyond M_tiles are zero in the image)
                mbar_expect_tx(smem_u32(a_full + slot), E_BYTES);
                bulk_load_hint(smem_u32(ringA + slot * E_BYTES), Ab + (size_t)u * p.G * TC_A_BYTES, E_BYTES,
                               smem_u32(a_full + slot), evict_first);
                ++na;
            }
        }
    } else if (warp == 1) {
        // the bounded barrier waits below start once the previous kernel has
        // completed (a programmatic launch can begin while it still runs)
        griddep_wait();
        if (gemm_deferred(p)) u1 = u0;
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long ma = 0, mb = 0, ml = 0;   // ring positions consumed (A, B, Phi_lo)
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
                    const int sa = (int)(ma % NE);
                    if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((ma / NE) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int r = 0; r < valid; ++r) {
                        const int sl = (int)(ml % TC_NLO);
                        if (TF) {   // tile r of the element rounded in place, its Phi_lo in slot sl
                            if (!mbar_wait(smem_u32(lo_full + sl), (uint32_t)((ml / TC_NLO) & 1), abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                        }
                        const uint64_t da = desc_sw128(smem_u32(ringA + sa * E_BYTES + r * TC_A_BYTES));
                        const uint32_t dt = tmem + (uint32_t)(r * p.acc_stride);
#pragma unroll
                        for (int kk = 0; kk < KE / KM; ++kk) {
                            const uint32_t acc = (u > seg_start || kk > 0) ? 1u : 0u;
                            if (TF) mma_tf32(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc, acc);
                            else mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc, acc);
                        }
                        if (TF) {
                            const uint64_t dl = desc_sw128(smem_u32(ringL + sl * TC_A_BYTES));
#pragma unroll
                            for (int kk = 0; kk < KE / KM; ++kk)
                                mma_tf32(dt, dl + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc_lo, 1u);
                            mma_commit(smem_u32(lo_empty + sl));   // the Phi_lo slot is free once these are done
                            ++ml;
                        }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(a_empty + sa));   // the element is free once its MMAs are done
                    ++ma;
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
        // ------- epilogue warps: (TF32) Phi_lo tiles; TMEM -> partial sums -------
        const int seg0 = p.seg_base[blockIdx.x];
        const int sub = warp & 3;   // TMEM lanes 32 sub .. 32 sub + 31 (warp id mod 4)
        const int ew = warp - 2;
        const int GR = p.G * TC_BM;
        const int NC = p.QS / 16;
        griddep_wait();
        if (gemm_deferred(p)) u1 = u0;
        int nseg = 0;
        long long ne = 0, nlo = 0;   // A ring elements and Phi_lo slots walked (converter warps)
        long long u = u0;
        bool ok = true;
        while (u < u1 && ok) {
            const int g = (int)(u / p.K_tiles);
            const long long seg_end = min(u1, (long long)(g + 1) * p.K_tiles);
            const int valid = min(p.G, p.M_tiles - g * p.G);
            if (TF && ew < 4) {
                for (long long uu = u; uu < seg_end && ok; ++uu) {
                    const int sa = (int)(ne % NE);
                    if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((ne / NE) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    ++ne;
                    for (int r = 0; r < valid; ++r) {
                        const int sl = (int)(nlo % TC_NLO);
                        const long long use = nlo / TC_NLO;
                        if (use > 0 &&
                            !mbar_wait(smem_u32(lo_empty + sl), (uint32_t)((use - 1) & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        // this warp's quarter of tile r: 1024 floats, 8 float4 per lane;
                        // x -> hi = tf32_rn(x) in place, lo = tf32_rn(x - hi) into slot sl
                        constexpr int PW = 256;   // float4 per converter warp
                        float4* src = reinterpret_cast<float4*>(ringA + sa * E_BYTES + r * TC_A_BYTES) + ew * PW;
                        float4* dst = reinterpret_cast<float4*>(ringL + sl * TC_A_BYTES) + ew * PW;
#pragma unroll
                        for (int i = 0; i < PW / 32; ++i) {
                            const float4 x = src[lane + 32 * i];
                            const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
                            src[lane + 32 * i] = h;
                            dst[lane + 32 * i] = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y),
                                                             tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(lo_full + sl));
                        ++nlo;
                    }
                }
                if (!ok) break;
            }
            if (!mbar_wait(smem_u32(acc_full), (uint32_t)(nseg & 1), abort_flag)) break;
            tc_fence_after();
            float* out = p.part + (size_t)(seg0 + nseg) * p.Q * GR;
            drain_tmem<TF>(tmem + ((uint32_t)(32 * sub) << 16), ew >> 2, tc_epi_warps(TF) / 4, valid, p.acc_stride,
                           p.Q, p.QH, NC, GR, out, 32 * sub + lane);
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
        for (int s = 0; s < NE; ++s) {
            const long long n_s = na > s ? (na - s + NE - 1) / NE : 0;
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

// ---------------------------------------------------------------------------
// Packed serving: one launch of the GEMM applies the operator products of
// several fits at once.  Each fit's (group, k tile) units are cut into fixed
// segments of at most PK_SEGK k tiles per group, independent of the other fits
// in the step, so a fit's partial sums (and its results) are the same bits
// alone and among others; the host concatenates the segments of the step's
// fits and gives each CTA a contiguous run of about equal bytes.  Segments of
// a fit not in its CG loop (phase != PH_CG) are skipped by every role alike.
// Roles, rings, bounded waits and the TMEM drain are those of k_gemm_tc; the
// dictionary ring is filled only after the programmatic wait (which segments
// run depends on the previous kernels).
// ---------------------------------------------------------------------------
template <bool TF>
__global__ void __launch_bounds__(tc_threads(TF), 1) k_gemm_tc_packed(TcBatch p) {
    constexpr int NA = TC_NA;
    constexpr int KE = TF ? TC_BK32 : TC_BK;
    constexpr int KM = TF ? 8 : 16;
    const int EPT = p.G;
    const int NE = NA / p.G;
    const uint32_t E_BYTES = (uint32_t)EPT * TC_A_BYTES;
    griddep_launch();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_MAX = (uint32_t)p.QSmax * 128u;   // ring element (the largest fit's split tile)
    uint8_t* ringA = smem;
    uint8_t* ringL = smem + NA * TC_A_BYTES;
    uint8_t* ringB = ringL + (TF ? TC_NLO * TC_A_BYTES : 0);
    uint64_t* bars = (uint64_t*)(ringB + TC_NB * B_MAX);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + NA;
    uint64_t* lo_full = bars + 2 * NA;
    uint64_t* lo_empty = lo_full + TC_NLO;
    uint64_t* b_full = lo_empty + TC_NLO;
    uint64_t* b_empty = b_full + TC_NB;
    uint64_t* acc_full = b_empty + TC_NB;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* drain = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 3);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NA; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), 1);
        }
        for (int i = 0; i < TC_NLO; ++i) {
            mbar_init(smem_u32(lo_full + i), 4);
            mbar_init(smem_u32(lo_empty + i), 1);
        }
        for (int i = 0; i < TC_NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(acc_empty), tc_epi_warps(TF));
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
    griddep_wait();   // phases and B operands come from the previous kernels
    const int i0 = p.cta_seg[blockIdx.x], i1 = p.cta_seg[blockIdx.x + 1];
    long long na = 0, nb = 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- bulk-copy producer ----------------
            uint64_t evict_first;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
            bool ok = true;
            for (int i = i0; i < i1 && ok; ++i) {
                const TcSeg sg = p.segs[i];
                const TcSlot& sl = p.slots[sg.slot];
                if (sl.ctl->phase != PH_CG) continue;
                const int valid = min(p.G, sl.M_tiles - sg.g * p.G);
                const uint32_t bbytes = (uint32_t)sl.QS * 128u;
                for (int k = sg.k0; k < sg.k1; ++k) {
                    int slot = (int)(nb % TC_NB);
                    long long use = nb / TC_NB;
                    if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(b_full + slot), bbytes);
                    bulk_load(smem_u32(ringB + slot * B_MAX), sl.B + (size_t)k * bbytes, bbytes,
                              smem_u32(b_full + slot));
                    ++nb;
                    const long long u = (long long)sg.g * sl.K_tiles + k;
                    // the unit's row tiles that hold rows (the image's tiles
                    // past the last row are zero and never multiplied)
                    const uint32_t a_bytes = (uint32_t)valid * TC_A_BYTES;
                    slot = (int)(na % NE);
                    use = na / NE;
                    if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(smem_u32(a_full + slot), a_bytes);
                    bulk_load_hint(smem_u32(ringA + slot * E_BYTES), sl.A + (size_t)u * p.G * TC_A_BYTES, a_bytes,
                                   smem_u32(a_full + slot), evict_first);
                    ++na;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long ma = 0, mb = 0, ml = 0;   // ring positions consumed (A, B, Phi_lo)
            int nseg = 0;
            bool ok = true;
            for (int i = i0; i < i1 && ok; ++i) {
                const TcSeg sg = p.segs[i];
                const TcSlot& sl = p.slots[sg.slot];
                if (sl.ctl->phase != PH_CG) continue;
                const int valid = min(p.G, sl.M_tiles - sg.g * p.G);
                const uint32_t idesc = sl.idesc, idesc_lo = sl.idesc_lo;
                if (nseg > 0 && !mbar_wait(smem_u32(acc_empty), (uint32_t)((nseg - 1) & 1), abort_flag)) break;
                tc_fence_after();
                for (int k = sg.k0; k < sg.k1; ++k) {
                    const int sb = (int)(mb % TC_NB);
                    if (!mbar_wait(smem_u32(b_full + sb), (uint32_t)((mb / TC_NB) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    const uint64_t db = desc_sw128(smem_u32(ringB + sb * B_MAX));
                    const int sa = (int)(ma % NE);
                    if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((ma / NE) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int r = 0; r < valid; ++r) {
                        const int sl_lo = (int)(ml % TC_NLO);
                        if (TF) {
                            if (!mbar_wait(smem_u32(lo_full + sl_lo), (uint32_t)((ml / TC_NLO) & 1), abort_flag)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                        }
                        const uint64_t da = desc_sw128(smem_u32(ringA + sa * E_BYTES + r * TC_A_BYTES));
                        const uint32_t dt = tmem + (uint32_t)(r * p.acc_stride);
#pragma unroll
                        for (int kk = 0; kk < KE / KM; ++kk) {
                            const uint32_t acc = (k > sg.k0 || kk > 0) ? 1u : 0u;
                            if (TF) mma_tf32(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, acc);
                            else mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc, acc);
                        }
                        if (TF) {
                            const uint64_t dl = desc_sw128(smem_u32(ringL + sl_lo * TC_A_BYTES));
#pragma unroll
                            for (int kk = 0; kk < KE / KM; ++kk)
                                mma_tf32(dt, dl + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), idesc_lo, 1u);
                            mma_commit(smem_u32(lo_empty + sl_lo));
                            ++ml;
                        }
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(a_empty + sa));
                    ++ma;
                    mma_commit(smem_u32(b_empty + sb));
                    ++mb;
                }
                if (!ok) break;
                mma_commit(smem_u32(acc_full));
                ++nseg;
            }
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else {
        // ------- epilogue warps: (TF32) Phi_lo tiles; TMEM -> the fit's partials -------
        const int sub = warp & 3;
        const int ew = warp - 2;
        const int GR = p.G * TC_BM;
        int nseg = 0;
        long long ne = 0, nlo = 0;   // A ring elements and Phi_lo slots walked (converter warps)
        bool ok = true;
        for (int i = i0; i < i1 && ok; ++i) {
            const TcSeg sg = p.segs[i];
            const TcSlot& sl = p.slots[sg.slot];
            if (sl.ctl->phase != PH_CG) continue;
            const int valid = min(p.G, sl.M_tiles - sg.g * p.G);
            if (TF && ew < 4) {
                for (int k = sg.k0; k < sg.k1 && ok; ++k) {
                    const int sa = (int)(ne % NE);
                    if (!mbar_wait(smem_u32(a_full + sa), (uint32_t)((ne / NE) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    ++ne;
                    for (int r = 0; r < valid; ++r) {
                        const int sl_lo = (int)(nlo % TC_NLO);
                        const long long use = nlo / TC_NLO;
                        if (use > 0 &&
                            !mbar_wait(smem_u32(lo_empty + sl_lo), (uint32_t)((use - 1) & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        constexpr int PW = 256;   // float4 per converter warp
                        float4* src = reinterpret_cast<float4*>(ringA + sa * E_BYTES + r * TC_A_BYTES) + ew * PW;
                        float4* dst = reinterpret_cast<float4*>(ringL + sl_lo * TC_A_BYTES) + ew * PW;
#pragma unroll
                        for (int e = 0; e < PW / 32; ++e) {
                            const float4 x = src[lane + 32 * e];
                            const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
                            src[lane + 32 * e] = h;
                            dst[lane + 32 * e] = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y),
                                                             tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncwarp();
                        if (lane == 0) mbar_arrive(smem_u32(lo_full + sl_lo));
                        ++nlo;
                    }
                }
                if (!ok) break;
            }
            if (!mbar_wait(smem_u32(acc_full), (uint32_t)(nseg & 1), abort_flag)) break;
            tc_fence_after();
            float* out = sl.part + (size_t)sg.out * sl.Q * GR;
            drain_tmem<TF>(tmem + ((uint32_t)(32 * sub) << 16), ew >> 2, tc_epi_warps(TF) / 4, valid, p.acc_stride,
                           sl.Q, sl.QH, sl.QS / 16, GR, out, 32 * sub + lane);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty));
            ++nseg;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        for (int s = 0; s < NE; ++s) {
            const long long n_s = na > s ? (na - s + NE - 1) / NE : 0;
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

// ---------------------------------------------------------------------------
// FP8 E4M3 dictionary.  The A image holds codes, 128 rows x 128 codes per
// 16 KiB tile, tiles ordered (group of 2 row tiles, 128-wide k tile, row
// tile); a unit's two tiles arrive as one 32 KiB bulk copy.  Eight converter
// warps widen each tile to two BF16 sub-tiles (128 x 64, 128-byte swizzle) in
// shared memory: the BF16 bit pattern (b & 0x80) << 8 | (b & 0x7F) << 4 is the
// code's value times 2^-120 exactly (zero and subnormals included), so the
// MMA sees the codes up to one power of two.  The split vector blocks carry
// 2^64 (SplitOut::scale) so that every product stays in the FP32 normal range;
// the T reduction applies s_i 2^56 and the U partials carry 2^-56.
// Warp roles (448 threads): 0 producer, 1 TMEM + MMA, 2-5 epilogue,
// 6-13 converters.  Accumulators are double-buffered (2 x 2 x 128 columns).
// Rings: 3 landing units (32 KiB each), 4 BF16 sub-tiles (one unit), 2 B
// tiles.  (2 landing units and 6 sub-tiles, which lets the converters work
// half a unit further ahead of the MMAs, measured slower: 0.246 against
// 0.237 ms per application at 8192 x 32768.)
// ---------------------------------------------------------------------------
constexpr int F8_THREADS = 448, F8_G = 2, F8_NL = 3, F8_NC = 4, F8_NB = 2, F8_CW = 8;   // F8_CW converter warps
constexpr uint32_t F8_LAND = F8_G * TC_A_BYTES;     // one unit of codes
static_assert(F8_NC % 2 == 0, "the converters fill the sub-tile ring in pairs");
constexpr float F8_BSCALE = 18446744073709551616.0f;   // 2^64 on the split vector blocks
constexpr float F8_RFAC = 72057594037927936.0f;        // 2^56 = 2^120 / 2^64 back on the products

__device__ __forceinline__ uint32_t f8_pair(uint32_t x) {   // codes in bytes 0 and 2
    return ((x << 4) & 0x07F007F0u) | ((x & 0x00800080u) << 8);
}

__global__ void __launch_bounds__(F8_THREADS, 1) k_gemm8(TcParams p) {
    griddep_launch();
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)p.QS * 128u;   // one 64-wide k tile of the split block
    uint8_t* land = smem;
    uint8_t* conv = land + F8_NL * F8_LAND;
    uint8_t* ringB = conv + F8_NC * TC_A_BYTES;
    uint64_t* bars = (uint64_t*)(ringB + F8_NB * 2 * B_BYTES);
    uint64_t* land_full = bars;
    uint64_t* land_empty = land_full + F8_NL;
    uint64_t* conv_full = land_empty + F8_NL;
    uint64_t* conv_empty = conv_full + F8_NC;
    uint64_t* b_full = conv_empty + F8_NC;
    uint64_t* b_empty = b_full + F8_NB;
    uint64_t* acc_full = b_empty + F8_NB;   // [2]
    uint64_t* acc_empty = acc_full + 2;     // [2]
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < F8_NL; ++i) {
            mbar_init(smem_u32(land_full + i), 1);
            mbar_init(smem_u32(land_empty + i), F8_CW);
        }
        for (int i = 0; i < F8_NC; ++i) {
            mbar_init(smem_u32(conv_full + i), F8_CW);
            mbar_init(smem_u32(conv_empty + i), 1);
        }
        for (int i = 0; i < F8_NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(acc_full + i), 1);
            mbar_init(smem_u32(acc_empty + i), 4);
        }
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
    griddep_wait();   // B is the previous kernel's output; bounded waits start after it completed

    const long long u0 = (long long)blockIdx.x * p.W / gridDim.x;
    const long long u1 = gemm_deferred(p) ? u0 : (long long)(blockIdx.x + 1) * p.W / gridDim.x;
    long long nl = 0, nb = 0;   // copies issued into the landing and B rings (producer thread)

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- bulk-copy producer ----------------
            uint64_t evict_first;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
            for (long long u = u0; u < u1; ++u) {
                const int k = (int)(u % p.K_tiles);
                int slot = (int)(nb % F8_NB);
                long long use = nb / F8_NB;
                if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag)) break;
                mbar_expect_tx(smem_u32(b_full + slot), 2 * B_BYTES);
                bulk_load(smem_u32(ringB + slot * 2 * B_BYTES), (const char*)p.B + (size_t)(2 * k) * B_BYTES,
                          2 * B_BYTES, smem_u32(b_full + slot));
                ++nb;
                slot = (int)(nl % F8_NL);
                use = nl / F8_NL;
                if (use > 0 && !mbar_wait(smem_u32(land_empty + slot), (uint32_t)((use - 1) & 1), abort_flag))
                    break;
                mbar_expect_tx(smem_u32(land_full + slot), F8_LAND);
                bulk_load_hint(smem_u32(land + slot * F8_LAND), (const char*)p.A + (size_t)u * F8_LAND, F8_LAND,
                               smem_u32(land_full + slot), evict_first);
                ++nl;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long mc = 0, mb = 0;
            int nseg = 0;
            long long u = u0;
            bool ok = true;
            while (u < u1 && ok) {
                const int g = (int)(u / p.K_tiles);
                const long long seg_end = min(u1, (long long)(g + 1) * p.K_tiles);
                const int buf = nseg & 1;
                if (nseg >= 2 &&
                    !mbar_wait(smem_u32(acc_empty + buf), (uint32_t)(((nseg - 2) >> 1) & 1), abort_flag))
                    break;
                tc_fence_after();
                const long long seg_start = u;
                for (; u < seg_end; ++u) {
                    const int sb = (int)(mb % F8_NB);
                    if (!mbar_wait(smem_u32(b_full + sb), (uint32_t)((mb / F8_NB) & 1), abort_flag)) {
                        ok = false;
                        break;
                    }
                    for (int sub = 0; sub < 2 * F8_G; ++sub) {   // (row tile r, k half h)
                        const int r = sub >> 1, h = sub & 1;
                        const int cs = (int)(mc % F8_NC);
                        if (!mbar_wait(smem_u32(conv_full + cs), (uint32_t)((mc / F8_NC) & 1), abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t da = desc_sw128(smem_u32(conv + cs * TC_A_BYTES));
                        const uint64_t db = desc_sw128(smem_u32(ringB + sb * 2 * B_BYTES + h * B_BYTES));
                        const uint32_t dt = tmem + (uint32_t)(buf * 2 * p.acc_stride + r * p.acc_stride);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc,
                                     (u > seg_start || h > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(smem_u32(conv_empty + cs));
                        ++mc;
                    }
                    if (!ok) break;
                    mma_commit(smem_u32(b_empty + sb));
                    ++mb;
                }
                if (!ok) break;
                mma_commit(smem_u32(acc_full + buf));
                ++nseg;
            }
            // every issued MMA must finish before TMEM is released
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else if (warp < 6) {
        // ---------------- epilogue warps: TMEM -> segment partials ----------------
        const int seg0 = p.seg_base[blockIdx.x];
        const int sub = warp & 3;
        const int GR = F8_G * TC_BM;
        const int NC = p.QS / 16;

        int nseg = 0;
        long long u = u0;
        while (u < u1) {
            const int g = (int)(u / p.K_tiles);
            const long long seg_end = min(u1, (long long)(g + 1) * p.K_tiles);
            const int valid = min(F8_G, p.M_tiles - g * F8_G);
            const int buf = nseg & 1;
            if (!mbar_wait(smem_u32(acc_full + buf), (uint32_t)((nseg >> 1) & 1), abort_flag)) break;
            tc_fence_after();
            float* out = p.part + (size_t)(seg0 + nseg) * p.Q * GR;
            drain_tmem<false>(tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(buf * 2 * p.acc_stride), 0, 1, valid,
                              p.acc_stride, p.Q, 0, NC, GR, out, 32 * sub + lane);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(acc_empty + buf));
            ++nseg;
            u = seg_end;
        }
    } else {
        // ---------------- converter warps: codes -> BF16 sub-tiles ----------------
        // One code tile (128 x 128) at a time into two consecutive sub-tile slots
        // (h = 0: codes 0..63, h = 1: codes 64..127).  Eight threads read one
        // 128-byte code row (no bank conflict); threads 4..7 of the eight write
        // their odd 16-byte chunk first, so each store touches all 32 banks once.
        const int ct = threadIdx.x - 192;   // 0 .. 255
        const int j8 = ct & 7, h = j8 >> 2, cpart = j8 & 3;
        long long cl = 0, cc = 0;           // landing units and sub-tiles converted
        bool ok = true;
        for (long long u = u0; u < u1 && ok; ++u) {
            const int ls = (int)(cl % F8_NL);
            if (!mbar_wait(smem_u32(land_full + ls), (uint32_t)((cl / F8_NL) & 1), abort_flag)) break;
            for (int r = 0; r < F8_G; ++r) {
                const int cs0 = (int)(cc % F8_NC), cs1 = (int)((cc + 1) % F8_NC);
                const long long use0 = cc / F8_NC, use1 = (cc + 1) / F8_NC;
                if ((use0 > 0 && !mbar_wait(smem_u32(conv_empty + cs0), (uint32_t)((use0 - 1) & 1), abort_flag)) ||
                    (use1 > 0 && !mbar_wait(smem_u32(conv_empty + cs1), (uint32_t)((use1 - 1) & 1), abort_flag))) {
                    ok = false;
                    break;
                }
                const uint8_t* src = land + ls * F8_LAND + r * TC_A_BYTES;
                uint8_t* dst = conv + (h ? cs1 : cs0) * TC_A_BYTES;
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int rr = (ct >> 3) + 32 * it;
                    const uint4 w = *reinterpret_cast<const uint4*>(src + rr * 128 + j8 * 16);
                    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
                    uint32_t o[8];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        o[2 * k] = f8_pair(__byte_perm(ws[k], 0u, 0x4140));
                        o[2 * k + 1] = f8_pair(__byte_perm(ws[k], 0u, 0x4342));
                    }
                    const int c8 = 2 * cpart;   // bf16 16-byte chunks c8, c8 + 1 of row rr
                    const uint4 lo = make_uint4(o[0], o[1], o[2], o[3]), hi = make_uint4(o[4], o[5], o[6], o[7]);
                    uint4* p0 = reinterpret_cast<uint4*>(dst + rr * 128 + ((c8 ^ (rr & 7)) << 4));
                    uint4* p1 = reinterpret_cast<uint4*>(dst + rr * 128 + (((c8 + 1) ^ (rr & 7)) << 4));
                    if (h) {
                        *p1 = hi;
                        *p0 = lo;
                    } else {
                        *p0 = lo;
                        *p1 = hi;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(conv_full + cs0));
                    mbar_arrive(smem_u32(conv_full + cs1));
                }
                cc += 2;
            }
            if (!ok) break;
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(land_empty + ls));
            ++cl;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        for (int s = 0; s < F8_NL; ++s) {
            const long long n_s = nl > s ? (nl - s + F8_NL - 1) / F8_NL : 0;
            if (n_s > 0) mbar_drain(smem_u32(land_full + s), (uint32_t)((n_s - 1) & 1));
        }
        for (int s = 0; s < F8_NB; ++s) {
            const long long n_s = nb > s ? (nb - s + F8_NB - 1) / F8_NB : 0;
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

// FP8 code images: tile (g, k, r) = rows (g G + r) 128 .. +127, codes
// k 128 .. +127 of the row-major code matrix (ld bytes per row), plain rows.
__global__ __launch_bounds__(128) void k_tile8_rows(const uint8_t* __restrict__ src, long long ld, int M_tiles,
                                                    int K_tiles, int G, uint8_t* __restrict__ dst) {
    const int k = blockIdx.x, gr = blockIdx.y, g = gr / G, r = gr % G;
    const int m = g * G + r, rr = threadIdx.x;
    uint8_t* tile = dst + (((size_t)g * K_tiles + k) * G + r) * TC_A_BYTES;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + ((size_t)m * TC_BM + rr) * ld + (size_t)k * 128);
#pragma unroll
    for (int c = 0; c < 8; ++c)
        reinterpret_cast<uint4*>(tile + rr * 128)[c] = m < M_tiles ? s4[c] : make_uint4(0u, 0u, 0u, 0u);
}

// Transposed code image: tile (g, k, r) holds element (rr, cc) =
// src[k 128 + cc][(g G + r) 128 + rr].
__global__ __launch_bounds__(128) void k_tile8_cols(const uint8_t* __restrict__ src, long long ld, int M_tiles,
                                                    int K_tiles, int G, uint8_t* __restrict__ dst) {
    __shared__ uint8_t sm[128][129];
    const int k = blockIdx.x, gr = blockIdx.y, g = gr / G, r = gr % G;
    const int m = g * G + r, t = threadIdx.x;
    for (int n = 0; n < 128; ++n)
        sm[n][t] = m < M_tiles ? src[((size_t)k * 128 + n) * ld + (size_t)m * TC_BM + t] : (uint8_t)0;
    __syncthreads();
    uint8_t* tile = dst + (((size_t)g * K_tiles + k) * G + r) * TC_A_BYTES;
    for (int c = 0; c < 128; ++c) tile[t * 128 + c] = sm[c][t];
}

// Vs = tiled swizzled image of the split of V (Q x Dp, FP32): bf16 3-term
// (fmt 1, row 3q + t) or TF32 hi / lo (fmt 2, rows q and QH + q).
__global__ void k_split(const float* __restrict__ V, long long Dp, SplitOut so) {
    const int q = blockIdx.y;
    const long long j = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (j >= Dp) return;
    store_split(so, q, j, *reinterpret_cast<const float4*>(V + (size_t)q * Dp + j));
}

// GEMM1 epilogue: T = sum of the segment partials of its group (fixed order),
// split into the B image of GEMM2, and ||T_q||^2 partials -> pi, gamma.
__device__ __forceinline__ void reduce_T_body(const float* __restrict__ part, const int* __restrict__ grp_seg, int GR,
                                              int Q, long long Np, const SplitOut& so, double* tt_part, int nblk,
                                              unsigned* counter, DevCtl* ctl, int mode,
                                              const float* __restrict__ rscale, float rfac, int q, int ib,
                                              unsigned total) {
    __shared__ double sh[8];
    const long long i = (long long)ib * 1024 + threadIdx.x * 4;
    float tt = 0.0f;
    if (i < Np) {
        const int g = (int)(i / GR), r = (int)(i % GR);
        const int s0 = grp_seg[2 * g], ns = grp_seg[2 * g + 1];
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 8
        for (int s = 0; s < ns; ++s) {
            const float4 b = __ldcg(reinterpret_cast<const float4*>(part + ((size_t)(s0 + s) * Q + q) * GR + r));
            a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
        }
        if (rscale) {   // FP8 dictionary: T_i = s_i 2^56 (Q V)_i; the second product takes s_i T_i
            const float4 sv = *reinterpret_cast<const float4*>(rscale + i);
            a = make_float4(a.x * (sv.x * rfac), a.y * (sv.y * rfac), a.z * (sv.z * rfac), a.w * (sv.w * rfac));
            store_split(so, q, i, make_float4(a.x * sv.x, a.y * sv.y, a.z * sv.z, a.w * sv.w));
        } else {
            store_split(so, q, i, a);
        }
        tt = a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
    }
    const double ttd = block_sum_f(tt, sh);
    if (threadIdx.x == 0) tt_part[(size_t)q * nblk + ib] = ttd;
    if (mode == OP_CG) {   // the update kernel reduces the partials (op_cg_begin)
        if (ib == 0 && q == 0 && threadIdx.x == 0) op_cg_begin(ctl, tt_part, nblk);
        return;
    }
    if (!last_block_arrive(counter, total)) return;
    op_finalize_block(ctl, tt_part, nblk, Q);
}

__global__ __launch_bounds__(256) void k_tc_reduce_T(const float* __restrict__ part, const int* __restrict__ grp_seg,
                                                     int GR, int Q, long long Np, SplitOut so, double* tt_part,
                                                     int nblk, unsigned* counter, DevCtl* ctl, int mode,
                                                     const float* __restrict__ rscale, float rfac) {
    griddep_launch();
    griddep_wait();   // the partials are the previous kernel's output
    reduce_T_body(part, grp_seg, GR, Q, Np, so, tt_part, nblk, counter, ctl, mode, rscale, rfac, blockIdx.y,
                  blockIdx.x, gridDim.x * gridDim.y);
}

// Packed serving: block b = (fit, column, 1024-row block) map[b] of the fits
// in their CG loop (the operator's first product -> split(T), ||T||^2 partials).
__global__ __launch_bounds__(256) void k_reduce_T_packed(const VSlot* __restrict__ vs, const int4* __restrict__ map,
                                                         const int* __restrict__ count) {
    griddep_launch();
    if ((int)blockIdx.x >= *count) return;   // the grid is sized for the server's capacity
    griddep_wait();
    const int4 m = map[blockIdx.x];
    const VSlot& f = vs[m.x];
    DevCtl* ctl = f.ctl;
    if (ctl->phase != PH_CG) return;
    const SplitOut st = f.st;
    const int nblk = (int)((f.Np + 1023) / 1024);
    reduce_T_body(f.t_part, f.t_grp, f.GR, f.Q, f.Np, st, f.tt_part, nblk, nullptr, ctl, OP_CG, nullptr, 1.0f, m.y,
                  m.z, 0u);
}

// GEMM2 epilogue for a stand-alone application: U (Q x Dp) = sum of the
// segment partials of its group.
__global__ __launch_bounds__(256) void k_tc_reduce_U(const float* __restrict__ part, const int* __restrict__ grp_seg,
                                                     int GR, int Q, long long Dp, float* __restrict__ U,
                                                     float uscale) {
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
    *reinterpret_cast<float4*>(U + (size_t)q * Dp + j) =
        make_float4(a.x * uscale, a.y * uscale, a.z * uscale, a.w * uscale);
}

// A image of GEMM1: tile (g, k, r) = rows (g G + r) 128 .. +127 and the k-th
// 128-byte column block of the row-major dictionary (ld elements per row),
// each row's eight 16-byte chunks swizzled (chunk c at c ^ (row & 7)); zero
// tiles beyond M_tiles.  TE = element type (64 bf16 or 32 fp32 per row).
template <typename TE>
__global__ __launch_bounds__(128) void k_tile_rows(const TE* __restrict__ src, long long ld, int M_tiles, int K_tiles,
                                                   int G, TE* __restrict__ dst) {
    constexpr int KE = 128 / sizeof(TE);
    const int k = blockIdx.x, gr = blockIdx.y, g = gr / G, r = gr % G;
    const int m = g * G + r, rr = threadIdx.x;
    char* tile = (char*)dst + (((size_t)g * K_tiles + k) * G + r) * TC_A_BYTES;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + ((size_t)m * TC_BM + rr) * ld + (size_t)k * KE);
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint4 v = m < M_tiles ? s4[c] : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(tile + rr * 128 + ((c ^ (rr & 7)) << 4)) = v;
    }
}

// A image of GEMM2 (rows of the transpose = columns of the dictionary): tile
// (g, k, r) holds element (rr, cc) = src[k KE + cc][(g G + r) 128 + rr], swizzled.
template <typename TE>
__global__ __launch_bounds__(128) void k_tile_cols(const TE* __restrict__ src, long long ld, int M_tiles, int K_tiles,
                                                   int G, TE* __restrict__ dst) {
    constexpr int KE = 128 / sizeof(TE), PER = 16 / sizeof(TE);
    __shared__ TE sm[KE][TC_BM + 8];
    const int k = blockIdx.x, gr = blockIdx.y, g = gr / G, r = gr % G;
    const int m = g * G + r, t = threadIdx.x;
    for (int n = 0; n < KE; ++n) sm[n][t] = m < M_tiles ? src[((size_t)k * KE + n) * ld + (size_t)m * TC_BM + t] : TE(0.0f);
    __syncthreads();
    char* tile = (char*)dst + (((size_t)g * K_tiles + k) * G + r) * TC_A_BYTES;
    for (int c = 0; c < 8; ++c) {
        TE v[PER];
#pragma unroll
        for (int e = 0; e < PER; ++e) v[e] = sm[c * PER + e][t];
        *reinterpret_cast<uint4*>(tile + t * 128 + ((c ^ (t & 7)) << 4)) = *reinterpret_cast<const uint4*>(v);
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct GemmPlan {
    TcParams p{};
    int nCTA = 0;
    int nseg = 0, groups = 0;
    int* seg_base = nullptr;         // device
    int* grp_seg = nullptr;          // device
    float* part = nullptr;           // device
    void* A = nullptr;               // device, tiled image of the A operand
    size_t A_bytes = 0;
};

struct TcPlan {
    bool tf = false;                 // TF32 format (FP32 dictionary)
    bool f8 = false;                 // FP8 E4M3 codes with row scales (k_gemm8)
    int Q = 0, QS = 0, QH = 0, G = 0;
    size_t smem = 0;
    void* Vs = nullptr;              // tiled image of split(P), QS x Dp
    void* Ts = nullptr;              // tiled image of split(T), QS x Np
    size_t esz = 2;                  // bytes per image element
    GemmPlan g1, g2;
    // packed serving: fixed segments of both products (PK_SEGK k tiles per
    // segment) and their partials, independent of the other fits in a step
    float *pk_part1 = nullptr, *pk_part2 = nullptr;
    int *pk_grp1 = nullptr, *pk_grp2 = nullptr;
    std::vector<TcSeg> pk_s1, pk_s2;
    std::vector<double> pk_c1, pk_c2;
    FusedPlan* fused = nullptr;      // single-pass form (then g1, g2 are unused)
    void* fimg = nullptr;            // its tiled image of Phi~ (groups of 2 row tiles)
    size_t fimg_bytes = 0;
    long long bytes = 0;
};

constexpr uint32_t make_idesc(int M, int N, bool tf) {
    const uint32_t fmt = tf ? 2u : 1u;   // TF32 : BF16
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

cudaError_t plan_gemm(GemmPlan& gp, int num_sms, long long M_rows, long long K_cols, int KE, int G, int acc_stride,
                      int QS, int QH, int Q, bool tf, unsigned* flags, long long* bytes, cudaStream_t st) {
    TcParams& p = gp.p;
    p.M_tiles = (int)((M_rows + TC_BM - 1) / TC_BM);
    p.K_tiles = (int)((K_cols + KE - 1) / KE);
    p.G = G;
    p.acc_stride = acc_stride;
    p.QS = QS;
    p.QH = QH;
    p.Q = Q;
    p.idesc = make_idesc(TC_BM, QS, tf);
    p.idesc_lo = make_idesc(TC_BM, QS, tf);   // TF32: Phi_lo times [P_hi | P_lo]
    p.flags = flags;
    p.defer = nullptr;
    gp.groups = (p.M_tiles + G - 1) / G;
    p.W = (long long)gp.groups * p.K_tiles;
    // at least ~16 units per CTA: small problems then leave SMs to other work
    // (concurrent requests) instead of paying the pipeline fill on every SM
    gp.nCTA = (int)std::max<long long>(1, std::min<long long>(num_sms, p.W / 16));
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
    if ((e = cudaMallocAsync(&gp.seg_base, seg_base.size() * sizeof(int), st))) return e;
    if ((e = cudaMallocAsync(&gp.grp_seg, grp.size() * sizeof(int), st))) return e;
    const size_t part_elems = (size_t)nseg * Q * G * TC_BM;
    if ((e = cudaMallocAsync(&gp.part, part_elems * sizeof(float), st))) return e;
    gp.A_bytes = (size_t)gp.groups * G * (size_t)p.K_tiles * TC_A_BYTES;
    if ((e = cudaMallocAsync(&gp.A, gp.A_bytes, st))) return e;
    *bytes += (long long)(seg_base.size() + grp.size()) * 4 + (long long)part_elems * 4 + (long long)gp.A_bytes;
    if ((e = cudaMemcpyAsync(gp.seg_base, seg_base.data(), seg_base.size() * sizeof(int), cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(gp.grp_seg, grp.data(), grp.size() * sizeof(int), cudaMemcpyHostToDevice, st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;   // the host tables go out of scope
    p.seg_base = gp.seg_base;
    p.part = gp.part;
    p.A = gp.A;
    return cudaSuccess;
}

void free_gemm(GemmPlan& gp, cudaStream_t st) {
    if (gp.seg_base) cudaFreeAsync(gp.seg_base, st);
    if (gp.grp_seg) cudaFreeAsync(gp.grp_seg, st);
    if (gp.part) cudaFreeAsync(gp.part, st);
    if (gp.A) cudaFreeAsync(gp.A, st);
    gp.seg_base = gp.grp_seg = nullptr;
    gp.part = nullptr;
    gp.A = nullptr;
}

size_t gemm8_smem(int QS) {
    return 1024 + (size_t)F8_NL * F8_LAND + (size_t)F8_NC * TC_A_BYTES + (size_t)F8_NB * 2 * QS * 128 + 512;
}

size_t gemm_smem(bool tf, int QS) {   // k_gemm_tc, k_gemm_tc_packed
    return 1024 + (size_t)TC_NA * TC_A_BYTES + (tf ? (size_t)TC_NLO * TC_A_BYTES : 0) + (size_t)TC_NB * QS * 128 + 512;
}

}  // namespace

void tc_release(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    if (!t) return;
    free_gemm(t->g1, c->stream);
    free_gemm(t->g2, c->stream);
    fused_destroy(t->fused, c->stream);
    if (t->fimg) cudaFreeAsync(t->fimg, c->stream);
    if (t->Vs) cudaFreeAsync(t->Vs, c->stream);
    if (t->Ts) cudaFreeAsync(t->Ts, c->stream);
    for (void* p : {(void*)t->pk_part1, (void*)t->pk_part2, (void*)t->pk_grp1, (void*)t->pk_grp2})
        if (p) cudaFreeAsync(p, c->stream);
    c->bytes -= t->bytes;
    delete t;
    c->tc = nullptr;
}

// Plan for a Q-column block: split factors, segment tables, and the tiled
// images of the dictionary (GEMM1) and of its transpose (GEMM2), built from the
// row-major copy (bf16 for the BF16 form, fp32 for the FP32 form).
cudaError_t tc_setup(cofem_ctx* c, int Q) {
    tc_release(c);
    TcPlan* t = new TcPlan();
    c->tc = t;
    t->f8 = c->phi8 != nullptr;
    t->tf = c->phi16 == nullptr && !t->f8;
    t->Q = Q;
    int KE, acc_stride;
    if (t->f8) {   // codes: 128 per 128-byte tile row; split blocks in BF16
        t->QH = 0;
        t->QS = ((3 * Q + 15) / 16) * 16;
        t->esz = 2;
        KE = 128;
        if (t->QS > 128) return cudaErrorNotSupported;
    } else if (t->tf) {
        t->QH = ((Q + 15) / 16) * 16;
        t->QS = 2 * t->QH;
        t->esz = 4;
        KE = TC_BK32;
    } else {
        t->QH = 0;
        t->QS = ((3 * Q + 15) / 16) * 16;
        t->esz = 2;
        KE = TC_BK;
    }
    if (t->f8) {
        t->G = F8_G;
        acc_stride = 128;
    } else if (t->QS <= 128) {
        t->G = 4;
        acc_stride = 128;
    } else {
        t->G = 2;
        acc_stride = 256;
    }
    cudaError_t e;
    unsigned* flags = &c->ctl->flags;
    cudaStream_t st = c->stream;
    // single-pass form: BF16, where it applies, on request (AUTO takes the
    // two-pass form, the faster of the two as measured on GB300 so far)
    int coop = 0, max_smem = 0;
    if ((e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device))) return e;
    if ((e = cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device))) return e;
    const bool can_fuse = !t->tf && !t->f8 && fused_supported(c->num_sms, c->Dp, t->QS, coop != 0, max_smem);
    const int path = c->opts.dense_path;
    if (path == COFEM_PATH_SINGLE_PASS && !can_fuse) return cudaErrorNotSupported;
    if (can_fuse && path == COFEM_PATH_SINGLE_PASS) {
        const int G = 2;
        const long long M_tiles = c->Np / TC_BM, K_tiles = c->Dp / TC_BK, groups = (M_tiles + G - 1) / G;
        t->fimg_bytes = (size_t)groups * G * K_tiles * TC_A_BYTES;
        if ((e = cudaMallocAsync(&t->fimg, t->fimg_bytes, st))) return e;
        if ((e = cudaMallocAsync(&t->Vs, (size_t)t->QS * c->Dp * t->esz, st))) return e;
        if ((e = cudaMallocAsync(&t->Ts, (size_t)t->QS * c->Np * t->esz, st))) return e;
        t->bytes += (long long)t->fimg_bytes + (long long)t->QS * (c->Dp + c->Np) * (long long)t->esz;
        if ((e = cudaMemsetAsync(t->Vs, 0, (size_t)t->QS * c->Dp * t->esz, st))) return e;
        if ((e = cudaMemsetAsync(t->Ts, 0, (size_t)t->QS * c->Np * t->esz, st))) return e;
        k_tile_rows<__nv_bfloat16><<<dim3((unsigned)K_tiles, (unsigned)(groups * G)), 128, 0, st>>>(
            c->phi16, c->Dp, (int)M_tiles, (int)K_tiles, G, (__nv_bfloat16*)t->fimg);
        if ((e = cudaGetLastError())) return e;
        if ((e = fused_create(&t->fused, c->num_sms, c->Np, c->Dp, Q, t->QS, t->fimg, t->Vs, t->Ts, c->U, c->ctl,
                              st, &t->bytes)))
            return e;
        c->bytes += t->bytes;
        t->smem = fused_smem_bytes(t->QS);
        return cudaStreamSynchronize(st);
    }
    if ((e = plan_gemm(t->g1, c->num_sms, c->Np, c->Dp, KE, t->G, acc_stride, t->QS, t->QH, Q, t->tf, flags,
                       &t->bytes, st)))
        return e;
    if ((e = plan_gemm(t->g2, c->num_sms, c->Dp, c->Np, KE, t->G, acc_stride, t->QS, t->QH, Q, t->tf, flags,
                       &t->bytes, st)))
        return e;
    if ((e = cudaMallocAsync(&t->Vs, (size_t)t->QS * c->Dp * t->esz, st))) return e;
    if ((e = cudaMallocAsync(&t->Ts, (size_t)t->QS * c->Np * t->esz, st))) return e;
    t->bytes += (long long)t->QS * (c->Dp + c->Np) * (long long)t->esz;
    c->bytes += t->bytes;
    if ((e = cudaMemsetAsync(t->Vs, 0, (size_t)t->QS * c->Dp * t->esz, st))) return e;   // padding rows stay zero
    if ((e = cudaMemsetAsync(t->Ts, 0, (size_t)t->QS * c->Np * t->esz, st))) return e;
    t->g1.p.B = t->Vs;
    t->g2.p.B = t->Ts;
    if (t->f8) {
        k_tile8_rows<<<dim3(t->g1.p.K_tiles, t->g1.groups * t->G), 128, 0, st>>>(
            c->phi8, c->Dp, t->g1.p.M_tiles, t->g1.p.K_tiles, t->G, (uint8_t*)t->g1.A);
        k_tile8_cols<<<dim3(t->g2.p.K_tiles, t->g2.groups * t->G), 128, 0, st>>>(
            c->phi8, c->Dp, t->g2.p.M_tiles, t->g2.p.K_tiles, t->G, (uint8_t*)t->g2.A);
    } else if (t->tf) {
        k_tile_rows<float><<<dim3(t->g1.p.K_tiles, t->g1.groups * t->G), 128, 0, st>>>(
            c->phi32, c->Dp, t->g1.p.M_tiles, t->g1.p.K_tiles, t->G, (float*)t->g1.A);
        k_tile_cols<float><<<dim3(t->g2.p.K_tiles, t->g2.groups * t->G), 128, 0, st>>>(
            c->phi32, c->Dp, t->g2.p.M_tiles, t->g2.p.K_tiles, t->G, (float*)t->g2.A);
    } else {
        k_tile_rows<__nv_bfloat16><<<dim3(t->g1.p.K_tiles, t->g1.groups * t->G), 128, 0, st>>>(
            c->phi16, c->Dp, t->g1.p.M_tiles, t->g1.p.K_tiles, t->G, (__nv_bfloat16*)t->g1.A);
        k_tile_cols<__nv_bfloat16><<<dim3(t->g2.p.K_tiles, t->g2.groups * t->G), 128, 0, st>>>(
            c->phi16, c->Dp, t->g2.p.M_tiles, t->g2.p.K_tiles, t->G, (__nv_bfloat16*)t->g2.A);
    }
    if ((e = cudaGetLastError())) return e;
    if ((e = cudaStreamSynchronize(st))) return e;
    t->smem = t->f8 ? gemm8_smem(t->QS) : gemm_smem(t->tf, t->QS);
    return cudaSuccess;
}

// The shared-memory limit of a kernel is one device-wide attribute; handles with
// different K running concurrently must not lower it under each other, so it is
// raised once, to the opt-in maximum, when the library first runs on a device.
cudaError_t tc_kernel_attributes(int max_smem) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e != cudaSuccess) return e;
    if ((e = fused_kernel_attributes(max_smem)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_gemm8, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_gemm_tc_packed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    if ((e = cudaFuncSetAttribute(k_gemm_tc_packed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem)))
        return e;
    return cudaFuncSetAttribute(k_gemm_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
}

SplitOut tc_direction_split(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    if (!t || c->kind != COFEM_OP_DENSE) return SplitOut{nullptr, 0, 0, 0};
    return SplitOut{t->Vs, t->tf ? 2 : 1, t->QS, t->QH, t->f8 ? F8_BSCALE : 1.0f};
}

OpOut op_output(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    if (c->kind == COFEM_OP_DENSE && t && t->fused) return OpOut{c->U, 1, (size_t)c->Qcap * c->Dp, nullptr, 0};
    if (c->kind == COFEM_OP_DENSE && t)
        return OpOut{t->g2.part, 1, 0, t->g2.grp_seg, t->G * TC_BM, t->f8 ? F8_RFAC : 1.0f};
    const int S2 = c->kind == COFEM_OP_DENSE ? c->S2 : 1;
    return OpOut{c->U, S2, (size_t)c->Qcap * c->Dp, nullptr, 0};
}

// The CG loop of the fit graph runs the operator's first product at the end
// of the loop body, after the direction kernel that writes its input (so that
// it joins the step by a programmatic edge), and the rest of the operator at
// the start of the next iteration: the two-pass tensor-core forms only.
bool tc_rotatable(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    return c->kind == COFEM_OP_DENSE && t && !t->fused;
}

void launch_tc_first_product(Sink& s, cofem_ctx* c, bool defer_rr) {
    TcPlan* t = (TcPlan*)c->tc;
    void (*gemm)(TcParams) = t->f8 ? k_gemm8 : (t->tf ? k_gemm_tc<true> : k_gemm_tc<false>);
    const unsigned nthreads = t->f8 ? F8_THREADS : (unsigned)tc_threads(t->tf);
    TcParams p = t->g1.p;
    p.defer = defer_rr ? c->ctl : nullptr;
    s.launch_pdl(gemm, dim3(t->g1.nCTA), dim3(nthreads), t->smem, p);
}

void launch_tc_rest(Sink& s, cofem_ctx* c, int Q, int mode) {
    TcPlan* t = (TcPlan*)c->tc;
    const SplitOut st{t->Ts, t->tf ? 2 : 1, t->QS, t->QH, t->f8 ? F8_BSCALE : 1.0f};
    void (*gemm)(TcParams) = t->f8 ? k_gemm8 : (t->tf ? k_gemm_tc<true> : k_gemm_tc<false>);
    const unsigned nthreads = t->f8 ? F8_THREADS : (unsigned)tc_threads(t->tf);
    const int nblk = (int)((c->Np + 1023) / 1024);
    s.launch_pdl(k_tc_reduce_T, dim3(nblk, Q), dim3(256), 0, t->g1.part, t->g1.grp_seg, t->G * TC_BM, Q, c->Np, st,
                 c->tt_part, nblk, c->counters + 8, c->ctl, mode, t->f8 ? (const float*)c->scale8 : (const float*)nullptr,
                 t->f8 ? F8_RFAC : 1.0f);
    s.launch_pdl(gemm, dim3(t->g2.nCTA), dim3(nthreads), t->smem, t->g2.p);
}

// In the CG loop (OP_CG, OP_TIME) the split of P is already in Vs (written by
// k_cg_init / k_cg_direction) and the update kernel reads GEMM2's segment
// partials directly; a stand-alone application (OP_PLAIN) splits V here and
// also sums the partials into U.
void launch_tc_operator(Sink& s, cofem_ctx* c, int Q, const float* V, int mode) {
    TcPlan* t = (TcPlan*)c->tc;
    const SplitOut sv{t->Vs, t->tf ? 2 : 1, t->QS, t->QH, t->f8 ? F8_BSCALE : 1.0f};
    const SplitOut st{t->Ts, t->tf ? 2 : 1, t->QS, t->QH, t->f8 ? F8_BSCALE : 1.0f};
    if (mode == OP_PLAIN)
        s.launch(k_split, dim3((unsigned)((c->Dp / 4 + 255) / 256), Q), dim3(256), 0, V, c->Dp, sv);
    if (t->fused) {   // writes U and finishes pi, gamma itself
        launch_fused(s, t->fused, mode);
        return;
    }
    void (*gemm)(TcParams) = t->f8 ? k_gemm8 : (t->tf ? k_gemm_tc<true> : k_gemm_tc<false>);
    const unsigned nthreads = t->f8 ? F8_THREADS : (unsigned)tc_threads(t->tf);
    // programmatic launches: each kernel waits (griddep_wait) for its
    // predecessor before it reads that kernel's output
    s.launch_pdl(gemm, dim3(t->g1.nCTA), dim3(nthreads), t->smem, t->g1.p);
    const int nblk = (int)((c->Np + 1023) / 1024);
    s.launch_pdl(k_tc_reduce_T, dim3(nblk, Q), dim3(256), 0, t->g1.part, t->g1.grp_seg, t->G * TC_BM, Q, c->Np, st,
             c->tt_part, nblk, c->counters + 8, c->ctl, mode, t->f8 ? (const float*)c->scale8 : (const float*)nullptr,
             t->f8 ? F8_RFAC : 1.0f);
    s.launch_pdl(gemm, dim3(t->g2.nCTA), dim3(nthreads), t->smem, t->g2.p);
    if (mode == OP_PLAIN)
        s.launch(k_tc_reduce_U, dim3((unsigned)((c->Dp + 1023) / 1024), Q), dim3(256), 0, t->g2.part,
                 t->g2.grp_seg, t->G * TC_BM, Q, c->Dp, c->U, t->f8 ? F8_RFAC : 1.0f);
}

// Operator form in use and kernels per application (CG loop, residual replacement).
void tc_operator_info(cofem_ctx* c, int* path, int* k_cg, int* k_rr) {
    TcPlan* t = (TcPlan*)c->tc;
    *path = t->fused ? COFEM_PATH_SINGLE_PASS : COFEM_PATH_TWO_PASS;
    *k_cg = t->fused ? 1 : 3;
    *k_rr = true_residual_kernels(c);
}

// ---------------------------------------------------------------------------
// Packed serving (host side)
// ---------------------------------------------------------------------------
namespace {

// Fixed segments of one product: row group g, k tiles [k0, k0 + PK_SEGK);
// segment g * spg + s; cost = bytes of the dictionary image it reads.
cudaError_t pack_product(TcPlan* t, const GemmPlan& gp, bool tf, int Q, std::vector<TcSeg>& segs,
                         std::vector<double>& cost, float** part, int** grp, cudaStream_t st) {
    const int K_tiles = gp.p.K_tiles, M_tiles = gp.p.M_tiles, G = gp.p.G, groups = gp.groups;
    const int spg = (K_tiles + PK_SEGK - 1) / PK_SEGK;
    segs.clear();
    cost.clear();
    std::vector<int> tab(2 * (size_t)groups);
    for (int g = 0; g < groups; ++g) {
        const int valid = std::min(G, M_tiles - g * G);
        tab[2 * g] = g * spg;
        tab[2 * g + 1] = spg;
        for (int sgi = 0; sgi < spg; ++sgi) {
            const int k0 = sgi * PK_SEGK, k1 = std::min(K_tiles, k0 + PK_SEGK);
            segs.push_back(TcSeg{0, g, k0, k1, g * spg + sgi});
            cost.push_back((double)(k1 - k0) * valid * TC_A_BYTES);
        }
    }
    const size_t part_elems = segs.size() * (size_t)Q * G * TC_BM;
    cudaError_t e;
    if ((e = cudaMallocAsync((void**)part, part_elems * sizeof(float), st))) return e;
    if ((e = cudaMallocAsync((void**)grp, tab.size() * sizeof(int), st))) return e;
    t->bytes += (long long)(part_elems * sizeof(float) + tab.size() * sizeof(int));
    if ((e = cudaMemcpyAsync(*grp, tab.data(), tab.size() * sizeof(int), cudaMemcpyHostToDevice, st))) return e;
    return cudaStreamSynchronize(st);   // the host table goes out of scope
}

}  // namespace

cudaError_t tc_pack_setup(cofem_ctx* c) {
    TcPlan* t = (TcPlan*)c->tc;
    if (!t || t->fused || t->f8) return cudaErrorNotSupported;
    if (t->pk_part1) return cudaSuccess;
    const long long before = t->bytes;
    cudaError_t e = pack_product(t, t->g1, t->tf, t->Q, t->pk_s1, t->pk_c1, &t->pk_part1, &t->pk_grp1, c->stream);
    if (e == cudaSuccess)
        e = pack_product(t, t->g2, t->tf, t->Q, t->pk_s2, t->pk_c2, &t->pk_part2, &t->pk_grp2, c->stream);
    c->bytes += t->bytes - before;
    return e;
}

void tc_pack_describe(cofem_ctx* c, PackedFit* out) {
    TcPlan* t = (TcPlan*)c->tc;
    auto fill = [&](TcSlot& sl, const GemmPlan& gp, const void* B, float* part) {
        sl.A = (const uint8_t*)gp.A;
        sl.B = (const uint8_t*)B;
        sl.ctl = c->ctl;
        sl.part = part;
        sl.idesc = gp.p.idesc;
        sl.idesc_lo = gp.p.idesc_lo;
        sl.K_tiles = gp.p.K_tiles;
        sl.M_tiles = gp.p.M_tiles;
        sl.QS = gp.p.QS;
        sl.QH = gp.p.QH;
        sl.Q = gp.p.Q;
    };
    fill(out->g1, t->g1, t->Vs, t->pk_part1);
    fill(out->g2, t->g2, t->Ts, t->pk_part2);
    out->s1 = t->pk_s1;
    out->s2 = t->pk_s2;
    out->c1 = t->pk_c1;
    out->c2 = t->pk_c2;
    out->tf = t->tf;
}

void tc_pack_vslot(cofem_ctx* c, VSlot* v) {
    TcPlan* t = (TcPlan*)c->tc;
    v->ctl = c->ctl;
    v->b = c->b;
    v->theta = c->theta;
    v->alpha = c->alpha;
    v->minv = c->minv;
    v->X = c->X;
    v->R = c->R;
    v->P = c->P;
    v->mu_out = c->mu_out;
    v->s_out = c->s_out;
    v->iters = c->iters_dev;
    v->D = c->D;
    v->Dp = c->Dp;
    v->Np = c->Np;
    v->nch = c->nch;
    v->Q = t->Q;
    v->part = c->part;
    v->counters = c->counters;
    v->so = SplitOut{t->Vs, t->tf ? 2 : 1, t->QS, t->QH, 1.0f};
    v->uo = OpOut{t->pk_part2, 1, 0, t->pk_grp2, t->G * TC_BM, 1.0f};
    v->t_part = t->pk_part1;
    v->t_grp = t->pk_grp1;
    v->GR = t->G * TC_BM;
    v->st = SplitOut{t->Ts, t->tf ? 2 : 1, t->QS, t->QH, 1.0f};
    v->tt_part = c->tt_part;
}

size_t tc_packed_smem(bool tf, int QSmax) { return gemm_smem(tf, QSmax); }

void launch_gemm_packed(Sink& s, bool tf, const TcBatch& b, int nCTA, size_t smem) {
    if (tf) s.launch_pdl(k_gemm_tc_packed<true>, dim3(nCTA), dim3(tc_threads(true)), smem, b);
    else s.launch_pdl(k_gemm_tc_packed<false>, dim3(nCTA), dim3(tc_threads(false)), smem, b);
}

void launch_reduce_T_packed(Sink& s, const VSlot* vs, const int4* map, const int* count, int nblocks) {
    s.launch_pdl(k_reduce_T_packed, dim3(nblocks), dim3(256), 0, vs, map, count);
}
