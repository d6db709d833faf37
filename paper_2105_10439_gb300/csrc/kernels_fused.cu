// Single-pass dense operator for a BF16 dictionary: U = Phi~^T (Phi~ V) with
// every byte of Phi~ read from HBM once per application (Alg. 2 "Apply
// matrix", Sec. III-B; the quantised dictionary of the BF16 form).
//
// The two-pass form (kernels_tc.cu) streams Phi~ for T = Phi~ V and a
// transposed copy for U = Phi~^T T: 2 N D bytes of HBM traffic.  Here the rows
// of Phi~ are taken in waves of GW groups (G row tiles of 128 rows each).  For
// wave w:
//   phase 1   T_w = Phi~_w V        stream-K over (group, 64-wide k tile) units
//                                   of the wave, one segment partial per (CTA,
//                                   group) as in the two-pass GEMM;
//   reduce    T_w = sum of the partials (fixed order), split into three bf16
//             terms (the B operand of phase 2), ||T_q||^2 partials for pi;
//   phase 2   U += Phi~_w^T T_w     each CTA owns fixed 128-column tiles of U and
//                                   keeps them in TMEM for the whole application.
// Phase 2 reads the same pre-tiled image tiles as phase 1, as an MN-major
// operand (the 128 x 64 tile read along its rows), shortly after phase 1
// fetched them, so they come from L2: one wave is 64 MiB at most and two
// waves are live at a time.  The CTAs are software-pipelined by one wave:
// phase 1 of wave w+1 is issued before phase 2 of wave w, so the grid-wide
// steps between phase 1 and phase 2 of a wave overlap the HBM stream.
//
// The grid is one CTA per SM, launched cooperatively (the CTAs wait on each
// other at two grid-wide counters per wave).  Every wait is bounded (mbarrier
// rounds, or 2 s of %globaltimer for a grid counter); a CTA that gives up sets
// COFEM_FLAG_DEVICE_TIMEOUT, which the other CTAs poll, and all of them drain
// their copies and MMAs, free TMEM and return.
//
// Warp roles (192 threads): warp 0 lane 0 issues the bulk copies, warp 1
// allocates TMEM and lane 0 issues the MMAs, warps 2-5 drain the phase-1
// accumulators, run the reduction and write U at the end.
#include <algorithm>
#include <vector>

#include "cofem_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int FU_NE = 4, FU_NB = 3, FU_THREADS = 192, FU_BM = 128, FU_G = 2;
constexpr uint32_t FU_TILE = 16384;                 // 128 rows x 64 bf16
constexpr uint32_t FU_EBYTES = FU_G * FU_TILE;      // A-ring element: one unit (G tiles), one bulk copy
constexpr int FU_ACC_STRIDE = 128;                  // TMEM columns per accumulator
constexpr int FU_DEPTH = 2;                         // waves of phase 1 issued ahead of phase 2

struct FusedParams {
    const uint8_t* A;      // tiled Phi~: tile (g, k, r) at byte ((g K_tiles + k) G + r) 16384
    const uint8_t* Bv;     // split(V) image: k tile (64 columns of D) at byte k QS 128
    uint8_t* Bt;           // split(T) image: k tile (64 rows of N) at byte k QS 128
    float* part;           // phase-1 segment partials, two wave buffers: [w & 1][segment][Q][G 128]
    float* U;              // Q x Dp result
    double* tt_part;       // [Q][gridDim.x] partials of ||T_q||^2
    unsigned* sync;        // [0] partials posted, [1] T ready, [2] CTAs done
    const int* seg_base;   // [wave][CTA + 1]: first segment of the CTA within the wave
    const int* grp_seg;    // [wave][group of the wave][2]: first segment, count
    DevCtl* ctl;
    unsigned* flags;       // DevCtl::flags
    long long Dp;
    int seg_cap;           // segments per wave buffer
    int K_tiles, M_tiles, groups, GW, NW, Dt;
    int Q, QS;
    uint32_t idesc_k;      // M = 128, N = QS, A and B K-major
    uint32_t idesc_t;      // the same with A MN-major
    int mode;
};

__device__ __forceinline__ void grid_arrive(unsigned* ctr) {
    __threadfence();
    atomicAdd(ctr, 1u);
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

__global__ void __launch_bounds__(FU_THREADS, 1) k_operator_fused(FusedParams p) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t B_BYTES = (uint32_t)p.QS * 128u;   // one 64-wide k tile of a split block
    const uint32_t BS_BYTES = 2 * B_BYTES;              // B-ring slot: two k tiles
    uint8_t* ringA = smem;
    uint8_t* ringB = smem + FU_NE * FU_EBYTES;
    uint64_t* bars = (uint64_t*)(ringB + FU_NB * BS_BYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + FU_NE;
    uint64_t* b_full = bars + 2 * FU_NE;
    uint64_t* b_empty = b_full + FU_NB;
    uint64_t* acc_full = b_empty + FU_NB;
    uint64_t* acc_empty = acc_full + 1;
    uint64_t* u_full = acc_full + 2;
    uint64_t* drain = acc_full + 3;
    uint32_t* tmem_slot = (uint32_t*)(acc_full + 4);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    volatile int* s_flag = (volatile int*)(tmem_slot + 2);   // epilogue broadcast / last-CTA flag
    float4* red = (float4*)(tmem_slot + 4);                   // 128 float4 (16-byte aligned)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n = gridDim.x, c = blockIdx.x;
    const int KT = p.K_tiles, G = FU_G, GR = FU_G * FU_BM;
    const int n_own = c < p.Dt ? (p.Dt - 1 - c) / n + 1 : 0;   // U tiles j = c, c + n, ...

    if (threadIdx.x == 0) {
        for (int i = 0; i < FU_NE; ++i) {
            mbar_init(smem_u32(a_full + i), 1);
            mbar_init(smem_u32(a_empty + i), 1);
        }
        for (int i = 0; i < FU_NB; ++i) {
            mbar_init(smem_u32(b_full + i), 1);
            mbar_init(smem_u32(b_empty + i), 1);
        }
        mbar_init(smem_u32(acc_full), 1);
        mbar_init(smem_u32(acc_empty), 4);
        mbar_init(smem_u32(u_full), 1);
        mbar_init(smem_u32(drain), 1);
        *abort_flag = 0;
        *s_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // unit range of this CTA in wave w (units g K_tiles + k of the wave's groups)
    auto wave_units = [&](int w, long long& u0, long long& u1) {
        const int g0 = w * p.GW, g1 = min(p.groups, g0 + p.GW);
        const long long U0 = (long long)g0 * KT, Wn = (long long)(g1 - g0) * KT;
        u0 = U0 + (long long)c * Wn / n;
        u1 = U0 + (long long)(c + 1) * Wn / n;
    };
    // row tiles of wave w that hold rows of Phi~
    auto wave_rows = [&](int w, int& r0, int& r1) {
        r0 = w * p.GW * G;
        r1 = min(p.M_tiles, r0 + p.GW * G);
    };

    long long na = 0, nb = 0;   // copies issued into the A and B rings (producer thread)
    if (warp == 0) {
        if (lane == 0) {
            // ---------------- bulk-copy producer ----------------
            uint64_t evict_first;
            asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(evict_first));
            auto getA = [&](const uint8_t* src, uint32_t bytes, bool last_use) -> bool {
                const int slot = (int)(na % FU_NE);
                const long long use = na / FU_NE;
                if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag))
                    return false;
                mbar_expect_tx(smem_u32(a_full + slot), bytes);
                if (last_use)
                    bulk_load_hint(smem_u32(ringA + (size_t)slot * FU_EBYTES), src, bytes, smem_u32(a_full + slot),
                                   evict_first);
                else
                    bulk_load(smem_u32(ringA + (size_t)slot * FU_EBYTES), src, bytes, smem_u32(a_full + slot));
                ++na;
                return true;
            };
            // an element passed over without data (a phase-2 pair must start at an
            // even ring position, so its two elements are adjacent in shared memory)
            auto skipA = [&]() -> bool {
                const int slot = (int)(na % FU_NE);
                const long long use = na / FU_NE;
                if (use > 0 && !mbar_wait(smem_u32(a_empty + slot), (uint32_t)((use - 1) & 1), abort_flag))
                    return false;
                mbar_arrive(smem_u32(a_full + slot));
                ++na;
                return true;
            };
            auto getB = [&](const uint8_t* src, uint32_t bytes) -> bool {
                const int slot = (int)(nb % FU_NB);
                const long long use = nb / FU_NB;
                if (use > 0 && !mbar_wait(smem_u32(b_empty + slot), (uint32_t)((use - 1) & 1), abort_flag))
                    return false;
                mbar_expect_tx(smem_u32(b_full + slot), bytes);
                bulk_load(smem_u32(ringB + (size_t)slot * BS_BYTES), src, bytes, smem_u32(b_full + slot));
                ++nb;
                return true;
            };
            auto phase1 = [&](int w) -> bool {
                long long u0, u1;
                wave_units(w, u0, u1);
                for (long long u = u0; u < u1; ++u) {
                    const int k = (int)(u % KT);
                    if (!getB(p.Bv + (size_t)k * B_BYTES, B_BYTES)) return false;
                    if (!getA(p.A + (size_t)u * G * FU_TILE, FU_EBYTES, false)) return false;
                }
                return true;
            };
            auto phase2 = [&](int w) -> bool {
                if (n_own == 0) return true;
                const int g0 = w * p.GW, g1 = min(p.groups, g0 + p.GW);
                bool ready = false;
                for (int g = g0; g < g1; ++g) {
                    const int valid = min(G, p.M_tiles - g * G);
                    for (int i = 0; i < n_own; ++i) {
                        const int j = c + i * n;   // units (g, 2j) and (g, 2j + 1): adjacent elements
                        if ((na & 1) && !skipA()) return false;
                        for (int h = 0; h < 2; ++h)
                            if (!getA(p.A + ((size_t)g * KT + 2 * j + h) * G * FU_TILE, FU_EBYTES, true)) return false;
                        if (i > 0) continue;
                        if (!ready) {   // the split of T_w is written by all CTAs
                            if (!grid_wait(p.sync + 1, (unsigned)((w + 1) * n), abort_flag, p.flags)) return false;
                            asm volatile("fence.proxy.async.global;" ::: "memory");
                            ready = true;
                        }
                        for (int rr = 0; rr < valid; ++rr)   // k tiles 2r, 2r + 1 of split(T), r = g G + rr
                            if (!getB(p.Bt + (size_t)(2 * (g * G + rr)) * B_BYTES, 2 * B_BYTES)) return false;
                    }
                }
                return true;
            };
            bool ok = true;
            for (int w = 0; ok && w < FU_DEPTH && w < p.NW; ++w) ok = phase1(w);
            for (int w = 0; ok && w < p.NW; ++w) {
                if (w + FU_DEPTH < p.NW) ok = phase1(w + FU_DEPTH);
                if (ok) ok = phase2(w);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            long long ma = 0, mb = 0;
            int nseg = 0;
            auto takeA = [&](int& slot) -> bool {
                slot = (int)(ma % FU_NE);
                if (!mbar_wait(smem_u32(a_full + slot), (uint32_t)((ma / FU_NE) & 1), abort_flag)) return false;
                ++ma;
                return true;
            };
            auto takeB = [&](int& slot) -> bool {
                slot = (int)(mb % FU_NB);
                if (!mbar_wait(smem_u32(b_full + slot), (uint32_t)((mb / FU_NB) & 1), abort_flag)) return false;
                ++mb;
                return true;
            };
            auto phase1 = [&](int w) -> bool {
                long long u0, u1;
                wave_units(w, u0, u1);
                long long u = u0;
                while (u < u1) {
                    const int g = (int)(u / KT);
                    const long long seg_end = min(u1, (long long)(g + 1) * KT);
                    if (nseg > 0 && !mbar_wait(smem_u32(acc_empty), (uint32_t)((nseg - 1) & 1), abort_flag))
                        return false;
                    tc_fence_after();
                    const long long seg_start = u;
                    for (; u < seg_end; ++u) {
                        int sb, sa;
                        if (!takeB(sb) || !takeA(sa)) return false;
                        tc_fence_after();
                        const uint64_t db = desc_sw128(smem_u32(ringB + (size_t)sb * BS_BYTES));
                        for (int r = 0; r < G; ++r) {
                            const uint64_t da = desc_sw128(smem_u32(ringA + (size_t)sa * FU_EBYTES + r * FU_TILE));
                            const uint32_t dt = tmem + (uint32_t)(r * FU_ACC_STRIDE);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_bf16(dt, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), p.idesc_k,
                                         (u > seg_start || kk > 0) ? 1u : 0u);
                        }
                        mma_commit(smem_u32(a_empty + sa));
                        mma_commit(smem_u32(b_empty + sb));
                    }
                    mma_commit(smem_u32(acc_full));
                    ++nseg;
                }
                return true;
            };
            auto phase2 = [&](int w) -> bool {
                if (n_own == 0) return true;
                const int g0 = w * p.GW, g1 = min(p.groups, g0 + p.GW);
                for (int g = g0; g < g1; ++g) {
                    const int valid = min(G, p.M_tiles - g * G);
                    int sbs[FU_G];
                    for (int i = 0; i < n_own; ++i) {
                        int sa, sa1;
                        if (ma & 1) {   // element passed over by the producer
                            if (!takeA(sa)) return false;
                            mbar_arrive(smem_u32(a_empty + sa));
                        }
                        if (!takeA(sa) || !takeA(sa1)) return false;
                        if (sa1 != sa + 1) {   // cannot happen: pairs start at even positions
                            *abort_flag = 1;
                            return false;
                        }
                        if (i == 0)
                            for (int rr = 0; rr < valid; ++rr)
                                if (!takeB(sbs[rr])) return false;
                        tc_fence_after();
                        const uint32_t dt = tmem + (uint32_t)((G + i) * FU_ACC_STRIDE);
                        for (int rr = 0; rr < valid; ++rr) {
                            // 128 x 128 block of Phi~ (row tile g G + rr, k tiles 2j and 2j + 1 in
                            // adjacent elements, 32 KiB apart), read as A = Phi~^T: M along the
                            // columns, K along the rows
                            const uint64_t da = desc_sw128_mn(
                                smem_u32(ringA + (size_t)sa * FU_EBYTES + rr * FU_TILE), FU_EBYTES, 1024);
                            const uint64_t db0 = desc_sw128(smem_u32(ringB + (size_t)sbs[rr] * BS_BYTES));
#pragma unroll
                            for (int s = 0; s < 8; ++s) {   // 16 rows per step: 2048 bytes of A
                                const uint64_t db =
                                    db0 + (uint64_t)(s < 4 ? 0u : (B_BYTES >> 4)) + (uint64_t)(2 * (s & 3));
                                mma_bf16(dt, da + (uint64_t)(128 * s), db, p.idesc_t,
                                         (w > 0 || g > g0 || rr > 0 || s > 0) ? 1u : 0u);
                            }
                        }
                        mma_commit(smem_u32(a_empty + sa));
                        mma_commit(smem_u32(a_empty + sa1));
                    }
                    for (int rr = 0; rr < valid; ++rr) mma_commit(smem_u32(b_empty + sbs[rr]));
                }
                return true;
            };
            bool ok = true;
            for (int w = 0; ok && w < FU_DEPTH && w < p.NW; ++w) ok = phase1(w);
            for (int w = 0; ok && w < p.NW; ++w) {
                if (w + FU_DEPTH < p.NW) ok = phase1(w + FU_DEPTH);
                if (ok) ok = phase2(w);
            }
            if (ok) mma_commit(smem_u32(u_full));
            // every issued MMA must finish before TMEM is released
            mma_commit(smem_u32(drain));
            mbar_drain(smem_u32(drain), 0);
        }
    } else {
        // ------- epilogue warps: phase-1 partials, reduction of T, U -------
        const int sub = warp & 3;
        const int e = threadIdx.x - 64;                 // 0 .. 127
        const int S = max(1, 128 / p.Q);                // segment slices per column
        const int q_e = e / S, sl_e = e % S;
        const bool has_q = e < S * p.Q;
        const int row = 32 * sub + lane;
        const SplitOut so{p.Bt, 1, p.QS, 0};
        float tt = 0.0f;                                // ||T_q||^2 of the rows reduced here (slice 0)
        int nseg = 0;
        bool ok = true;
        for (int w = 0; ok && w < p.NW; ++w) {
            // (1) this CTA's phase-1 segments of wave w -> partials
            long long u0, u1;
            wave_units(w, u0, u1);
            const int* sbase = p.seg_base + (size_t)w * (n + 1);
            long long u = u0;
            int sl = 0;
            while (u < u1) {
                const int g = (int)(u / KT);
                const long long seg_end = min(u1, (long long)(g + 1) * KT);
                if (!mbar_wait(smem_u32(acc_full), (uint32_t)(nseg & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                // two buffers by wave parity: a CTA writes wave w + 1's partials while
                // slower CTAs may still read wave w's in their reduction
                float* out = p.part + ((size_t)(w & 1) * p.seg_cap + sbase[c] + sl) * p.Q * GR;
                for (int r = 0; r < G; ++r) {
                    const uint32_t tbase = tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(r * FU_ACC_STRIDE);
                    for (int qb = 0; qb * 16 < p.Q; ++qb) {
                        uint32_t v[48];
                        const int c0 = 3 * qb, NC = p.QS / 16;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc)
                            if (c0 + cc < NC) tmem_ld16(tbase + (uint32_t)((c0 + cc) * 16), v + 16 * cc);
                        tmem_ld_wait(v, 48);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int q = 16 * qb + i;
                            if (q < p.Q)
                                out[(size_t)q * GR + r * FU_BM + row] = __uint_as_float(v[3 * i]) +
                                                                       __uint_as_float(v[3 * i + 1]) +
                                                                       __uint_as_float(v[3 * i + 2]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(acc_empty));
                ++nseg;
                ++sl;
                u = seg_end;
            }
            if (!ok) break;
            // (2) all partials of wave w posted
            epi_sync();
            if (e == 0) {
                grid_arrive(p.sync + 0);
                *s_flag = grid_wait(p.sync + 0, (unsigned)((w + 1) * n), abort_flag, p.flags) ? 1 : 0;
            }
            epi_sync();
            if (!*s_flag) {
                ok = false;
                break;
            }
            // (3) T_w: chunks of 4 rows, chunk ci handled by CTA ci mod n; thread
            // (q, slice) sums the slice's segments, slice 0 adds the slices in order
            int r0, r1;
            wave_rows(w, r0, r1);
            const int RC = (r1 - r0) * (FU_BM / 4);
            for (int ci = c; ci < RC; ci += n) {
                const long long i = (long long)r0 * FU_BM + 4LL * ci;       // first row of the chunk
                const int gw = (int)(i / GR) - w * p.GW, rig = (int)(i % GR);
                const int* gs = p.grp_seg + ((size_t)w * p.GW + gw) * 2;
                const int s0 = (w & 1) * p.seg_cap + gs[0], ns = gs[1];
                float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
                if (has_q) {
                    // eight independent loads in flight, added in segment order
                    const float* base = p.part + ((size_t)s0 * p.Q + q_e) * GR + rig;
                    const size_t sstride = (size_t)p.Q * GR;
                    for (int s = sl_e; s < ns; s += 8 * S) {
                        float4 b[8];
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const int ss = s + t * S;
                            b[t] = ss < ns ? __ldcg(reinterpret_cast<const float4*>(base + (size_t)ss * sstride))
                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                        }
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            a.x += b[t].x; a.y += b[t].y; a.z += b[t].z; a.w += b[t].w;
                        }
                    }
                    red[e] = a;
                }
                epi_sync();
                if (has_q && sl_e == 0) {
                    for (int t = 1; t < S; ++t) {
                        const float4 b = red[e + t];
                        a.x += b.x; a.y += b.y; a.z += b.z; a.w += b.w;
                    }
                    store_split(so, q_e, i, a);
                    tt += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
                }
                epi_sync();
            }
            // (4) the split of T_w is complete once every CTA arrived
            asm volatile("fence.proxy.async.global;" ::: "memory");
            epi_sync();
            if (e == 0) grid_arrive(p.sync + 1);
        }
        // (5) U tiles owned by this CTA
        if (ok && n_own > 0) {
            if (mbar_wait(smem_u32(u_full), 0u, abort_flag)) {
                tc_fence_after();
                for (int ii = 0; ii < n_own; ++ii) {
                    const long long j0 = (long long)(c + ii * n) * FU_BM;
                    const uint32_t tbase =
                        tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)((G + ii) * FU_ACC_STRIDE);
                    for (int qb = 0; qb * 16 < p.Q; ++qb) {
                        uint32_t v[48];
                        const int c0 = 3 * qb, NC = p.QS / 16;
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc)
                            if (c0 + cc < NC) tmem_ld16(tbase + (uint32_t)((c0 + cc) * 16), v + 16 * cc);
                        tmem_ld_wait(v, 48);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int q = 16 * qb + i;
                            if (q < p.Q)
                                p.U[(size_t)q * p.Dp + j0 + row] = __uint_as_float(v[3 * i]) +
                                                                   __uint_as_float(v[3 * i + 1]) +
                                                                   __uint_as_float(v[3 * i + 2]);
                        }
                    }
                }
            }
        }
        if (has_q && sl_e == 0) p.tt_part[(size_t)q_e * n + c] = (double)tt;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) {
        // some role gave up: the latest copy issued into every ring slot must
        // land before the CTA exits
        for (int s = 0; s < FU_NE; ++s) {
            const long long n_s = na > s ? (na - s + FU_NE - 1) / FU_NE : 0;
            if (n_s > 0) mbar_drain(smem_u32(a_full + s), (uint32_t)((n_s - 1) & 1));
        }
        for (int s = 0; s < FU_NB; ++s) {
            const long long n_s = nb > s ? (nb - s + FU_NB - 1) / FU_NB : 0;
            if (n_s > 0) mbar_drain(smem_u32(b_full + s), (uint32_t)((n_s - 1) & 1));
        }
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
    if (threadIdx.x == 0) {
        if (*abort_flag) atomicOr(p.flags, COFEM_FLAG_DEVICE_TIMEOUT);
        __threadfence();
        *s_flag = atomicAdd(p.sync + 2, 1u) == (unsigned)(n - 1) ? 2 : 0;
    }
    __syncthreads();
    if (*s_flag == 2) {
        // last CTA: every other CTA has passed all its waits; reset the counters
        // for the next launch and finish pi / gamma
        __threadfence();
        if (threadIdx.x == 0) {
            p.sync[0] = 0;
            p.sync[1] = 0;
            p.sync[2] = 0;
        }
        if (p.mode == OP_CG) {   // the update kernel reduces the partials
            if (threadIdx.x == 0) op_cg_begin(p.ctl, p.tt_part, n);
        } else {
            op_finalize_block(p.ctl, p.tt_part, n, p.Q);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct FusedPlan {
    FusedParams p{};
    int nCTA = 0;
    size_t smem = 0;
    int* tables = nullptr;          // seg_base then grp_seg
    float* part = nullptr;
    double* tt = nullptr;
    unsigned* sync = nullptr;
    long long bytes = 0;
};

size_t fused_smem_bytes(int QS) {
    return 1024 + (size_t)FU_NE * FU_EBYTES + (size_t)FU_NB * 2 * QS * 128 + 8 * (2 * FU_NE + 2 * FU_NB + 4) + 16 +
           128 * 16 + 64;
}

// Whether the single-pass form applies: BF16 images, N = 3Q terms in one
// accumulator (QS <= 128), at most two 128-column U tiles per CTA in TMEM, and
// a cooperative launch of one CTA per SM.
bool fused_supported(int num_sms, long long Dp, int QS, bool coop, int max_smem) {
    const long long Dt = Dp / FU_BM;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_operator_fused) != cudaSuccess) return false;
    return coop && QS <= 128 && Dt <= 2LL * num_sms &&
           (long long)fused_smem_bytes(QS) + (long long)fa.sharedSizeBytes <= max_smem;
}

cudaError_t fused_create(FusedPlan** out, int num_sms, long long Np, long long Dp, int Q, int QS,
                         const void* A_image, const void* Bv, void* Bt, float* U, DevCtl* ctl, cudaStream_t st,
                         long long* bytes) {
    FusedPlan* fp = new FusedPlan();
    *out = fp;
    FusedPlan& f = *fp;
    FusedParams& p = f.p;
    p.K_tiles = (int)(Dp / 64);
    p.M_tiles = (int)((Np + FU_BM - 1) / FU_BM);
    p.groups = (p.M_tiles + FU_G - 1) / FU_G;
    p.GW = 2;                                  // 4 row tiles: 512 rows, 32 MiB at D = 32768
    p.NW = (p.groups + p.GW - 1) / p.GW;
    p.Dt = (int)(Dp / FU_BM);
    p.Q = Q;
    p.QS = QS;
    p.Dp = Dp;
    p.idesc_k = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(QS >> 3) << 17) | ((uint32_t)(FU_BM >> 4) << 24);
    p.idesc_t = p.idesc_k | (1u << 15);        // A MN-major
    p.A = (const uint8_t*)A_image;
    p.Bv = (const uint8_t*)Bv;
    p.Bt = (uint8_t*)Bt;
    p.U = U;
    p.ctl = ctl;
    p.flags = &ctl->flags;
    f.nCTA = num_sms;
    const int n = f.nCTA;
    // per wave: the segment tables of the stream-K split
    std::vector<int> seg_base((size_t)p.NW * (n + 1)), grp((size_t)p.NW * p.GW * 2, 0);
    int max_seg = 0;
    for (int w = 0; w < p.NW; ++w) {
        const int g0 = w * p.GW, g1 = std::min(p.groups, g0 + p.GW);
        const long long U0 = (long long)g0 * p.K_tiles, Wn = (long long)(g1 - g0) * p.K_tiles;
        int nseg = 0;
        std::vector<int> first(p.GW, -1), count(p.GW, 0);
        for (int c = 0; c < n; ++c) {
            seg_base[(size_t)w * (n + 1) + c] = nseg;
            const long long u0 = U0 + (long long)c * Wn / n, u1 = U0 + (long long)(c + 1) * Wn / n;
            long long u = u0;
            while (u < u1) {
                const int g = (int)(u / p.K_tiles);
                if (first[g - g0] < 0) first[g - g0] = nseg;
                ++count[g - g0];
                ++nseg;
                u = std::min(u1, (long long)(g + 1) * p.K_tiles);
            }
        }
        seg_base[(size_t)w * (n + 1) + n] = nseg;
        for (int gw = 0; gw < p.GW; ++gw) {
            grp[((size_t)w * p.GW + gw) * 2] = first[gw] < 0 ? 0 : first[gw];
            grp[((size_t)w * p.GW + gw) * 2 + 1] = count[gw];
        }
        max_seg = std::max(max_seg, nseg);
    }
    cudaError_t e;
    const size_t ntab = seg_base.size() + grp.size();
    if ((e = cudaMallocAsync(&f.tables, ntab * sizeof(int), st))) return e;
    p.seg_cap = max_seg;
    const size_t part_elems = 2 * (size_t)max_seg * Q * FU_G * FU_BM;
    if ((e = cudaMallocAsync(&f.part, part_elems * sizeof(float), st))) return e;
    if ((e = cudaMallocAsync(&f.tt, (size_t)Q * n * sizeof(double), st))) return e;
    if ((e = cudaMallocAsync(&f.sync, 4 * sizeof(unsigned), st))) return e;
    f.bytes = (long long)ntab * 4 + (long long)part_elems * 4 + (long long)Q * n * 8 + 16;
    *bytes += f.bytes;
    if ((e = cudaMemcpyAsync(f.tables, seg_base.data(), seg_base.size() * sizeof(int), cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemcpyAsync(f.tables + seg_base.size(), grp.data(), grp.size() * sizeof(int),
                             cudaMemcpyHostToDevice, st)))
        return e;
    if ((e = cudaMemsetAsync(f.sync, 0, 4 * sizeof(unsigned), st))) return e;
    if ((e = cudaStreamSynchronize(st))) return e;   // the host tables go out of scope
    p.seg_base = f.tables;
    p.grp_seg = f.tables + seg_base.size();
    p.part = f.part;
    p.tt_part = f.tt;
    p.sync = f.sync;
    f.smem = fused_smem_bytes(QS);
    return cudaSuccess;
}

void fused_destroy(FusedPlan* f, cudaStream_t st) {
    if (!f) return;
    if (f->tables) cudaFreeAsync(f->tables, st);
    if (f->part) cudaFreeAsync(f->part, st);
    if (f->tt) cudaFreeAsync(f->tt, st);
    if (f->sync) cudaFreeAsync(f->sync, st);
    delete f;
}

void launch_fused(Sink& s, const FusedPlan* f, int mode) {
    FusedParams p = f->p;
    p.mode = mode;
    s.launch_cooperative(k_operator_fused, dim3(f->nCTA), dim3(FU_THREADS), f->smem, p);
}

cudaError_t fused_kernel_attributes(int max_smem) {
    // the opt-in limit covers static plus dynamic shared memory
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, k_operator_fused);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_operator_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_smem - (int)fa.sharedSizeBytes);
}
