// Tensor-core (tcgen05) update of far-from-diagonal tiles for the
// mixed-precision Cholesky:  C[r, c] -= inv_s_r inv_s_c * (A B')[r, c]  with
// the panel rows scaled by a power of two s_r each (max |x| s_r < 2^14) and
// held as FP16 (or BF16), FP32 accumulation in tensor memory, FP64 C.
// With two terms the panel is split x s = hi + lo (both FP16) and the tile
// accumulates hi hi' + hi lo' + lo hi' (three MMAs per K step): about 22
// significant bits per operand instead of 11.
//
// Persistent: one CTA per SM walks a compact list of the 128 x 128 output
// tiles of the far class (nb-tile distance > band), K in 64-wide blocks.
//   warp 0 (one lane): TMA producer, 3-stage ring of (A, B) tiles (hi, and lo
//                      with two terms), 128 x 64 FP16 each, 128-byte swizzle,
//                      running ahead across tile boundaries;
//   warp 1: allocates 256 TMEM columns (two 128-column accumulators); one
//           lane issues tcgen05.mma (M = 128, N = 128, K = 16, kind::f16,
//           FP32 accumulate) into the accumulator of the tile's parity and
//           commits each stage back to the producer and each finished tile
//           to the epilogue;
//   warps 2-9: epilogue, tcgen05.ld of the accumulator (warp w reads TMEM
//           lanes 32 (w % 4) .. + 31 = tile rows, half of the columns each),
//           scale (in FP32: the scales are powers of two), FP64
//           read-modify-write of C with stores contiguous across
//           each warp; then it frees the accumulator, so the epilogue of one
//           tile overlaps the MMAs of the next.
// Every wait on an mbarrier is bounded by a clock budget; on expiry the
// thread records an error code in the status word and the CTA drains (its
// copies and MMAs in flight), frees its TMEM and returns.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "geo_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace tc {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int TILE_A_BYTES = BM * BK * 2;
constexpr int TILE_B_BYTES = BN * BK * 2;
constexpr int TILE_BYTES = TILE_A_BYTES;                   // A and B tiles have the same shape
constexpr int STAGE_BYTES = 4 * TILE_BYTES;                // A_hi, B_hi, A_lo, B_lo
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 1024;   // + alignment slack

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) { return smem_desc_sw128(saddr); }

// Instruction descriptor, kind::f16: D = F32, A = B = F16 (or BF16), both K-major, N = 128, M = 128.
__host__ __device__ constexpr uint32_t instr_desc(int bf16) { return instr_desc_f16(bf16, BM, BN); }

// The far tiles of one trailing update: nb-tiles (I, J) with I - J > band,
// T0 <= J, I <= T1, enumerated row by row (u = I - T0 - band - 1, v = J - T0
// <= u), each split into (nb / 128)^2 output tiles of 128 x 128; with col_only
// only the column J = T0 (u = I - T0 - band - 1, v = 0).
struct TcArgs {
    double *C;
    long long ldc;
    int N;                 // matrix order: rows and cols >= N are outside
    int prow0;             // global row of panel row 0 (A / B operand row = global - prow0)
    int K;                 // panel width (multiple of 64)
    int nb, band, T0;      // class geometry
    int col_only;          // 1: only nb-tile column T0
    long long ntiles;      // output tiles in the list
    const double *inv_scale;   // per panel row
    int terms;                 // 1: hi only, 2: hi + lo
    DevStatus *st;
};

constexpr int EPI_WARPS = 8;
constexpr int THREADS_P = 64 + 32 * EPI_WARPS;
constexpr int TMEM_COLS_P = 2 * BN;

// Global row / col of output tile L; false if it lies beyond the matrix.
__device__ __forceinline__ bool tile_coords(const TcArgs &a, long long L, int *gr, int *gc) {
    const int per = a.nb / BM;                       // 128-tiles per nb along each side
    const long long sub = L % ((long long)per * per), f = L / ((long long)per * per);
    long long u = f, v = 0;
    if (!a.col_only) {
        u = (long long)((sqrt(8.0 * (double)f + 1.0) - 1.0) * 0.5);
        while ((u + 1) * (u + 2) / 2 <= f) ++u;
        while (u * (u + 1) / 2 > f) --u;
        v = f - u * (u + 1) / 2;
    }
    const int I = a.T0 + a.band + 1 + (int)u, J = a.T0 + (int)v;
    *gr = I * a.nb + (int)(sub / per) * BM;
    *gc = J * a.nb + (int)(sub % per) * BN;
    return *gr < a.N;
}

__global__ void __launch_bounds__(THREADS_P, 1)
    k_tc_update(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map_lo,
                const TcArgs args, const uint32_t idesc) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], acc_full[2], acc_empty[2], drain_bar;
    __shared__ uint32_t tmem_slot;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    if (args.st->info) return;   // uniform: an earlier step failed
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int nk = args.K / BK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS_P)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    int *tword = &args.st->timeout;

    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;   // stages issued
            bool ok = true;
            for (long long L = blockIdx.x; L < args.ntiles && ok; L += gridDim.x) {
                int gr, gc;
                if (!tile_coords(args, L, &gr, &gc)) continue;
                const int arow = gr - args.prow0, brow = gc - args.prow0;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    if (g >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)(((g / STAGES) & 1) ^ 1), tword, 1)) {
                        ok = false;
                        break;
                    }
                    uint8_t *sa = smem + (size_t)s * STAGE_BYTES;
                    uint8_t *sb = sa + TILE_BYTES;
                    mbar_arrive_expect_tx(&full_bar[s], (args.terms == 2 ? 4 : 2) * TILE_BYTES);
                    tma_load_2d(&map, &full_bar[s], sa, kb * BK, arow);
                    tma_load_2d(&map, &full_bar[s], sb, kb * BK, brow);
                    if (args.terms == 2) {
                        tma_load_2d(&map_lo, &full_bar[s], sa + 2 * TILE_BYTES, kb * BK, arow);
                        tma_load_2d(&map_lo, &full_bar[s], sb + 2 * TILE_BYTES, kb * BK, brow);
                    }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the copies still in flight
                for (long long q = (g > STAGES ? g - STAGES : 0); q < g; ++q)
                    mbar_wait(&full_bar[q % STAGES], (uint32_t)((q / STAGES) & 1), tword, 2);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long long g = 0;
            int lt = 0;   // tiles of this CTA
            bool ok = true;
            for (long long L = blockIdx.x; L < args.ntiles && ok; L += gridDim.x) {
                int gr, gc;
                if (!tile_coords(args, L, &gr, &gc)) continue;
                const int b = lt & 1;
                if (lt >= 2 && !mbar_wait(&acc_empty[b], (uint32_t)(((lt >> 1) & 1) ^ 1), tword, 5)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(b * BN);
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((g / STAGES) & 1), tword, 3)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = smem_u32(smem + (size_t)s * STAGE_BYTES);
                    const uint32_t sb = sa + TILE_BYTES;
                    const uint32_t sal = sa + 2 * TILE_BYTES, sbl = sb + 2 * TILE_BYTES;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        mma_f16(acc, smem_desc(sa + kk * 32), smem_desc(sb + kk * 32), idesc, (kb | kk) != 0);
                        if (args.terms == 2) {
                            mma_f16(acc, smem_desc(sa + kk * 32), smem_desc(sbl + kk * 32), idesc, 1);
                            mma_f16(acc, smem_desc(sal + kk * 32), smem_desc(sb + kk * 32), idesc, 1);
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full[b]);
                ++lt;
            }
            // every MMA issued so far has completed before TMEM can be freed
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, tword, 6);
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..9; TMEM lane quarter q = warp % 4, column half h
        const int q = warp % 4, h = (warp - 2) / 4;
        int lt = 0;
        for (long long L = blockIdx.x; L < args.ntiles; L += gridDim.x) {
            int gr, gc;
            if (!tile_coords(args, L, &gr, &gc)) continue;
            const int b = lt & 1;
            bool ok = mbar_wait(&acc_full[b], (uint32_t)((lt >> 1) & 1), tword, 4);
            ok = __all_sync(0xffffffffu, ok);   // every lane takes part in tcgen05.ld
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int grow = gr + q * 32 + lane;
            const bool rin = grow < args.N;
            // the scales are powers of two: v / (s_r s_c) is exact in FP32 as well
            const float si = rin ? (float)args.inv_scale[grow - args.prow0] : 0.f;
            for (int c = 0; c < BN / 64; ++c) {
                const int col0 = h * (BN / 2) + c * 32;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * BN + col0), v);
                if (rin) {
#pragma unroll
                    for (int j0 = 0; j0 < 32; j0 += 8) {
                        double cv[8];
                        double *pc[8];
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int gcol = gc + col0 + j0 + j;
                            pc[j] = (gcol < args.N) ? args.C + (long long)gcol * args.ldc + grow : nullptr;
                            cv[j] = pc[j] ? *pc[j] : 0.0;
                        }
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (pc[j]) {
                                const float sj = (float)args.inv_scale[gc + col0 + j0 + j - args.prow0];
                                *pc[j] = cv[j] - (double)((v[j0 + j] * si) * sj);
                            }
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty[b]))
                                        : "memory");
            ++lt;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS_P)
                     : "memory");
    }
}

}  // namespace tc
