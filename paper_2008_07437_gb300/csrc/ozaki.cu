// FP64-accurate matrix products on the BF16 tensor cores (the Ozaki scheme:
// error-free splitting into short integer digits), and the dense Cholesky
// factorisation of Sec. 5.2 with its trailing updates (the SYRK / GEMM tile
// tasks of Sec. 5.1) computed that way.
//
// GB300 runs FP64 at about 1.26 TFLOP/s but BF16 MMAs at ~1,900 TFLOP/s.
// Ozaki, Ogita, Oishi and Rump (Numer. Algorithms 59, 2012) split each
// operand into slices whose pairwise products a lower-precision unit computes
// without rounding error; summing the products in high precision recovers the
// FP64 product.  Here:
//
//   row scale   every operand row r gets e_r with max_k |x_rk| < 2^e_r;
//   digits      X = rint(x 2^(7S - 1 - e_r)) is an integer of at most 7S bits;
//               its balanced base-128 digits d_1 .. d_S (d_1 the most
//               significant, |d_1| <= 64, -64 <= d_t < 64 after it) give
//               x ~= 2^e_r sum_t d_t 2^(1 - 7t), with |error| <= 2^(e_r - 7S);
//   products    level l = t + u collects d_t(a) d_u(b), scale 2^(2 - 7l); the
//               levels l <= S + 1 are kept (S(S+1)/2 products), the rest
//               would change the result by about 2^-7S relative;
//   exactness   each digit is an integer in [-64, 64], exact in BF16, each
//               product is an integer of magnitude <= 2^12, and a level holds
//               at most S products: over a depth K with S K 2^12 <= 2^24 every
//               partial sum in the FP32 tensor-memory accumulator is an
//               integer below 2^24, so the tensor cores add without rounding
//               (the depth of one launch is capped at kmax = 4096 / S);
//   recombine   the epilogue converts each level to an integer and folds
//               groups of four levels (2..5, 6..9) into 64-bit integers
//               (exact: below 2^46), then applies
//               C -= 2^(e_r + e_c) sum_w W_w 2^(2 - 7 hi_w), hi_w the last
//               level of group w, with one FP64 FMA per group.
//
//   level cut  (optional, trailing updates of the factorisation) the levels
//               kept for an output tile follow its operands' magnitudes: with
//               E the largest row exponent of the launch's A rows plus that of
//               its B rows, and e_i + e_j the same over the tile's own rows,
//               the tile keeps the levels l <= S + 1 - q, q = floor((E - e_i - e_j) / 7).
//               A level-l term is at most 2^(e_i + e_j + 14 - 7 l), so the
//               first level such a tile drops, S + 2 - q, is at most
//               2^(e_i + e_j + 7 q - 7 S) <= 2^(E - 7 S): no larger than the
//               first level the launch's largest tile drops without the cut.
//               Every entry's error thus stays within the bound of the
//               launch's largest products; tiles whose operands are tiny
//               against the largest (far from the diagonal in a spatially
//               ordered covariance) skip levels or vanish entirely.
//
// The kernel is persistent (one CTA per SM) over 128 x BN output tiles, the
// K range in chunks of BK.  TMEM (512 columns) holds 512 / BN level
// accumulators of 128 x BN FP32: with BN = 64 all eight levels of 8 slices
// fit and a tile is one pass over K; with BN = 128 (used from 6 slices on,
// where the 128-row A operand read per 128 x 64 MMA otherwise keeps the MMA
// issue path twice as busy as the math) the level groups run as passes over
// K, each loading only the slices its levels use and writing its part of C.
//   warp 0, one lane: TMA producer, ring of K chunks (32 or 64-byte rows,
//     swizzled to match), each chunk holding the digit slices of the A rows
//     (128 x BK BF16 each) and of the B rows (BN x BK each);
//   warp 1: allocates the 512 TMEM columns; one lane issues tcgen05.mma
//     kind::f16 (M 128, N BN, K 16) level by level from precomputed shared
//     memory descriptors and commits chunks back to the producer;
//   warps 2-9: epilogue; tcgen05.ld of each level, releasing that
//     accumulator slot as soon as it is read (the MMAs of the next pass or
//     tile may start into it while the epilogue folds the values in
//     registers), then the FP64 read-modify-write of C (with the level cut,
//     C comes through shared memory by cp.async, four columns at a time,
//     double-buffered, so that no register waits on a load of C).
// With the level cut each CTA first computes the cut of all its tiles into a
// shared-memory table, and the MMA thread counts the products it issues
// (the device-side tensor work of the profile).
// Every mbarrier wait is bounded; on expiry the thread records a code in the
// status word, the CTA drains what it has in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "geo_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace {

using namespace tc;

constexpr int OZ_BM = 128;        // output rows per tile (MMA M, TMEM lanes)
constexpr int OZ_KALIGN = 32;     // slice arrays: K padded to a multiple of 32 (64-byte rows)
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_SMEM_CAP = 200 * 1024;   // the ring of K chunks; the rest: level-cut table, C staging
constexpr int OZ_LC_CAP = 8192;           // tiles per CTA whose level cut is computed up front
constexpr int OZ_GROUP = 8;       // row blocks swept together (operand reuse in L2)
constexpr int OZ_LPW = 4;         // levels folded into one 64-bit word
constexpr int OZ_E_NONE = -4096;  // block exponent of rows that are all zero (or absent)

// Tile width BN (MMA N), K chunk BK (16: 32-byte rows, 32-byte swizzle; 32:
// 64-byte rows, 64-byte swizzle).  TMEM holds 512 / BN level accumulators, so
// the S levels are processed in passes of WPP words over the whole K range;
// each pass loads only the slices its levels use.
template <int S, int BN, int BK>
struct OzCfg {
    static constexpr int NWT = (S + OZ_LPW - 1) / OZ_LPW;            // words of <= 4 levels (levels 2 .. S+1)
    static constexpr int WPP = OZ_TMEM_COLS / (BN * OZ_LPW);          // words per pass
    static constexpr int PASSES = (NWT + WPP - 1) / WPP;
    static constexpr int WREG = WPP < NWT ? WPP : NWT;                // words an epilogue thread holds
    static constexpr int A_BYTES = OZ_BM * BK * 2;
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = S * (A_BYTES + B_BYTES);      // the widest pass uses every slice
    static constexpr int STAGES = (OZ_SMEM_CAP / STAGE_BYTES) < 6 ? (OZ_SMEM_CAP / STAGE_BYTES) : 6;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
    static constexpr int CPT = BN / 2;                                // columns per epilogue thread
    // levels of pass g: [lev_lo, lev_hi]; slices it reads: 1 .. tmax
    __host__ __device__ static constexpr int lev_lo(int g) { return 2 + OZ_LPW * WPP * g; }
    __host__ __device__ static constexpr int lev_hi(int g) {
        return (1 + OZ_LPW * WPP * (g + 1)) < (S + 1) ? (1 + OZ_LPW * WPP * (g + 1)) : (S + 1);
    }
    __host__ __device__ static constexpr int tmax(int g) { return (lev_hi(g) - 1) < S ? (lev_hi(g) - 1) : S; }
    // last level of word w (its unit is 2^(2 - 7 hi))
    __host__ __device__ static constexpr int word_hi(int w) {
        return (5 + OZ_LPW * w) < (S + 1) ? (5 + OZ_LPW * w) : (S + 1);
    }
};

struct OzArgs {
    double *C;
    long long ldc;
    int r0, c0;          // global row / col of the region's first output
    int m_end, n_end;    // outputs with global row >= m_end or col >= n_end are not written
    int mt, nt;          // 128-row x BN-col tiles of the region
    int tri;             // write only global row >= global col; skip tiles entirely above the diagonal
    int overwrite;       // 1: C = -A B' (C is not read)
    int a_off, b_off;    // slice row of the region's first row (A) / first column (B)
    int nk;              // K chunks of BK
    const int *ea, *eb;  // per-row exponents of the A / B slices
    // level cut: per 32-row block maxima of the row exponents over every row (ba, bb) and over the
    // reference rows (ra, rb) of the A / B slices, nba / nbb blocks; cut = 0 keeps every level
    const int *ba, *bb, *ra, *rb;
    int nba, nbb, cut;
    unsigned long long *tc_flops;   // tensor-core flops issued, summed over CTAs (may be NULL)
    DevStatus *st;
};

__device__ __forceinline__ long long ntiles_all(const OzArgs &a) { return (long long)a.mt * a.nt; }

__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Highest level an output tile keeps (< 2: the tile is skipped); eref = E_A + E_B.
template <int S, int BN>
__device__ __forceinline__ int oz_lcut(const OzArgs &a, int ar, int br, int eref) {
    if (!a.cut) return S + 1;
    int ei = OZ_E_NONE, ej = OZ_E_NONE;
    const int a1 = min((ar + OZ_BM - 1) >> 5, a.nba - 1), b1 = min((br + BN - 1) >> 5, a.nbb - 1);
    for (int b = ar >> 5; b <= a1; ++b) ei = max(ei, a.ba[b]);
    for (int b = br >> 5; b <= b1; ++b) ej = max(ej, a.bb[b]);
    if (ei == OZ_E_NONE || ej == OZ_E_NONE) return 1;   // every row of one side is zero: nothing to add
    return S + 1 - max(0, eref - ei - ej) / 7;
}

template <int BN>
__device__ __forceinline__ bool oz_tile(const OzArgs &a, long long L, int *gr, int *gc, int *ar, int *br) {
    const long long per_band = (long long)OZ_GROUP * a.nt;
    const long long band = L / per_band;
    const int i0 = (int)band * OZ_GROUP;
    const int gm = min(OZ_GROUP, a.mt - i0);
    const long long w = L - band * per_band;
    const int j = (int)(w / gm), i = i0 + (int)(w % gm);
    *gr = a.r0 + i * OZ_BM;
    *gc = a.c0 + j * BN;
    *ar = a.a_off + i * OZ_BM;
    *br = a.b_off + j * BN;
    return !(a.tri && *gr + OZ_BM - 1 < *gc);
}

// 2^e as a double (0 below the normal range, where the scaled terms are
// below 2^-1000 and vanish against any entry of C that matters).
__device__ __forceinline__ double pow2i(int e) {
    if (e < -1022) return 0.0;
    if (e > 1023) e = 1024;   // infinity: only reachable from non-finite operands
    return __longlong_as_double((long long)(e + 1023) << 52);
}

template <int BK>
__device__ __forceinline__ uint64_t oz_desc(uint32_t saddr) {
    if constexpr (BK == 16) {
        uint64_t d = 0;   // SWIZZLE_32B: 8 rows x 32 bytes = 256-byte groups
        d |= (uint64_t)((saddr >> 4) & 0x3FFF);
        d |= (uint64_t)1 << 16;
        d |= (uint64_t)(256 >> 4) << 32;
        d |= (uint64_t)1 << 46;
        d |= (uint64_t)6 << 61;
        return d;
    } else {
        return smem_desc_sw64(saddr);
    }
}

template <int S, int BN, int BK>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_update(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const OzArgs args) {
    using Cfg = OzCfg<S, BN, BK>;
    constexpr int ST = Cfg::STAGES;
    constexpr int STAGE_BYTES = Cfg::STAGE_BYTES;
    constexpr int A_BYTES = Cfg::A_BYTES, B_BYTES = Cfg::B_BYTES;
    constexpr int PASSES = Cfg::PASSES, CPT = Cfg::CPT, WREG = Cfg::WREG;
    extern __shared__ uint8_t smem_raw[];
    constexpr int NSLOT = OZ_TMEM_COLS / BN;   // accumulator slots of BN columns
    __shared__ uint64_t full_bar[ST], empty_bar[ST], acc_full, slot_empty[NSLOT], drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int skip, emax_a, emax_b;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // one read for the whole CTA: a factorisation step on another stream may set it meanwhile
    if (threadIdx.x == 0) {
        skip = *(volatile const int *)&args.st->info;
        emax_a = emax_b = OZ_E_NONE;
    }
    __syncthreads();
    if (skip) return;   // an earlier step failed
    if (args.cut) {   // the launch's reference exponents E_A, E_B
        int ma = OZ_E_NONE, mb = OZ_E_NONE;
        for (int b = threadIdx.x; b < args.nba; b += OZ_THREADS) ma = max(ma, args.ra[b]);
        for (int b = threadIdx.x; b < args.nbb; b += OZ_THREADS) mb = max(mb, args.rb[b]);
        for (int o = 16; o > 0; o >>= 1) {
            ma = max(ma, __shfl_xor_sync(0xffffffffu, ma, o));
            mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
        }
        if (lane == 0) {
            atomicMax(&emax_a, ma);
            atomicMax(&emax_b, mb);
        }
        __syncthreads();
    }
    const int eref = emax_a + emax_b;
    // the level cut of this CTA's tiles (the i-th tile it visits is L = blockIdx.x + i gridDim.x),
    // computed once here so that no role waits on the exponent loads inside its tile loop
    __shared__ uint8_t lc_tab[OZ_LC_CAP];
    __shared__ __align__(16) double c_stage[OZ_EPI_WARPS * 2 * 4 * 32];   // epilogue: C columns in flight
    if (args.cut) {
        const long long mine = (ntiles_all(args) - blockIdx.x + gridDim.x - 1) / gridDim.x;
        for (int i = threadIdx.x; i < OZ_LC_CAP && i < mine; i += OZ_THREADS) {
            int gr, gc, ar, br;
            const long long L = blockIdx.x + (long long)i * gridDim.x;
            lc_tab[i] = oz_tile<BN>(args, L, &gr, &gc, &ar, &br) ? (uint8_t)max(0, oz_lcut<S, BN>(args, ar, br, eref))
                                                                 : (uint8_t)0;
        }
        __syncthreads();
    }
    auto tile_lc = [&](long long i, int ar, int br) -> int {
        if (!args.cut) return S + 1;
        return i < OZ_LC_CAP ? (int)lc_tab[i] : oz_lcut<S, BN>(args, ar, br, eref);
    };
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const long long ntiles = (long long)args.mt * args.nt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        for (int j = 0; j < NSLOT; ++j) mbar_init(&slot_empty[j], OZ_EPI_WARPS);
        mbar_init(&drain_bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    int *tword = &args.st->timeout;

    if (warp == 0) {
        if (lane == 0) {
            long long g = 0;   // chunks issued
            bool ok = true;
            for (long long L = blockIdx.x, it = 0; L < ntiles && ok; L += gridDim.x, ++it) {
                int gr, gc, ar, br;
                if (!oz_tile<BN>(args, L, &gr, &gc, &ar, &br)) continue;
                const int lc = tile_lc(it, ar, br);
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps) {
                    if (Cfg::lev_lo(ps) > lc) break;   // every level of this pass (and later ones) is cut
                    const int tm = min(Cfg::tmax(ps), lc - 1);
                    for (int kb = 0; kb < args.nk && ok; ++kb, ++g) {
                        const int s = (int)(g % ST);
                        if (g >= ST && !mbar_wait(&empty_bar[s], (uint32_t)(((g / ST) & 1) ^ 1), tword, 21)) {
                            ok = false;
                            break;
                        }
                        uint8_t *base = smem + (size_t)s * STAGE_BYTES;
                        mbar_arrive_expect_tx(&full_bar[s], (uint32_t)(tm * (A_BYTES + B_BYTES)));
                        for (int t = 0; t < tm; ++t) {
                            tma_load_3d(&mapA, &full_bar[s], base + t * A_BYTES, kb * BK, ar, t);
                            tma_load_3d(&mapB, &full_bar[s], base + S * A_BYTES + t * B_BYTES, kb * BK, br, t);
                        }
                    }
                }
            }
            if (!ok) {
                for (long long q = (g > ST ? g - ST : 0); q < g; ++q)
                    mbar_wait(&full_bar[q % ST], (uint32_t)((q / ST) & 1), tword, 22);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc_f16(1, OZ_BM, BN);
            long long g = 0;
            int use[NSLOT];   // jobs that have used each accumulator slot so far
#pragma unroll
            for (int j = 0; j < NSLOT; ++j) use[j] = 0;
            unsigned long long nmma = 0;
            bool ok = true;
            for (long long L = blockIdx.x, it = 0; L < ntiles && ok; L += gridDim.x, ++it) {
                int gr, gc, ar, br;
                if (!oz_tile<BN>(args, L, &gr, &gc, &ar, &br)) continue;
                const int lc = tile_lc(it, ar, br);
#pragma unroll
                for (int ps = 0; ps < PASSES; ++ps) {
                    if (!ok || Cfg::lev_lo(ps) > lc) break;
                    // every slot of the pass takes part in the release protocol; only levels <= lc get MMAs
                    const int llo = Cfg::lev_lo(ps), lhi = Cfg::lev_hi(ps);
                    for (int kb = 0; kb < args.nk; ++kb, ++g) {
                        const int s = (int)(g % ST);
                        if (!mbar_wait(&full_bar[s], (uint32_t)((g / ST) & 1), tword, 23)) {
                            ok = false;
                            break;
                        }
                        fence_after_sync();
                        const uint32_t a0 = smem_u32(smem + (size_t)s * STAGE_BYTES);
                        const uint64_t da0 = oz_desc<BK>(a0), db0 = oz_desc<BK>(a0 + S * A_BYTES);
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
#pragma unroll
                            for (int l = 2; l <= S + 1; ++l) {
                                if (l < llo || l > lhi) continue;
                                const int tlo = (l - S > 1) ? l - S : 1, thi = (l - 1 < S) ? l - 1 : S;
                                const int slot = l - llo;
                                if (kb == 0 && kk == 0 && use[slot] >= 1) {
                                    // the epilogue has read this slot's previous contents (per-slot release)
                                    if (!mbar_wait(&slot_empty[slot], (uint32_t)((use[slot] - 1) & 1), tword, 25)) {
                                        ok = false;
                                        break;
                                    }
                                    fence_after_sync();
                                }
                                if (l > lc) continue;
                                nmma += (unsigned long long)(thi - tlo + 1);
#pragma unroll
                                for (int t = tlo; t <= thi; ++t) {
                                    const int u = l - t;
                                    const uint32_t acc = tmem + (uint32_t)((l - llo) * BN);
                                    // start-address field += offset / 16 (no carry: smem addresses < 2^18)
                                    mma_f16(acc, da0 + (uint64_t)(((t - 1) * A_BYTES + kk * 32) >> 4),
                                            db0 + (uint64_t)(((u - 1) * B_BYTES + kk * 32) >> 4), idesc,
                                            (kb != 0 || kk != 0 || t != tlo) ? 1u : 0u);
                                }
                            }
                            if (!ok) break;
                        }
                        if (!ok) break;
                        mma_commit(&empty_bar[s]);
                    }
                    if (!ok) break;
                    mma_commit(&acc_full);
#pragma unroll
                    for (int l = 2; l <= S + 1; ++l)
                        if (l >= llo && l <= lhi) ++use[l - llo];
                }
            }
            // every MMA issued so far has completed before TMEM can be freed
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, tword, 26);
            if (args.tc_flops) atomicAdd(args.tc_flops, nmma * (unsigned long long)(2 * OZ_BM * BN * 16));
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..9; TMEM lane quarter q = warp % 4 (tile rows 32q..), column half h
        const int q = warp % 4, h = (warp - 2) / 4;
        const int row = q * 32 + lane;
        int job = 0;
        bool ok = true;
        // C entries of this thread's row, CQ columns at a time, double-buffered through shared
        // memory by cp.async: the copies for the next columns are in flight while the current
        // ones are updated, and no register waits on a load of C
        constexpr int CQ = 4;
        double *cbuf = &c_stage[(warp - 2) * 2 * CQ * 32];
        for (long long L = blockIdx.x, it = 0; L < ntiles && ok; L += gridDim.x, ++it) {
            int gr, gc, ar, br;
            if (!oz_tile<BN>(args, L, &gr, &gc, &ar, &br)) continue;
            const int lc = tile_lc(it, ar, br);
            const int grow = gr + row;
            const int er = (grow < args.m_end) ? args.ea[ar + row] : 0;
#pragma unroll
            for (int ps = 0; ps < PASSES; ++ps) {
                if (Cfg::lev_lo(ps) > lc) break;
                ok = mbar_wait(&acc_full, (uint32_t)(job & 1), tword, 24);
                ok = __all_sync(0xffffffffu, ok);   // every lane takes part in tcgen05.ld
                if (!ok) break;
                fence_after_sync();
                const int llo = Cfg::lev_lo(ps), lhi = Cfg::lev_hi(ps);
                const int w0 = ps * Cfg::WPP;
                long long acc[WREG][CPT];
#pragma unroll
                for (int l = 2; l <= S + 1; ++l) {
                    if (l < llo || l > lhi) continue;
                    const int wi = (l - 2) / OZ_LPW - w0;   // word of this level within the pass
                    const bool first = ((l - 2) % OZ_LPW) == 0;
                    const bool live = l <= lc;   // a cut level's slot holds stale values: taken as 0
#pragma unroll
                    for (int c32 = 0; c32 < CPT / 32; ++c32) {
                        float v[32];
                        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((l - llo) * BN + h * CPT + c32 * 32),
                                  v);
                        if (c32 == CPT / 32 - 1) {
                            // this warp has read the slot: the MMAs of the next job may overwrite it
                            fence_before_sync();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&slot_empty[l - llo]);
                        }
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const long long d = live ? (long long)__float2int_rn(v[j]) : 0;   // exact, below 2^24
                            acc[wi][c32 * 32 + j] = first ? d : acc[wi][c32 * 32 + j] * 128 + d;
                        }
                    }
                }
                ++job;
                if (grow < args.m_end) {
                    const bool over = args.overwrite && ps == 0;
                    auto live_col = [&](int j) {
                        const int gcol = gc + h * CPT + j;
                        return gcol < args.n_end && !(args.tri && grow < gcol);
                    };
                    auto stage = [&](int j0, int b) {
#pragma unroll
                        for (int jj = 0; jj < CQ; ++jj)
                            if (live_col(j0 + jj))
                                cp_async8(&cbuf[(b * CQ + jj) * 32 + lane],
                                          args.C + (long long)(gc + h * CPT + j0 + jj) * args.ldc + grow);
                        cp_async_commit();
                    };
                    if (!args.cut || over) {
                        // every level kept: the MMAs, not these loads, set the pace
#pragma unroll
                        for (int j = 0; j < CPT; ++j) {
                            if (!live_col(j)) continue;
                            const int e = er + args.eb[br + h * CPT + j];
                            double *pc = args.C + (long long)(gc + h * CPT + j) * args.ldc + grow;
                            double c = over ? 0.0 : *pc;
#pragma unroll
                            for (int wi = WREG - 1; wi >= 0; --wi) {
                                if (w0 + wi >= Cfg::NWT || 2 + OZ_LPW * (w0 + wi) > lc) continue;
                                c = fma(-(double)acc[wi][j], pow2i(e + 2 - 7 * Cfg::word_hi(w0 + wi)), c);
                            }
                            *pc = c;
                        }
                        continue;
                    }
                    stage(0, 0);
#pragma unroll
                    for (int j0 = 0; j0 < CPT; j0 += CQ) {
                        const int b = (j0 / CQ) & 1;
                        if (j0 + CQ < CPT) {
                            stage(j0 + CQ, b ^ 1);
                            cp_async_wait<1>();
                        } else {
                            cp_async_wait<0>();
                        }
#pragma unroll
                        for (int jj = 0; jj < CQ; ++jj) {
                            const int j = j0 + jj;
                            if (!live_col(j)) continue;
                            const int e = er + args.eb[br + h * CPT + j];
                            double c = cbuf[(b * CQ + jj) * 32 + lane];
#pragma unroll
                            for (int wi = WREG - 1; wi >= 0; --wi) {
                                if (w0 + wi >= Cfg::NWT || 2 + OZ_LPW * (w0 + wi) > lc) continue;
                                c = fma(-(double)acc[wi][j], pow2i(e + 2 - 7 * Cfg::word_hi(w0 + wi)), c);
                            }
                            args.C[(long long)(gc + h * CPT + j) * args.ldc + grow] = c;
                        }
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
    }
}

// Digit slices of rows [0, R) of the column-major FP64 panel P (ld), columns
// [k0, k0 + kc) for the K chunk blockIdx.y (kc = kchunk, the last one
// shorter): slice t of row r at out[t * slice_stride + r * Kp + k] (BF16,
// zero for k beyond the panel), the row exponent at exps[chunk * exp_stride + r].
// Per 32-row block b the largest exponent of its non-zero rows goes to
// bexps[2 chunk bstride + b], and that of its non-zero rows below ref_rows to
// bexps[(2 chunk + 1) bstride + b] (OZ_E_NONE where there is none).
// One CTA per 32 rows: a column sweep for the row maxima, then 32 x 32
// tiles through shared memory so that each slice row is written along K, four
// digits (8 bytes) per store.  Everything runs on the integer pipes: the
// maxima compare the magnitudes' bit patterns (ordered like the values), and
// X = rint(x 2^(7S - 1 - e)) is the 53-bit significand shifted by the
// difference of exponents with round-to-nearest-even, the same integer the
// FP64 product and conversion would give.
__device__ __forceinline__ long long oz_scaled_int(unsigned long long b, int k) {
    // rint(x 2^k) for the double with bits b (|x 2^k| < 2^62)
    const int E = (int)((b >> 52) & 0x7FF);
    if (E == 0) return 0;   // zero or subnormal: below 2^-1022, far below 1/2 after any scaling used here
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = 1075 - E - k;   // x 2^k = m 2^-sh
    unsigned long long q;
    if (sh <= 0) {
        q = m << (-sh);
    } else if (sh >= 64) {
        q = 0;
    } else {
        q = m >> sh;
        const unsigned long long rem = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (q & 1))) ++q;
    }
    return (b >> 63) ? -(long long)q : (long long)q;
}

// BF16 bits of a small integer d, |d| <= 64 (exact: at most 7 significant bits).
__device__ __forceinline__ unsigned int oz_bf16_bits(int d) {
    if (d == 0) return 0u;
    const unsigned int u = (unsigned int)(d < 0 ? -d : d);
    const int p = 31 - __clz(u);   // 0 .. 6
    return (d < 0 ? 0x8000u : 0u) | ((unsigned int)(127 + p) << 7) | ((u << (7 - p)) & 0x7Fu);
}

__global__ void __launch_bounds__(256) k_oz_slice(const double *P, long long ld, int R, int K, int kchunk, int S,
                                                  __nv_bfloat16 *out, long long slice_stride, int Kp, int *exps,
                                                  long long exp_stride, int *bexps, long long bstride, int ref_rows,
                                                  const DevStatus *st) {
    __shared__ unsigned long long tile[32][33];
    __shared__ unsigned long long red[8][32];
    __shared__ int ex[32];
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *(volatile const int *)&st->info;
    __syncthreads();
    if (skip) return;
    const int r0 = blockIdx.x * 32;
    const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);
    const int kpad_end = min(Kp, kbeg + (kchunk + OZ_KALIGN - 1) / OZ_KALIGN * OZ_KALIGN);
    const int rr = threadIdx.x % 32, g = threadIdx.x / 32;
    const unsigned long long *Pb = reinterpret_cast<const unsigned long long *>(P);
    constexpr unsigned long long MAG = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long mx = 0;
    if (r0 + rr < R)
        for (int k = kbeg + g; k < kend; k += 8) mx = max(mx, Pb[(long long)k * ld + r0 + rr] & MAG);
    red[g][rr] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned long long m = red[0][rr];
        for (int q = 1; q < 8; ++q) m = max(m, red[q][rr]);
        // max |x| = f 2^e with f in [1/2, 1): |x| < 2^e on the row (e = biased exponent - 1022)
        int e = 0;
        if (m > 0) e = max((int)(m >> 52) - 1022, -960);
        ex[rr] = e;
        if (r0 + rr < R) exps[(long long)blockIdx.y * exp_stride + r0 + rr] = e;
        const bool live = r0 + rr < R && m > 0;
        int eall = live ? e : OZ_E_NONE, eref = (live && r0 + rr < ref_rows) ? e : OZ_E_NONE;
        for (int o = 16; o > 0; o >>= 1) {
            eall = max(eall, __shfl_xor_sync(0xffffffffu, eall, o));
            eref = max(eref, __shfl_xor_sync(0xffffffffu, eref, o));
        }
        if (rr == 0) {
            bexps[2LL * blockIdx.y * bstride + blockIdx.x] = eall;
            bexps[(2LL * blockIdx.y + 1) * bstride + blockIdx.x] = eref;
        }
    }
    __syncthreads();
    // this thread's row and four consecutive columns of each 32 x 32 tile
    const int r = threadIdx.x / 8, cq = (threadIdx.x % 8) * 4;
    const int kshift = 7 * S - 1 - ex[r];
    for (int c0 = kbeg; c0 < kpad_end; c0 += 32) {
        for (int t = threadIdx.x; t < 32 * 32; t += 256) {
            const int c = t / 32, rw = t % 32;
            tile[c][rw] = (r0 + rw < R && c0 + c < kend) ? Pb[(long long)(c0 + c) * ld + r0 + rw] : 0ull;
        }
        __syncthreads();
        if (r0 + r < R) {
            long long X[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) X[i] = oz_scaled_int(tile[cq + i][r], kshift);
            unsigned int *o = reinterpret_cast<unsigned int *>(out + (long long)(r0 + r) * Kp + c0 + cq);
            for (int sl = S - 1; sl >= 1; --sl) {
                int d[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    d[i] = (int)(((X[i] + 64) & 127) - 64);   // balanced digit in [-64, 63]
                    X[i] = (X[i] - d[i]) >> 7;                 // exact: X - d is a multiple of 128
                }
                uint2 v;
                v.x = oz_bf16_bits(d[0]) | (oz_bf16_bits(d[1]) << 16);
                v.y = oz_bf16_bits(d[2]) | (oz_bf16_bits(d[3]) << 16);
                *reinterpret_cast<uint2 *>(o + (long long)sl * slice_stride / 2) = v;
            }
            uint2 v;   // leading digits, |X| <= 64
            v.x = oz_bf16_bits((int)X[0]) | (oz_bf16_bits((int)X[1]) << 16);
            v.y = oz_bf16_bits((int)X[2]) | (oz_bf16_bits((int)X[3]) << 16);
            *reinterpret_cast<uint2 *>(o) = v;
        }
        __syncthreads();
    }
}

template <int S, int BN, int BK>
cudaError_t launch_oz_kernel(const CUtensorMap &ma, const CUtensorMap &mb, const OzArgs &a, int grid,
                             cudaStream_t s) {
    using Cfg = OzCfg<S, BN, BK>;
    static_assert(Cfg::STAGES >= 2, "shared memory holds fewer than two chunks");
    cudaError_t e = cudaFuncSetAttribute(k_oz_update<S, BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)Cfg::SMEM);
    if (e != cudaSuccess) return e;
    k_oz_update<S, BN, BK><<<grid, OZ_THREADS, Cfg::SMEM, s>>>(ma, mb, a);
    return cudaGetLastError();
}

// Kernel shape per slice count (measured on GB300 with C 8192 x 8192, K = 512):
// with 6 or more slices the 128-column tile in passes of four levels keeps the
// tensor pipe busiest (8 slices: 1,290 against 1,063 TFLOP/s of BF16 work for
// the single-pass 64-column tile); with fewer the passes get short and the
// 64-column single pass wins (5 slices: 902 against 655).  With the level cut
// at 5 slices the 128-column tile wins again: the second pass (the last
// level) is cut on most tiles, so the epilogue, which sets the pace of cut
// tiles, works on half as many C entries per MMA (N = 100,000: 4.3 against
// 5.8 s per factorisation).
struct OzShape {
    int bn, bk;
};

OzShape oz_shape(int S, int cut) { return (S >= 6 || (S == 5 && cut)) ? OzShape{128, 16} : OzShape{64, 32}; }

template <int S>
cudaError_t launch_oz_shape(OzShape sh, const CUtensorMap &ma, const CUtensorMap &mb, const OzArgs &a, int grid,
                            cudaStream_t s) {
    if constexpr (S >= 6) {
        return launch_oz_kernel<S, 128, 16>(ma, mb, a, grid, s);
    } else if constexpr (S == 5) {
        if (sh.bn == 128) return launch_oz_kernel<S, 128, 16>(ma, mb, a, grid, s);
        return launch_oz_kernel<S, 64, 32>(ma, mb, a, grid, s);
    } else {
        return launch_oz_kernel<S, 64, 32>(ma, mb, a, grid, s);
    }
}

// 3-D tensor map over the slices: (k, row, slice), box bk x rows_box x 1,
// swizzle = the K chunk's row width (32 or 64 bytes).
cudaError_t slice_map(CUtensorMap *map, const OzSlices &sl, int chunk, int rows_box, int bk) {
    tc::EncodeTiledFn enc = tc::encode_fn();
    if (!enc) return cudaErrorNotSupported;
    void *base = (__nv_bfloat16 *)sl.d + (size_t)chunk * sl.kchunk;   // 64-byte aligned: kchunk is a multiple of 32
    cuuint64_t dims[3] = {(cuuint64_t)std::min(sl.kchunk, sl.Kp - chunk * sl.kchunk), (cuuint64_t)sl.valid,
                          (cuuint64_t)sl.S};
    cuuint64_t strides[2] = {(cuuint64_t)sl.Kp * 2, (cuuint64_t)sl.slice_stride * 2};
    cuuint32_t box[3] = {(cuuint32_t)bk, (cuuint32_t)rows_box, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int oz_kmax(int S) { return (4096 / S) / OZ_KALIGN * OZ_KALIGN; }

size_t oz_slices_bytes(long long rows, int K, int S) {
    const long long Kp = (K + OZ_KALIGN - 1) / OZ_KALIGN * OZ_KALIGN;
    const int nchunk = (K + oz_kmax(S) - 1) / oz_kmax(S);
    return (size_t)S * (size_t)rows * (size_t)Kp * 2 + sizeof(int) * (size_t)rows * nchunk +
           sizeof(int) * 2 * (size_t)((rows + 31) / 32) * nchunk + 768;
}

OzSlices oz_slices_carve(void *ws, long long rows, int K, int S) {
    OzSlices o;
    o.S = S;
    o.rows = rows;
    o.K = K;
    o.kchunk = oz_kmax(S);
    o.Kp = (K + OZ_KALIGN - 1) / OZ_KALIGN * OZ_KALIGN;
    o.nchunk = (K + o.kchunk - 1) / o.kchunk;
    o.valid = rows;
    o.slice_stride = (long long)rows * o.Kp;
    o.d = ws;
    uintptr_t e = (uintptr_t)ws + (size_t)S * o.slice_stride * 2;
    o.e = (int *)((e + 255) & ~(uintptr_t)255);
    o.bstride = (rows + 31) / 32;
    o.be = (int *)(((uintptr_t)(o.e + rows * o.nchunk) + 255) & ~(uintptr_t)255);
    o.ref_rows = -1;
    return o;
}

cudaError_t oz_slice(const double *P, long long ld, int R, const OzSlices &o, const DevStatus *st, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    if (R > o.rows || R > o.valid) return cudaErrorInvalidValue;
    dim3 grid((R + 31) / 32, o.nchunk);
    KScope ks(GEO_K_AUX, s, 0.0, (double)R * o.K * (16.0 + 2.0 * o.S));
    k_oz_slice<<<grid, 256, 0, s>>>(P, ld, R, o.K, o.kchunk, o.S, (__nv_bfloat16 *)o.d, o.slice_stride, o.Kp, o.e,
                                    o.rows, o.be, o.bstride, o.ref_rows < 0 ? R : (int)std::min<long long>(o.ref_rows, R),
                                    st);
    return cudaGetLastError();
}

cudaError_t oz_update(const OzSlices &A, const OzSlices &B, double *C, long long ldc, int r0, int c0, int rows,
                      int cols, int m_end, int n_end, int a_off, int b_off, int tri, int grid_cap, DevStatus *st,
                      cudaStream_t s, int overwrite, int cut) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (A.S != B.S || A.K != B.K || A.S < 3 || A.S > 8) return cudaErrorInvalidValue;
    if (cut && overwrite) return cudaErrorInvalidValue;   // a skipped tile would leave C unwritten
    const int S = A.S;
    OzArgs a;
    a.C = C;
    a.ldc = ldc;
    a.r0 = r0;
    a.c0 = c0;
    a.m_end = m_end;
    a.n_end = n_end;
    const OzShape sh = oz_shape(S, cut);
    a.mt = (rows + OZ_BM - 1) / OZ_BM;
    a.nt = (cols + sh.bn - 1) / sh.bn;
    a.tri = tri;
    a.a_off = a_off;
    a.overwrite = 0;
    a.b_off = b_off;
    a.st = st;
    a.cut = cut ? 1 : 0;
    a.nba = (int)((A.valid + 31) / 32);
    a.nbb = (int)((B.valid + 31) / 32);
    a.tc_flops = t_prof ? t_prof->d_tc_flops : nullptr;
    const long long ntiles = (long long)a.mt * a.nt;
    const int grid = (int)std::min<long long>(ntiles, std::max(1, std::min(grid_cap, tc::num_sms())));
    // algorithmic work: 2 K flops per output written (lower triangle when tri)
    const double rr = rows, cc = cols;
    const double outs = tri ? std::max(0.0, rr * cc - cc * (cc - 1.0) / 2.0) : rr * cc;
    for (int ch = 0; ch < A.nchunk; ++ch) {
        const int kc = std::min(A.kchunk, A.K - ch * A.kchunk);
        a.nk = (kc + sh.bk - 1) / sh.bk;
        a.ea = A.e + (long long)ch * A.rows;
        a.eb = B.e + (long long)ch * B.rows;
        a.ba = A.be + 2LL * ch * A.bstride;
        a.ra = a.ba + A.bstride;
        a.bb = B.be + 2LL * ch * B.bstride;
        a.rb = a.bb + B.bstride;
        CUtensorMap ma, mb;
        cudaError_t e;
        if ((e = slice_map(&ma, A, ch, OZ_BM, sh.bk)) != cudaSuccess ||
            (e = slice_map(&mb, B, ch, sh.bn, sh.bk)) != cudaSuccess)
            return e;
        a.overwrite = (overwrite && ch == 0) ? 1 : 0;   // later K chunks accumulate onto the first
        KScope ks(GEO_K_TCGEMM, s, 2.0 * kc * outs, 16.0 * outs + 2.0 * S * kc * (rr + cc));
        switch (S) {
            case 3: e = launch_oz_shape<3>(sh, ma, mb, a, grid, s); break;
            case 4: e = launch_oz_shape<4>(sh, ma, mb, a, grid, s); break;
            case 5: e = launch_oz_shape<5>(sh, ma, mb, a, grid, s); break;
            case 6: e = launch_oz_shape<6>(sh, ma, mb, a, grid, s); break;
            case 7: e = launch_oz_shape<7>(sh, ma, mb, a, grid, s); break;
            default: e = launch_oz_shape<8>(sh, ma, mb, a, grid, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

namespace {

// W = -L^-1 for the lower-triangular jb x jb tile L (column-major, ld),
// written column-major with leading dimension ldw (zeros above the diagonal).
// Column-oriented forward substitution L w = e_c for the TRTRI_COLS columns of
// a CTA: at step k the owner of row k divides by L_kk and publishes w_k, every
// thread then updates its rows below with column k of L (read along the
// column, coalesced).  The broadcast buffer is double-buffered, so one barrier
// per step suffices; the reciprocals of the diagonal are taken up front, off
// the chain of steps.  Four columns per CTA: the FP64 work of a step (two
// FMAs per clock per SM) is split over jb / 4 CTAs.
constexpr int TRTRI_COLS = 4, TRTRI_THREADS = 256, TRTRI_RPT = 4;   // rows per thread: jb <= 1024

__global__ void __launch_bounds__(TRTRI_THREADS) k_trtri_neg(const double *__restrict__ L, long long ld, int jb,
                                                          double *W, long long ldw, const DevStatus *st) {
    __shared__ double wk[2][TRTRI_COLS];
    __shared__ double dinv[TRTRI_THREADS * TRTRI_RPT];
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *(volatile const int *)&st->info;
    __syncthreads();
    if (skip) return;
    for (int r = threadIdx.x; r < jb; r += TRTRI_THREADS) dinv[r] = 1.0 / L[(long long)r * ld + r];
    __syncthreads();
    const int c0 = blockIdx.x * TRTRI_COLS;
    const int ncol = min(TRTRI_COLS, jb - c0);
    double w[TRTRI_RPT][TRTRI_COLS];
#pragma unroll
    for (int q = 0; q < TRTRI_RPT; ++q) {
        const int r = threadIdx.x + q * TRTRI_THREADS;
#pragma unroll
        for (int c = 0; c < TRTRI_COLS; ++c) w[q][c] = (r == c0 + c) ? 1.0 : 0.0;
    }
    // column k of L for this thread's rows (and the diagonal entry for the owner of row k),
    // loaded one step ahead so that the load latency is off the chain of barriers
    double lcol[TRTRI_RPT];
    auto load_col = [&](int k, double *dst) {
#pragma unroll
        for (int q = 0; q < TRTRI_RPT; ++q) {
            const int r = threadIdx.x + q * TRTRI_THREADS;
            dst[q] = (k < jb && r >= k && r < jb) ? L[(long long)k * ld + r] : 0.0;
        }
    };
    load_col(c0, lcol);
    for (int k = c0; k < jb; ++k) {
        double lnext[TRTRI_RPT];
        load_col(k + 1, lnext);
        const int owner_q = k / TRTRI_THREADS, owner_t = k % TRTRI_THREADS;
        if (threadIdx.x == owner_t) {
            const double inv = dinv[k];
#pragma unroll
            for (int q = 0; q < TRTRI_RPT; ++q)
                if (q == owner_q) {
#pragma unroll
                    for (int c = 0; c < TRTRI_COLS; ++c) {
                        w[q][c] *= inv;
                        wk[k & 1][c] = w[q][c];
                    }
                }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < TRTRI_RPT; ++q) {
            const int r = threadIdx.x + q * TRTRI_THREADS;
            if (r > k && r < jb) {
#pragma unroll
                for (int c = 0; c < TRTRI_COLS; ++c) w[q][c] = fma(-lcol[q], wk[k & 1][c], w[q][c]);
            }
        }
#pragma unroll
        for (int q = 0; q < TRTRI_RPT; ++q) lcol[q] = lnext[q];
    }
#pragma unroll
    for (int q = 0; q < TRTRI_RPT; ++q) {
        const int r = threadIdx.x + q * TRTRI_THREADS;
        if (r >= jb) continue;
#pragma unroll
        for (int c = 0; c < TRTRI_COLS; ++c)
            if (c < ncol) W[(long long)(c0 + c) * ldw + r] = (r >= c0 + c) ? -w[q][c] : 0.0;
    }
}

cudaError_t launch_trtri_neg(const double *L, long long ld, int jb, double *W, long long ldw, const DevStatus *st,
                             cudaStream_t s) {
    if (jb > TRTRI_THREADS * TRTRI_RPT) return cudaErrorInvalidValue;
    KScope ks(GEO_K_TRSM, s, (double)jb * jb * jb / 3.0, 16.0 * jb * jb);
    k_trtri_neg<<<(jb + TRTRI_COLS - 1) / TRTRI_COLS, TRTRI_THREADS, 0, s>>>(L, ld, jb, W, ldw, st);
    return cudaGetLastError();
}

}  // namespace

constexpr int OZ_TILE_IB = 64;   // inner block of the diagonal tiles (the rank of their updates)

size_t oz_chol_workspace_bytes(int nrows, int nb, int S) {
    return oz_slices_bytes((long long)nrows + 128, nb, S) + oz_slices_bytes(nb, nb, S) + sizeof(double) * (size_t)nb * nb +
           oz_slices_bytes(nb, OZ_TILE_IB, S) + 1280;
}

namespace {
// The rank-64 updates inside a diagonal tile as emulated products: the rows
// below the inner block (their columns kA .. kA + k) as digit slices, then the
// lower triangle of the rest of the tile.  Runs on the side stream with at most
// `sms` CTAs, beside the trailing update.
struct TileUpdate {
    OzSlices sl;
    int sms;
};

cudaError_t tile_update(const PanelUpdate *u, double *A, long long ld, int rC, int cC, int m, int n, int kA, int k,
                        DevStatus *st, cudaStream_t s) {
    const TileUpdate &t = *(const TileUpdate *)u->ctx;
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    if (rC != cC || k > t.sl.K || m > t.sl.rows) return cudaErrorInvalidValue;
    OzSlices p = t.sl;
    p.K = k;
    p.nchunk = (k + p.kchunk - 1) / p.kchunk;
    p.valid = m;
    cudaError_t e = oz_slice(A + (long long)kA * ld + rC, ld, m, p, st, s);
    if (e != cudaSuccess) return e;
    return oz_update(p, p, A, ld, rC, cC, m, n, rC + m, cC + n, 0, 0, 1, t.sms, st, s, 0, 0);
}
}  // namespace

// Right-looking over panels of width nb with a lookahead of one (as the mixed
// form).  Step j slices its solved panel (the rows below the diagonal tile,
// right-hand-side rows included) and updates the next panel's tile column
// first; on a high-priority second stream the next diagonal tile is factored
// (native FP64 POTRF) and inverted, W = -L_kk^-1, while the rest of the
// trailing update runs (its persistent launch leaves SIDE_SMS SMs free).
// After the join the rows below the new diagonal tile are solved as one
// emulated product, L_ik = A_ik L_kk^-T = -(A_ik W'), written over A_ik.
// Every trailing update and panel solve is emulated; POTRF of the diagonal
// tiles and their inversion are native FP64, and so is the last panel.
cudaError_t chol_oz_factor(double *A, long long ld, int N, int nrows, int nb, int S, int cut, void *ws,
                           size_t ws_bytes, DevStatus *st, cudaStream_t s) {
    constexpr int SIDE_SMS = 8;
    if (nb < 64 || nb % 64 != 0 || nb > TRTRI_THREADS * TRTRI_RPT || S < 3 || S > 8) return cudaErrorInvalidValue;
    if (ws_bytes < oz_chol_workspace_bytes(nrows, nb, S)) return cudaErrorInvalidValue;
    const OzSlices sl = oz_slices_carve(ws, (long long)nrows + 128, nb, S);
    uintptr_t wp = ((uintptr_t)ws + oz_slices_bytes((long long)nrows + 128, nb, S) + 255) & ~(uintptr_t)255;
    const OzSlices slw0 = oz_slices_carve((void *)wp, nb, nb, S);
    wp = (wp + oz_slices_bytes(nb, nb, S) + 255) & ~(uintptr_t)255;
    double *W = (double *)wp;   // nb x nb, ld nb
    wp = (wp + sizeof(double) * (size_t)nb * nb + 255) & ~(uintptr_t)255;
    TileUpdate tu{oz_slices_carve((void *)wp, nb, OZ_TILE_IB, S), SIDE_SMS};
    const PanelUpdate tile_upd{tile_update, &tu};
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaStream_t s2 = nullptr;
    cudaEvent_t e_upd = nullptr, e_pan = nullptr;
    cudaError_t e;
    if ((e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio_hi)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&e_upd, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&e_pan, cudaEventDisableTiming)) != cudaSuccess) {
        cudaStreamDestroy(s2);
        if (e_upd) cudaEventDestroy(e_upd);
        return e;
    }
    const int all = tc::num_sms();
    // rows [x0, x1) of panel [t0, t0 + jb) <- A L^-T with W = -L^-1 already in place
    auto panel_solve = [&](int t0, int jb, int x0, int x1, cudaStream_t st_) -> cudaError_t {
        if (x0 >= x1) return cudaSuccess;
        OzSlices p = sl, q = slw0;
        p.K = q.K = jb;
        p.nchunk = q.nchunk = (jb + p.kchunk - 1) / p.kchunk;
        p.valid = x1 - x0;
        q.valid = jb;
        cudaError_t r;
        if ((r = oz_slice(A + (long long)t0 * ld + x0, ld, x1 - x0, p, st, st_)) != cudaSuccess ||
            (r = oz_slice(W, nb, jb, q, st, st_)) != cudaSuccess)
            return r;
        return oz_update(p, q, A, ld, x0, t0, x1 - x0, jb, x1, t0 + jb, 0, 0, 0, all, st, st_, 1, 0);
    };
    // native FP64 factorisation of the diagonal tile [t0, t0 + jb) and its inverse
    auto diag = [&](int t0, int jb, cudaStream_t st_) -> cudaError_t {
        cudaError_t r = chol64_panel(A, ld, t0, jb, t0 + jb, t0 + jb, st, st_, true, &tile_upd);
        if (r != cudaSuccess) return r;
        return launch_trtri_neg(A + (long long)t0 * ld + t0, ld, jb, W, nb, st, st_);
    };
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        const int jb0 = std::min(nb, N);
        if (jb0 == N) return chol64_panel(A, ld, 0, N, N, nrows, st, s);   // one tile: native
        if ((r = diag(0, jb0, s)) != cudaSuccess || (r = panel_solve(0, jb0, jb0, nrows, s)) != cudaSuccess)
            return r;
        for (int j0 = 0;;) {
            const int jb = std::min(nb, N - j0);
            const int t0 = j0 + jb;
            if (t0 >= N) break;
            // the solved panel's rows below the diagonal tile as digit slices
            OzSlices p = sl;
            p.K = jb;
            p.nchunk = (jb + p.kchunk - 1) / p.kchunk;
            p.valid = nrows - t0;
            p.ref_rows = N - t0;   // the reference scale is the matrix's, not the right-hand side rows'
            if ((r = oz_slice(A + (long long)j0 * ld + t0, ld, nrows - t0, p, st, s)) != cudaSuccess) return r;
            const int n1 = std::min(N, t0 + nb);
            // the next panel's tile column: rows [t0, nrows), cols [t0, n1)
            if ((r = oz_update(p, p, A, ld, t0, t0, nrows - t0, n1 - t0, nrows, n1, 0, 0, 1, all, st, s, 0, cut)) !=
                cudaSuccess)
                return r;
            if (n1 >= N) {
                r = chol64_panel(A, ld, t0, N - t0, N, nrows, st, s);   // last panel: diagonal tile + RHS rows
                if (r != cudaSuccess) return r;
                j0 = t0;
                continue;
            }
            if ((r = cudaEventRecord(e_upd, s)) != cudaSuccess) return r;
            if ((r = cudaStreamWaitEvent(s2, e_upd, 0)) != cudaSuccess) return r;
            if ((r = diag(t0, n1 - t0, s2)) != cudaSuccess) return r;
            if ((r = cudaEventRecord(e_pan, s2)) != cudaSuccess) return r;
            // the rest of the trailing update meanwhile: rows [n1, nrows), cols [n1, N)
            if ((r = oz_update(p, p, A, ld, n1, n1, nrows - n1, N - n1, nrows, N, n1 - t0, n1 - t0, 1,
                               all - SIDE_SMS, st, s, 0, cut)) != cudaSuccess)
                return r;
            if ((r = cudaStreamWaitEvent(s, e_pan, 0)) != cudaSuccess) return r;
            if ((r = panel_solve(t0, n1 - t0, n1, nrows, s)) != cudaSuccess) return r;
            j0 = t0;
        }
        return cudaSuccess;
    };
    e = run();
    if (e != cudaSuccess) cudaStreamSynchronize(s2);
    cudaEventDestroy(e_upd);
    cudaEventDestroy(e_pan);
    cudaStreamDestroy(s2);
    return e;
}

// C (m x n) -= A (m x k) B (n x k)' for column-major FP64 operands, through
// the digit slices of A's rows and B's rows (workspace ws of
// oz_gemm_workspace_bytes).
size_t oz_gemm_workspace_bytes(int m, int n, int k, int S) {
    return oz_slices_bytes(m, k, S) + oz_slices_bytes(n, k, S) + 256;
}

cudaError_t oz_gemm(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb, double *C,
                    long long ldc, int S, void *ws, DevStatus *st, cudaStream_t s) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    const OzSlices sa = oz_slices_carve(ws, m, k, S);
    uintptr_t wb = (uintptr_t)ws + oz_slices_bytes(m, k, S);
    wb = (wb + 255) & ~(uintptr_t)255;
    const OzSlices sb = oz_slices_carve((void *)wb, n, k, S);
    cudaError_t e;
    if ((e = oz_slice(A, lda, m, sa, st, s)) != cudaSuccess || (e = oz_slice(B, ldb, n, sb, st, s)) != cudaSuccess)
        return e;
    return oz_update(sa, sb, C, ldc, 0, 0, m, n, m, n, 0, 0, 0, tc::num_sms(), st, s, 0, 0);
}
