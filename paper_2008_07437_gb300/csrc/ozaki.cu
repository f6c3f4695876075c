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
//   recombine   the epilogue converts each level to an integer and folds the
//               levels 2..5 and 6..S+1 into two 64-bit integers (exact), then
//               applies C -= 2^(e_r + e_c) (H 2^(2 - 7 h) + L 2^(2 - 7(S+1)))
//               with two FP64 FMAs.
//
// The kernel is persistent (one CTA per SM) over 128 x 64 output tiles:
//   warp 0, one lane: TMA producer, ring of K chunks of 32 (64-byte rows,
//     64-byte swizzle), each chunk holding the S digit slices of the A rows
//     (128 x 32 BF16 each) and of the B rows (64 x 32 each);
//   warp 1: allocates the 512 TMEM columns (S <= 8 accumulators of 64
//     columns), one lane issues tcgen05.mma kind::f16 (M 128, N 64, K 16)
//     level by level and commits chunks back to the producer;
//   warps 2-9: epilogue; tcgen05.ld of each level, fold into registers,
//     release TMEM (the next tile's MMAs start), then the FP64
//     read-modify-write of C.
// Every mbarrier wait is bounded; on expiry the thread records a code in the
// status word, the CTA drains what it has in flight, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "geo_internal.cuh"
#include "tcgen05_ptx.cuh"

namespace {

using namespace tc;

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 32;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_A_BYTES = OZ_BM * OZ_BK * 2;
constexpr int OZ_B_BYTES = OZ_BN * OZ_BK * 2;
constexpr int OZ_SMEM_CAP = 225 * 1024;
constexpr int OZ_GROUP = 8;   // row blocks swept together (operand reuse in L2)

template <int S>
struct OzCfg {
    static constexpr int STAGE_BYTES = S * (OZ_A_BYTES + OZ_B_BYTES);
    static constexpr int STAGES = (OZ_SMEM_CAP / STAGE_BYTES) < 4 ? (OZ_SMEM_CAP / STAGE_BYTES) : 4;
    static constexpr size_t SMEM = (size_t)STAGES * STAGE_BYTES + 1024;
    static constexpr int HEND = (S + 1) < 5 ? (S + 1) : 5;   // last level folded into the high word
};

struct OzArgs {
    double *C;
    long long ldc;
    int r0, c0;          // global row / col of the region's first output
    int m_end, n_end;    // outputs with global row >= m_end or col >= n_end are not written
    int mt, nt;          // 128-row x 64-col tiles of the region
    int tri;             // write only global row >= global col; skip tiles entirely above the diagonal
    int a_off, b_off;    // slice row of the region's first row (A) / first column (B)
    int nk;              // K chunks of 32
    const int *ea, *eb;  // per-row exponents of the A / B slices
    DevStatus *st;
};

__device__ __forceinline__ bool oz_tile(const OzArgs &a, long long L, int *gr, int *gc, int *ar, int *br) {
    const long long per_band = (long long)OZ_GROUP * a.nt;
    const long long band = L / per_band;
    const int i0 = (int)band * OZ_GROUP;
    const int gm = min(OZ_GROUP, a.mt - i0);
    const long long w = L - band * per_band;
    const int j = (int)(w / gm), i = i0 + (int)(w % gm);
    *gr = a.r0 + i * OZ_BM;
    *gc = a.c0 + j * OZ_BN;
    *ar = a.a_off + i * OZ_BM;
    *br = a.b_off + j * OZ_BN;
    return !(a.tri && *gr + OZ_BM - 1 < *gc);
}

// 2^e as a double (0 below the normal range, where the scaled terms are
// below 2^-1000 and vanish against any entry of C that matters).
__device__ __forceinline__ double pow2i(int e) {
    if (e < -1022) return 0.0;
    if (e > 1023) e = 1024;   // infinity: only reachable from non-finite operands
    return __longlong_as_double((long long)(e + 1023) << 52);
}

template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1)
    k_oz_update(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                const OzArgs args) {
    constexpr int ST = OzCfg<S>::STAGES;
    constexpr int STAGE_BYTES = OzCfg<S>::STAGE_BYTES;
    constexpr int HEND = OzCfg<S>::HEND;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[ST], empty_bar[ST], acc_full, acc_empty, drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int skip;

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    // one read for the whole CTA: a factorisation step on another stream may set it meanwhile
    if (threadIdx.x == 0) skip = *(volatile const int *)&args.st->info;
    __syncthreads();
    if (skip) return;   // an earlier step failed
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const long long ntiles = (long long)args.mt * args.nt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < ST; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&acc_full, 1);
        mbar_init(&acc_empty, OZ_EPI_WARPS);
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
            for (long long L = blockIdx.x; L < ntiles && ok; L += gridDim.x) {
                int gr, gc, ar, br;
                if (!oz_tile(args, L, &gr, &gc, &ar, &br)) continue;
                for (int kb = 0; kb < args.nk; ++kb, ++g) {
                    const int s = (int)(g % ST);
                    if (g >= ST && !mbar_wait(&empty_bar[s], (uint32_t)(((g / ST) & 1) ^ 1), tword, 21)) {
                        ok = false;
                        break;
                    }
                    uint8_t *base = smem + (size_t)s * STAGE_BYTES;
                    mbar_arrive_expect_tx(&full_bar[s], STAGE_BYTES);
#pragma unroll
                    for (int t = 0; t < S; ++t) {
                        tma_load_3d(&mapA, &full_bar[s], base + t * OZ_A_BYTES, kb * OZ_BK, ar, t);
                        tma_load_3d(&mapB, &full_bar[s], base + S * OZ_A_BYTES + t * OZ_B_BYTES, kb * OZ_BK, br, t);
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
            const uint32_t idesc = instr_desc_f16(1, OZ_BM, OZ_BN);
            long long g = 0;
            int lt = 0;   // tiles of this CTA
            bool ok = true;
            for (long long L = blockIdx.x; L < ntiles && ok; L += gridDim.x) {
                int gr, gc, ar, br;
                if (!oz_tile(args, L, &gr, &gc, &ar, &br)) continue;
                if (lt >= 1 && !mbar_wait(&acc_empty, (uint32_t)((lt - 1) & 1), tword, 25)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                for (int kb = 0; kb < args.nk; ++kb, ++g) {
                    const int s = (int)(g % ST);
                    if (!mbar_wait(&full_bar[s], (uint32_t)((g / ST) & 1), tword, 23)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t a0 = smem_u32(smem + (size_t)s * STAGE_BYTES);
                    const uint32_t b0 = a0 + S * OZ_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
                        for (int l = 2; l <= S + 1; ++l) {
                            const int tlo = (l - S > 1) ? l - S : 1, thi = (l - 1 < S) ? l - 1 : S;
#pragma unroll
                            for (int t = tlo; t <= thi; ++t) {
                                const int u = l - t;
                                const uint32_t acc = tmem + (uint32_t)((l - 2) * OZ_BN);
                                mma_f16(acc, smem_desc_sw64(a0 + (t - 1) * OZ_A_BYTES + kk * 32),
                                        smem_desc_sw64(b0 + (u - 1) * OZ_B_BYTES + kk * 32), idesc,
                                        (kb != 0 || kk != 0 || t != tlo) ? 1u : 0u);
                            }
                        }
                    }
                    mma_commit(&empty_bar[s]);
                }
                if (!ok) break;
                mma_commit(&acc_full);
                ++lt;
            }
            // every MMA issued so far has completed before TMEM can be freed
            mma_commit(&drain_bar);
            mbar_wait(&drain_bar, 0, tword, 26);
        }
        __syncwarp();
    } else {
        // epilogue: warps 2..9; TMEM lane quarter q = warp % 4 (tile rows 32q..), column half h
        const int q = warp % 4, h = (warp - 2) / 4;
        const int row = q * 32 + lane;
        int lt = 0;
        for (long long L = blockIdx.x; L < ntiles; L += gridDim.x) {
            int gr, gc, ar, br;
            if (!oz_tile(args, L, &gr, &gc, &ar, &br)) continue;
            bool ok = mbar_wait(&acc_full, (uint32_t)(lt & 1), tword, 24);
            ok = __all_sync(0xffffffffu, ok);   // every lane takes part in tcgen05.ld
            if (!ok) break;
            fence_after_sync();
            long long hw[32], lw[32];
#pragma unroll
            for (int l = 2; l <= S + 1; ++l) {
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((l - 2) * OZ_BN + h * 32), v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const long long d = (long long)__float2int_rn(v[j]);   // an exact integer below 2^24
                    if (l == 2)
                        hw[j] = d;
                    else if (l <= HEND)
                        hw[j] = hw[j] * 128 + d;
                    else if (l == 6)
                        lw[j] = d;
                    else
                        lw[j] = lw[j] * 128 + d;
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty);
            const int grow = gr + row;
            if (grow < args.m_end) {
                const int er = args.ea[ar + row];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int gcol = gc + h * 32 + j;
                    if (gcol >= args.n_end || (args.tri && grow < gcol)) continue;
                    const int e = er + args.eb[br + h * 32 + j];
                    double *pc = args.C + (long long)gcol * args.ldc + grow;
                    double c = *pc;
                    if (S + 1 > 5) c = fma(-(double)lw[j], pow2i(e + 2 - 7 * (S + 1)), c);
                    c = fma(-(double)hw[j], pow2i(e + 2 - 7 * HEND), c);
                    *pc = c;
                }
            }
            ++lt;
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
// One CTA per 32 rows: a column sweep for the row maxima, then 32 x 32
// tiles through shared memory so that each slice row is written along K.
__global__ void __launch_bounds__(256) k_oz_slice(const double *P, long long ld, int R, int K, int kchunk, int S,
                                                  __nv_bfloat16 *out, long long slice_stride, int Kp, int *exps,
                                                  long long exp_stride, const DevStatus *st) {
    __shared__ double tile[32][33];
    __shared__ double red[8][32];
    __shared__ int ex[32];
    __shared__ int skip;
    if (threadIdx.x == 0) skip = *(volatile const int *)&st->info;
    __syncthreads();
    if (skip) return;
    const int r0 = blockIdx.x * 32;
    const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);
    const int kpad_end = min(Kp, kbeg + (kchunk + OZ_BK - 1) / OZ_BK * OZ_BK);
    const int rr = threadIdx.x % 32, g = threadIdx.x / 32;
    double mx = 0.0;
    if (r0 + rr < R)
        for (int k = kbeg + g; k < kend; k += 8) mx = fmax(mx, fabs(P[(long long)k * ld + r0 + rr]));
    red[g][rr] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double m = red[0][rr];
        for (int q = 1; q < 8; ++q) m = fmax(m, red[q][rr]);
        int e = 0;
        if (m > 0.0) frexp(m, &e);   // m = f 2^e, f in [0.5, 1): |x| < 2^e on the row
        e = max(e, -960);
        ex[rr] = e;
        if (r0 + rr < R) exps[(long long)blockIdx.y * exp_stride + r0 + rr] = e;
    }
    __syncthreads();
    for (int c0 = kbeg; c0 < kpad_end; c0 += 32) {
        for (int t = threadIdx.x; t < 32 * 32; t += 256) {
            const int c = t / 32, r = t % 32;
            tile[c][r] = (r0 + r < R && c0 + c < kend) ? P[(long long)(c0 + c) * ld + r0 + r] : 0.0;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 32 * 32; t += 256) {
            const int r = t / 32, c = t % 32;
            if (r0 + r >= R || c0 + c >= Kp) continue;
            // x 2^(7S - 1 - e) is exact (a power-of-two scaling) and below 2^(7S - 1) in magnitude
            const double scale = __longlong_as_double((long long)(7 * S - 1 - ex[r] + 1023) << 52);
            long long X = __double2ll_rn(tile[c][r] * scale);
            __nv_bfloat16 *o = out + (long long)(r0 + r) * Kp + c0 + c;
            for (int s = S - 1; s >= 1; --s) {
                const long long d = ((X + 64) & 127) - 64;   // balanced digit in [-64, 63]
                o[(long long)s * slice_stride] = __float2bfloat16_rn((float)d);
                X = (X - d) >> 7;   // exact: X - d is a multiple of 128
            }
            o[0] = __float2bfloat16_rn((float)X);   // leading digit, |X| <= 64
        }
        __syncthreads();
    }
}

template <int S>
cudaError_t launch_oz_kernel(const CUtensorMap &ma, const CUtensorMap &mb, const OzArgs &a, int grid,
                             cudaStream_t s) {
    cudaError_t e = cudaFuncSetAttribute(k_oz_update<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)OzCfg<S>::SMEM);
    if (e != cudaSuccess) return e;
    k_oz_update<S><<<grid, OZ_THREADS, OzCfg<S>::SMEM, s>>>(ma, mb, a);
    return cudaGetLastError();
}

// 3-D tensor map over the slices: (k, row, slice), box 32 x rows_box x 1, 64-byte swizzle.
cudaError_t slice_map(CUtensorMap *map, const OzSlices &sl, int chunk, int rows_box) {
    tc::EncodeTiledFn enc = tc::encode_fn();
    if (!enc) return cudaErrorNotSupported;
    void *base = (__nv_bfloat16 *)sl.d + (size_t)chunk * sl.kchunk;   // 64-byte aligned: kchunk is a multiple of 32
    cuuint64_t dims[3] = {(cuuint64_t)std::min(sl.kchunk, sl.Kp - chunk * sl.kchunk), (cuuint64_t)sl.valid,
                          (cuuint64_t)sl.S};
    cuuint64_t strides[2] = {(cuuint64_t)sl.Kp * 2, (cuuint64_t)sl.slice_stride * 2};
    cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)rows_box, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult cr = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace

int oz_kmax(int S) { return (4096 / S) / OZ_BK * OZ_BK; }

size_t oz_slices_bytes(long long rows, int K, int S) {
    const long long Kp = (K + OZ_BK - 1) / OZ_BK * OZ_BK;
    const int nchunk = (K + oz_kmax(S) - 1) / oz_kmax(S);
    return (size_t)S * (size_t)rows * (size_t)Kp * 2 + sizeof(int) * (size_t)rows * nchunk + 512;
}

OzSlices oz_slices_carve(void *ws, long long rows, int K, int S) {
    OzSlices o;
    o.S = S;
    o.rows = rows;
    o.K = K;
    o.kchunk = oz_kmax(S);
    o.Kp = (K + OZ_BK - 1) / OZ_BK * OZ_BK;
    o.nchunk = (K + o.kchunk - 1) / o.kchunk;
    o.valid = rows;
    o.slice_stride = (long long)rows * o.Kp;
    o.d = ws;
    uintptr_t e = (uintptr_t)ws + (size_t)S * o.slice_stride * 2;
    o.e = (int *)((e + 255) & ~(uintptr_t)255);
    return o;
}

cudaError_t oz_slice(const double *P, long long ld, int R, const OzSlices &o, const DevStatus *st, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    if (R > o.rows || R > o.valid) return cudaErrorInvalidValue;
    dim3 grid((R + 31) / 32, o.nchunk);
    KScope ks(GEO_K_AUX, s, 0.0, (double)R * o.K * (16.0 + 2.0 * o.S));
    k_oz_slice<<<grid, 256, 0, s>>>(P, ld, R, o.K, o.kchunk, o.S, (__nv_bfloat16 *)o.d, o.slice_stride, o.Kp, o.e,
                                    o.rows, st);
    return cudaGetLastError();
}

cudaError_t oz_update(const OzSlices &A, const OzSlices &B, double *C, long long ldc, int r0, int c0, int rows,
                      int cols, int m_end, int n_end, int a_off, int b_off, int tri, int grid_cap, DevStatus *st,
                      cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (A.S != B.S || A.K != B.K || A.S < 3 || A.S > 8) return cudaErrorInvalidValue;
    const int S = A.S;
    OzArgs a;
    a.C = C;
    a.ldc = ldc;
    a.r0 = r0;
    a.c0 = c0;
    a.m_end = m_end;
    a.n_end = n_end;
    a.mt = (rows + OZ_BM - 1) / OZ_BM;
    a.nt = (cols + OZ_BN - 1) / OZ_BN;
    a.tri = tri;
    a.a_off = a_off;
    a.b_off = b_off;
    a.st = st;
    const long long ntiles = (long long)a.mt * a.nt;
    const int grid = (int)std::min<long long>(ntiles, std::max(1, std::min(grid_cap, tc::num_sms())));
    // algorithmic work: 2 K flops per output written (lower triangle when tri)
    const double rr = rows, cc = cols;
    const double outs = tri ? std::max(0.0, rr * cc - cc * (cc - 1.0) / 2.0) : rr * cc;
    for (int ch = 0; ch < A.nchunk; ++ch) {
        const int kc = std::min(A.kchunk, A.K - ch * A.kchunk);
        a.nk = (kc + OZ_BK - 1) / OZ_BK;
        a.ea = A.e + (long long)ch * A.rows;
        a.eb = B.e + (long long)ch * B.rows;
        CUtensorMap ma, mb;
        cudaError_t e;
        if ((e = slice_map(&ma, A, ch, OZ_BM)) != cudaSuccess || (e = slice_map(&mb, B, ch, OZ_BN)) != cudaSuccess)
            return e;
        KScope ks(GEO_K_TCGEMM, s, 2.0 * kc * outs, 16.0 * outs + 2.0 * S * kc * (rr + cc));
        switch (S) {
            case 3: e = launch_oz_kernel<3>(ma, mb, a, grid, s); break;
            case 4: e = launch_oz_kernel<4>(ma, mb, a, grid, s); break;
            case 5: e = launch_oz_kernel<5>(ma, mb, a, grid, s); break;
            case 6: e = launch_oz_kernel<6>(ma, mb, a, grid, s); break;
            case 7: e = launch_oz_kernel<7>(ma, mb, a, grid, s); break;
            default: e = launch_oz_kernel<8>(ma, mb, a, grid, s); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t oz_chol_workspace_bytes(int nrows, int nb, int S) { return oz_slices_bytes((long long)nrows + 128, nb, S); }

// Right-looking over panels of width nb with a lookahead of one (as the
// mixed form): step j slices its panel (rows below the diagonal tile,
// right-hand-side rows included), updates the next panel's tile column
// first, factors that panel's diagonal tile (and solves its right-hand-side
// rows) on a high-priority second stream while the rest of the trailing
// update runs (its persistent launch leaves SIDE_SMS SMs free), and solves
// the rows below the new diagonal tile in FP64 after the join.  POTRF and
// TRSM stay native FP64; every trailing update is emulated.
cudaError_t chol_oz_factor(double *A, long long ld, int N, int nrows, int nb, int S, void *ws, size_t ws_bytes,
                           DevStatus *st, cudaStream_t s) {
    constexpr int SIDE_SMS = 8;
    if (nb < 64 || nb % 64 != 0 || S < 3 || S > 8) return cudaErrorInvalidValue;
    if (ws_bytes < oz_chol_workspace_bytes(nrows, nb, S)) return cudaErrorInvalidValue;
    const OzSlices sl = oz_slices_carve(ws, (long long)nrows + 128, nb, S);
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
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        const int jb0 = std::min(nb, N);
        if ((r = chol64_panel(A, ld, 0, jb0, jb0, nrows, st, s)) != cudaSuccess) return r;
        for (int j0 = 0;;) {
            const int jb = std::min(nb, N - j0);
            const int t0 = j0 + jb;
            if (t0 >= N) break;
            // the panel's rows below the diagonal tile (right-hand-side rows included) as digit slices
            OzSlices p = sl;
            p.K = jb;
            p.nchunk = (jb + p.kchunk - 1) / p.kchunk;
            p.valid = nrows - t0;
            if ((r = oz_slice(A + (long long)j0 * ld + t0, ld, nrows - t0, p, st, s)) != cudaSuccess) return r;
            const int n1 = std::min(N, t0 + nb);
            // the next panel's tile column: rows [t0, nrows), cols [t0, n1)
            if ((r = oz_update(p, p, A, ld, t0, t0, nrows - t0, n1 - t0, nrows, n1, 0, 0, 1, all, st, s)) !=
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
            if ((r = chol64_panel(A, ld, t0, n1 - t0, N, nrows, st, s2)) != cudaSuccess) return r;
            if ((r = cudaEventRecord(e_pan, s2)) != cudaSuccess) return r;
            // the rest of the trailing update meanwhile: rows [n1, nrows), cols [n1, N)
            if ((r = oz_update(p, p, A, ld, n1, n1, nrows - n1, N - n1, nrows, N, n1 - t0, n1 - t0, 1,
                               all - SIDE_SMS, st, s)) != cudaSuccess)
                return r;
            if ((r = cudaStreamWaitEvent(s, e_pan, 0)) != cudaSuccess) return r;
            if ((r = chol64_panel(A, ld, t0, n1 - t0, n1, N, st, s, false)) != cudaSuccess) return r;
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
    return oz_update(sa, sb, C, ldc, 0, 0, m, n, m, n, 0, 0, 0, tc::num_sms(), st, s);
}
