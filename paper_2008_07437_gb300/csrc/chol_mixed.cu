// Mixed-precision tiled Cholesky (the precision pattern the library offers on
// top of the paper's exact and TLR forms; the paper itself runs FP64 only).
//
// Tiles of width nb (a multiple of 128).  For panel k:
//   * diagonal tile: FP64 storage, FP64 POTRF (inner 64-wide blocks);
//   * rows below it: TRSM in FP32 (L_ik = A_ik L_kk^-T, inner 64-wide blocks,
//     FP32 SIMT), written back to the FP64 matrix;
//   * trailing update of tile (I, J), d = I - J:
//       d <= band : FP32 operands, FP32 SIMT FMA, FP64 read-modify-write of C
//                   (the diagonal tiles d = 0 included: they stay FP64 in
//                   storage and in their factorisation, their updates are FP32);
//       d >  band : FP16 operands split in two terms (hi + lo, three MMAs) or
//                   one BF16 term, with a power-of-two scale per panel row,
//                   tcgen05 tensor cores with FP32 accumulation in TMEM, FP64
//                   read-modify-write of C;
//   * the extra right-hand-side row N (Z', becoming (L^-1 Z)') is solved and
//     updated in FP64 throughout.
#include <cuda.h>

#include <algorithm>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "geo_internal.cuh"
#include "tc_gemm.cuh"

namespace {

constexpr int SB = 128, SK = 16;   // SIMT FP32 GEMM: 128 x 128 tile, K slices of 16, double-buffered

// Asynchronous global -> shared copies (cp.async, bytes beyond src_bytes
// are zero-filled; src_bytes = 0 reads nothing).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int src_bytes) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// C[i, j] -= sum_k A[i, k] B[j, k] (i < m, j < n); A, B column-major FP32; C
// column-major TC.  gr0 / gc0: global row / col of C(0, 0) for the class
// filter (nb-tile distance in [dlo, dhi]) and, when tri, the skip of tiles
// entirely above the diagonal.
//
// 256 threads; thread (tx, ty) = (t % 16, t / 16) owns rows {4 tx .. 4 tx + 3,
// 64 + 4 tx ..} and cols {4 ty .., 64 + 4 ty ..} of the tile: the fragments
// are float4 reads of shared memory, and the epilogue updates 4 consecutive
// rows of a column per access (32 bytes of FP64 C).  K slices of 16 are
// copied into two shared-memory stages with cp.async while the other stage
// is used.  vec: A, B, C and their leading dimensions allow 16-byte accesses.
template <typename TC>
__global__ void __launch_bounds__(256, 2) k_sgemm_nt(TC *C, long long ldc, const float *__restrict__ A, long long lda,
                                                     const float *__restrict__ B, long long ldb, int m, int n, int k,
                                                     int gr0, int gc0, int nb, int dlo, int dhi, int tri, int vec,
                                                     const DevStatus *st) {
    __shared__ __align__(16) float As[2][SK][SB + 4];
    __shared__ __align__(16) float Bs[2][SK][SB + 4];
    if (st->info) return;
    const int tm = blockIdx.x * SB, tn = blockIdx.y * SB;
    const int gr = gr0 + tm, gc = gc0 + tn;
    if (nb > 0) {
        const int dmin = gr / nb - (gc + SB - 1) / nb, dmax = (gr + SB - 1) / nb - gc / nb;
        if (dmax < dlo || dmin > dhi) return;
        // a CTA tile never straddles classes when nb is a multiple of 128 and the region is nb-aligned
    }
    if (tri && gr + SB - 1 < gc) return;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    // slice element e = threadIdx.x + 256 q (q = 0, 1): k row e / 32, rows 4 (e % 32) .. + 3
    auto load = [&](int k0, int buf) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int e = threadIdx.x + 256 * q;
            const int kk = e / 32, r = 4 * (e % 32);
            const bool kin = k0 + kk < k;
            const int va = kin ? max(0, min(4, m - (tm + r))) : 0;   // valid elements of the 4
            const int vb = kin ? max(0, min(4, n - (tn + r))) : 0;
            const float *pa = va ? A + (long long)(k0 + kk) * lda + tm + r : A;
            const float *pb = vb ? B + (long long)(k0 + kk) * ldb + tn + r : B;
            if (vec) {
                cp_async16(&As[buf][kk][r], pa, 4 * va);
                cp_async16(&Bs[buf][kk][r], pb, 4 * vb);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    cp_async4(&As[buf][kk][r + i], i < va ? pa + i : A, i < va ? 4 : 0);
                    cp_async4(&Bs[buf][kk][r + i], i < vb ? pb + i : B, i < vb ? 4 : 0);
                }
            }
        }
        cp_async_commit();
    };
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    load(0, 0);
    int buf = 0;
    for (int k0 = 0; k0 < k; k0 += SK) {
        if (k0 + SK < k) {
            load(k0 + SK, buf ^ 1);   // the other stage: released by the barrier that ended its last use
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SK; ++kk) {
            float a[8], b[8];
            const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][tx * 4]);
            const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][64 + tx * 4]);
            const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][ty * 4]);
            const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][64 + ty * 4]);
            a[0] = a0.x, a[1] = a0.y, a[2] = a0.z, a[3] = a0.w, a[4] = a1.x, a[5] = a1.y, a[6] = a1.z, a[7] = a1.w;
            b[0] = b0.x, b[1] = b0.y, b[2] = b0.z, b[3] = b0.w, b[4] = b1.x, b[5] = b1.y, b[6] = b1.z, b[7] = b1.w;
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();   // every thread is done with this stage before it is refilled
        buf ^= 1;
    }
    // epilogue: C -= acc, 4 consecutive rows of a column per access
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = tn + (j < 4 ? ty * 4 + j : 64 + ty * 4 + (j - 4));
        if (c >= n) continue;
        TC *col = C + (long long)c * ldc + tm;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int r = h * 64 + tx * 4;
            if (vec && tm + r + 3 < m) {
                if constexpr (sizeof(TC) == 8) {
                    double2 *pc = reinterpret_cast<double2 *>(col + r);
                    double2 u = pc[0], w = pc[1];
                    u.x -= (double)acc[4 * h + 0][j];
                    u.y -= (double)acc[4 * h + 1][j];
                    w.x -= (double)acc[4 * h + 2][j];
                    w.y -= (double)acc[4 * h + 3][j];
                    pc[0] = u;
                    pc[1] = w;
                } else {
                    float4 *pc = reinterpret_cast<float4 *>(col + r);
                    float4 u = *pc;
                    u.x -= acc[4 * h + 0][j];
                    u.y -= acc[4 * h + 1][j];
                    u.z -= acc[4 * h + 2][j];
                    u.w -= acc[4 * h + 3][j];
                    *pc = u;
                }
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (tm + r + i < m) col[r + i] -= (TC)acc[4 * h + i][j];
            }
        }
    }
}

// FP32 TRSM on a column-major FP32 block X (rows, 64 cols, ldx): X <- X L^-T,
// L = the 64 x 64 lower block of the FP64 diagonal tile (read as FP32).
constexpr int TR_ROWS = 64;
__global__ void __launch_bounds__(256) k_trsm32(float *X, long long ldx, int rows, const double *L, long long ldl,
                                               int cb, const DevStatus *st) {
    __shared__ float Ls[64][65];
    __shared__ float Xs[64][TR_ROWS + 1];
    if (st->info) return;
    const int rb = blockIdx.x * TR_ROWS;
    const int nr = min(TR_ROWS, rows - rb);
    for (int t = threadIdx.x; t < cb * cb; t += 256) {
        const int c = t / cb, r = t % cb;
        Ls[c][r] = (r >= c) ? (float)L[(long long)c * ldl + r] : 0.f;
    }
    for (int t = threadIdx.x; t < cb * TR_ROWS; t += 256) {
        const int c = t / TR_ROWS, r = t % TR_ROWS;
        Xs[c][r] = (r < nr) ? X[(long long)c * ldx + rb + r] : 0.f;
    }
    __syncthreads();
    const int row = threadIdx.x % TR_ROWS, grp = threadIdx.x / TR_ROWS;
    for (int c = 0; c < cb; ++c) {
        if (grp == 0) Xs[c][row] /= Ls[c][c];
        __syncthreads();
        const float xc = Xs[c][row];
        for (int kk = c + 1 + grp; kk < cb; kk += 4) Xs[kk][row] -= xc * Ls[c][kk];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * TR_ROWS; t += 256) {
        const int c = t / TR_ROWS, r = t % TR_ROWS;
        if (r < nr) X[(long long)c * ldx + rb + r] = Xs[c][r];
    }
}

// FP64 panel block -> FP32 (column-major, ldp), rows [0, rows), cols [0, cols).
__global__ void k_to_f32(const double *A, long long lda, int rows, int cols, float *P, long long ldp) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)rows * cols) return;
    const int c = (int)(t / rows), r = (int)(t % rows);
    P[(long long)c * ldp + r] = (float)A[(long long)c * lda + r];
}

// FP32 panel -> FP64 matrix.
__global__ void k_to_f64(const float *P, long long ldp, int rows, int cols, double *A, long long lda) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)rows * cols) return;
    const int c = (int)(t / rows), r = (int)(t % rows);
    A[(long long)c * lda + r] = (double)P[(long long)c * ldp + r];
}

// Per panel row r: power-of-two scale s_r with max_c |x[r, c]| s_r < 2^14, and
// the K-major (row-major) low-precision copies x s = hi + lo (lo only when
// two terms are kept); 1 / s_r goes to inv_scale[r].  One CTA per 64 rows:
// a column sweep for the row maxima (coalesced along rows), then 64 x 64
// tiles transposed through shared memory so that the stores run along K.
template <typename T16>
__global__ void __launch_bounds__(256) k_to_lowp(const float *P, long long ldp, int rows, int cols, T16 *Hhi,
                                                 T16 *Hlo, int Kp, double *inv_scale) {
    __shared__ float red[4][64];
    __shared__ float sc[64];
    __shared__ float tile[64][65];
    const int rb = blockIdx.x * 64;
    const int rr = threadIdx.x % 64, g = threadIdx.x / 64;
    float mx = 0.f;
    if (rb + rr < rows)
        for (int c = g; c < cols; c += 4) mx = fmaxf(mx, fabsf(P[(long long)c * ldp + rb + rr]));
    red[g][rr] = mx;
    __syncthreads();
    if (threadIdx.x < 64) {
        const float m = fmaxf(fmaxf(red[0][rr], red[1][rr]), fmaxf(red[2][rr], red[3][rr]));
        int e = 0;
        if (m > 0.f) frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
        const float s = (m > 0.f) ? ldexpf(1.f, 14 - e) : 1.f;
        sc[rr] = s;
        if (rb + rr < rows) inv_scale[rb + rr] = 1.0 / (double)s;
    }
    __syncthreads();
    for (int c0 = 0; c0 < Kp; c0 += 64) {
        for (int t = threadIdx.x; t < 64 * 64; t += 256) {
            const int c = t / 64, r = t % 64;
            tile[c][r] = (rb + r < rows && c0 + c < cols) ? P[(long long)(c0 + c) * ldp + rb + r] * sc[r] : 0.f;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < 64 * 64; t += 256) {
            const int r = t / 64, c = t % 64;
            if (rb + r >= rows) continue;
            const float v = tile[c][r];
            const T16 hi = (T16)v;
            Hhi[(long long)(rb + r) * Kp + c0 + c] = hi;
            if (Hlo) Hlo[(long long)(rb + r) * Kp + c0 + c] = (T16)(v - (float)hi);
        }
        __syncthreads();
    }
}

using tc::EncodeTiledFn;
using tc::encode_fn;
using tc::num_sms;

template <typename TC>
cudaError_t sgemm(TC *C, long long ldc, const float *A, long long lda, const float *B, long long ldb, int m, int n,
                  int k, int gr0, int gc0, int nb, int dlo, int dhi, int tri, const DevStatus *st, double flops,
                  cudaStream_t s) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid((m + SB - 1) / SB, (n + SB - 1) / SB);
    // 16-byte vector accesses when every tile row start is 16-byte aligned
    const int vec = ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && ((uintptr_t)C % 16 == 0) && lda % 4 == 0 &&
                    ldb % 4 == 0 && (ldc * (long long)sizeof(TC)) % 16 == 0;
    KScope ks(GEO_K_SGEMM, s, flops, 0.0);
    k_sgemm_nt<TC><<<grid, 256, 0, s>>>(C, ldc, A, lda, B, ldb, m, n, k, gr0, gc0, nb, dlo, dhi, tri, vec, st);
    return cudaGetLastError();
}

}  // namespace

namespace {

// One panel's workspace: FP32 copy of the rows below the diagonal tile,
// FP32 copy of the diagonal tile, FP16 (or BF16) hi / lo copies, row scales.
struct PanelWs {
    float *P32, *LD32;
    void *P16, *P16lo;
    double *inv_scale;
};

size_t panel_ws_bytes(int N, int nb) {
    const size_t rows = (size_t)N + 128;
    const size_t ldp = (rows + 3) / 4 * 4;
    return sizeof(float) * ldp * nb              // FP32 panel
           + sizeof(float) * (size_t)nb * nb     // FP32 copy of the diagonal tile
           + 4 * rows * (size_t)nb               // FP16 / BF16 panel, hi and lo
           + sizeof(double) * rows               // row scales
           + 4096;
}

PanelWs carve(uint8_t *w, size_t rows_max, long long ldp, int nb) {
    PanelWs W;
    W.P32 = (float *)w;
    w += sizeof(float) * ldp * nb;
    W.LD32 = (float *)w;
    w += sizeof(float) * (size_t)nb * nb;
    w = (uint8_t *)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    W.P16 = w;
    w += 2 * rows_max * (size_t)nb;
    W.P16lo = w;
    w += 2 * rows_max * (size_t)nb;
    w = (uint8_t *)(((uintptr_t)w + 255) & ~(uintptr_t)255);
    W.inv_scale = (double *)w;
    return W;
}

struct MixedGeom {
    double *A;
    long long ld;
    int N, nrows, nb, band, lowp;
    long long ldp;
    DevStatus *st;
};

// Diagonal tile of panel [j0, j0 + jb) in FP64, carrying the right-hand-side
// rows [N, nrows): a chain of small latency-bound launches.
cudaError_t mixed_panel_diag(const MixedGeom &G, int j0, cudaStream_t s) {
    const int jb = min(G.nb, G.N - j0);
    const int t0 = j0 + jb;
    return chol64_panel(G.A, G.ld, j0, jb, (G.nrows > G.N) ? G.N : t0, (G.nrows > G.N) ? G.nrows : t0, G.st, s);
}

// Rows below the diagonal tile of panel j0: solved in FP32 against the
// factored tile and written back, plus their low-precision copy with
// per-row scales.
cudaError_t mixed_panel_rows(const MixedGeom &G, int j0, const PanelWs &W, cudaStream_t s) {
    double *A = G.A;
    const long long ld = G.ld, ldp = G.ldp;
    const int N = G.N, nb = G.nb;
    DevStatus *st = G.st;
    const int jb = min(nb, N - j0);
    const int t0 = j0 + jb;
    cudaError_t e;
    if (t0 >= N) return cudaSuccess;
    const int R = N - t0;   // rows of the panel below the diagonal tile
    {
        const long long tot = (long long)R * jb;
        KScope ks(GEO_K_AUX, s);
        k_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A + (long long)j0 * ld + t0, ld, R, jb, W.P32, ldp);
    }
    {
        const long long tot = (long long)jb * jb;
        KScope ks(GEO_K_AUX, s);
        k_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(A + (long long)j0 * ld + j0, ld, jb, jb, W.LD32, nb);
    }
    for (int c0 = 0; c0 < jb; c0 += 64) {
        const int cb = min(64, jb - c0);
        {
            KScope ks(GEO_K_TRSM, s, (double)R * cb * cb, 0.0);
            k_trsm32<<<(R + TR_ROWS - 1) / TR_ROWS, 256, 0, s>>>(W.P32 + (long long)c0 * ldp, ldp, R,
                                                                 A + (long long)(j0 + c0) * ld + j0 + c0, ld, cb, st);
        }
        if (c0 + cb < jb) {
            // P32[:, c0+cb:] -= P32[:, c0:c0+cb] LD[c0+cb:, c0:c0+cb]'
            e = sgemm<float>(W.P32 + (long long)(c0 + cb) * ldp, ldp, W.P32 + (long long)c0 * ldp, ldp,
                             W.LD32 + (long long)c0 * nb + c0 + cb, nb, R, jb - c0 - cb, cb, 0, 0, 0, 0, 0, 0, st,
                             2.0 * R * (jb - c0 - cb) * cb, s);
            if (e != cudaSuccess) return e;
        }
    }
    {
        const long long tot = (long long)R * jb;
        KScope ks(GEO_K_AUX, s);
        k_to_f64<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(W.P32, ldp, R, jb, A + (long long)j0 * ld + t0, ld);
    }
    // low-precision copy with per-row scales (only needed when far tiles exist)
    const bool far = (N - 1) / nb - t0 / nb > G.band;
    if (far) {
        const int nblk = (R + 63) / 64;
        KScope ks(GEO_K_AUX, s);
        if (G.lowp)
            k_to_lowp<__nv_bfloat16><<<nblk, 256, 0, s>>>(W.P32, ldp, R, jb, (__nv_bfloat16 *)W.P16, nullptr, nb,
                                                          W.inv_scale);
        else
            k_to_lowp<__half><<<nblk, 256, 0, s>>>(W.P32, ldp, R, jb, (__half *)W.P16, (__half *)W.P16lo, nb,
                                                   W.inv_scale);
    }
    return cudaGetLastError();
}

// Update of the trailing columns [ca, cb) (nb-aligned, ca >= t0) by panel j0:
// tiles within the band in FP32 SIMT, tiles beyond on the tensor cores, the
// right-hand-side rows in FP64.
cudaError_t mixed_update(const MixedGeom &G, int j0, int ca, int cb, const PanelWs &W, EncodeTiledFn enc,
                         uint32_t idesc, int grid_cap, cudaStream_t s) {
    double *A = G.A;
    const long long ld = G.ld, ldp = G.ldp;
    const int N = G.N, nrows = G.nrows, nb = G.nb, band = G.band;
    DevStatus *st = G.st;
    const int jb = min(nb, N - j0);
    const int t0 = j0 + jb;
    const int R = N - t0;
    cudaError_t e;
    // band and diagonal tiles in FP32: rows [ca, N), cols [ca, cb)
    {
        double ent = 0.0;
        const int Ja = ca / nb, Jb = (cb - 1) / nb, T1 = (N - 1) / nb;
        for (int I = Ja; I <= T1; ++I) {
            const double hi = min(N, (I + 1) * nb) - I * nb;
            for (int J = max(Ja, I - band); J <= min(I, Jb); ++J) {
                const double wj = min(N, (J + 1) * nb) - J * nb;
                ent += (I == J) ? hi * (hi + 1) / 2 : hi * wj;
            }
        }
        e = sgemm<double>(A + (long long)ca * ld + ca, ld, W.P32 + (ca - t0), ldp, W.P32 + (ca - t0), ldp, N - ca,
                          cb - ca, jb, ca, ca, nb, 0, band, 1, st, 2.0 * jb * ent, s);
        if (e != cudaSuccess) return e;
    }
    // far tiles on the tensor cores
    const int T0 = t0 / nb, Ja = ca / nb, T1 = (N - 1) / nb;
    const bool col_only = (cb - ca <= nb) && Ja == T0;
    const long long far_rows = std::max(0, T1 - Ja - band);
    if (far_rows > 0) {
        const int terms = G.lowp ? 1 : 2;   // FP16 keeps hi + lo; BF16 keeps one term
        CUtensorMap map;
        cuuint64_t dims[2] = {(cuuint64_t)nb, (cuuint64_t)R};
        cuuint64_t strides[1] = {(cuuint64_t)nb * 2};
        cuuint32_t box[2] = {64, 128};
        cuuint32_t es[2] = {1, 1};
        CUresult cr = enc(&map, G.lowp ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, W.P16,
                          dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
        CUtensorMap map_lo = map;
        if (terms == 2) {
            cr = enc(&map_lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, W.P16lo, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
        }
        tc::TcArgs a;
        a.C = A;
        a.ldc = ld;
        a.N = N;
        a.prow0 = t0;
        a.K = nb;   // columns jb..nb of the low-precision copy are zero
        a.nb = nb;
        a.band = band;
        a.T0 = Ja;
        a.col_only = col_only ? 1 : 0;
        const long long per2 = (long long)(nb / tc::BM) * (nb / tc::BM);
        a.ntiles = (col_only ? far_rows : far_rows * (far_rows + 1) / 2) * per2;
        a.inv_scale = W.inv_scale;
        a.terms = terms;
        a.st = st;
        double ent = 0.0;
        const int Jb = (cb - 1) / nb;
        for (int I = Ja; I <= T1; ++I) {
            const double hi = min(N, (I + 1) * nb) - I * nb;
            for (int J = Ja; J < I - band && J <= Jb; ++J) ent += hi * nb;
        }
        const int grid = (int)std::min<long long>(a.ntiles, std::max(1, std::min(grid_cap, num_sms())));
        KScope ks(GEO_K_TCGEMM, s, 2.0 * jb * ent * (terms == 2 ? 3 : 1), 16.0 * ent + 2.0 * terms * (double)R * jb);
        if (grid > 0) tc::k_tc_update<<<grid, tc::THREADS_P, tc::SMEM_BYTES, s>>>(map, map_lo, a, idesc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // right-hand-side rows in FP64
    if (nrows > N) return chol64_gemm_update(A, ld, N, ca, nrows - N, cb - ca, j0, jb, st, s);
    return cudaSuccess;
}

}  // namespace

size_t mixed_workspace_bytes(int N, int nb) { return panel_ws_bytes(N, nb); }

// Right-looking over panels with a lookahead of one: step j first updates the
// next panel's tile column; the diagonal tile of that panel (a chain of small
// FP64 launches) is then factored on a second, high-priority stream while the
// rest of step j's trailing update runs (its persistent tensor-core launch
// leaves SIDE_SMS SMs free for it); the rows below it are solved after the
// join.  Every entry receives the same operations in the same order as
// without the lookahead.
constexpr int SIDE_SMS = 8;

cudaError_t chol_mixed_factor(double *A, long long ld, int N, int nrows, int nb, int band, int lowp, void *ws,
                              size_t ws_bytes, DevStatus *st, cudaStream_t s) {
    if (nb % 128 != 0 || nb <= 0) return cudaErrorInvalidValue;
    if (ws_bytes < mixed_workspace_bytes(N, nb)) return cudaErrorInvalidValue;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(tc::k_tc_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc::SMEM_BYTES);
    if (e != cudaSuccess) return e;
    const size_t rows_max = (size_t)N + 128;
    MixedGeom G{A, ld, N, nrows, nb, band, lowp, (long long)((rows_max + 3) / 4 * 4), st};
    const PanelWs W = carve((uint8_t *)ws, rows_max, G.ldp, nb);
    const uint32_t idesc = tc::instr_desc(lowp ? 1 : 0);
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaStream_t s2 = nullptr;
    cudaEvent_t e_upd = nullptr, e_pan = nullptr;
    if ((e = cudaStreamCreateWithPriority(&s2, cudaStreamNonBlocking, prio_hi)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&e_upd, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&e_pan, cudaEventDisableTiming)) != cudaSuccess) {
        cudaStreamDestroy(s2);
        if (e_upd) cudaEventDestroy(e_upd);
        return e;
    }
    const int all = num_sms();
    auto run = [&]() -> cudaError_t {
        cudaError_t r;
        if ((r = mixed_panel_diag(G, 0, s)) != cudaSuccess || (r = mixed_panel_rows(G, 0, W, s)) != cudaSuccess)
            return r;
        for (int j0 = 0; j0 < N; j0 += nb) {
            const int t0 = j0 + min(nb, N - j0);
            if (t0 >= N) break;
            const int n1 = min(N, t0 + nb);
            // the next panel's tile column first, then its diagonal tile on the second stream
            if ((r = mixed_update(G, j0, t0, n1, W, enc, idesc, all, s)) != cudaSuccess) return r;
            if ((r = cudaEventRecord(e_upd, s)) != cudaSuccess) return r;
            if ((r = cudaStreamWaitEvent(s2, e_upd, 0)) != cudaSuccess) return r;
            if ((r = mixed_panel_diag(G, t0, s2)) != cudaSuccess) return r;
            if ((r = cudaEventRecord(e_pan, s2)) != cudaSuccess) return r;
            // the rest of this step's trailing update meanwhile
            if (n1 < N && (r = mixed_update(G, j0, n1, N, W, enc, idesc, all - SIDE_SMS, s)) != cudaSuccess)
                return r;
            if ((r = cudaStreamWaitEvent(s, e_pan, 0)) != cudaSuccess) return r;
            if ((r = mixed_panel_rows(G, t0, W, s)) != cudaSuccess) return r;
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
