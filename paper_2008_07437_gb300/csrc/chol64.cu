// Dense FP64 tiled Cholesky, Sigma = L L' (Sec. 5.2; the tile algorithm of
// Sec. 5.1 / Fig. 1 / Fig. 2: POTRF on the diagonal tile, TRSM on the panel,
// SYRK / GEMM on the trailing matrix).
//
// On GB300 the FP64 pipe runs at about 1.2 TFLOP/s (roughly two FP64 FMAs per
// clock per SM), some 60x below the FP32 pipe, so the dense FP64 path is
// bound by FP64 issue, not by memory: a rank-nb update reads 16 bytes per
// 2*nb flops.  The schedule is a right-looking blocked factorisation in
// stream order with two levels:
//   outer tiles of width nb (the tile size of the options): after the panel
//     of tile column k is factored, ONE launch updates the whole trailing
//     lower triangle (the SYRK and GEMM tasks of step k fused, rank nb);
//   inner blocks of width IB = 64 inside the panel: a one-CTA POTRF of the
//     64 x 64 diagonal block, a TRSM of every row below it, and a rank-64
//     update of the rest of the panel.
// Rows N .. nrows-1 are extra right-hand-side rows: they take part in every
// TRSM and update, so row N ends up holding (L^-1 z)' when it starts as z'
// (the forward substitution of Eq. 1 comes out of the factorisation).
#include "geo_internal.cuh"

namespace {

constexpr int IB = 64;

__device__ __forceinline__ void set_info(DevStatus *st, int row1) {
    // keep the smallest failing row
    int old = st->info;
    while (old == 0 || old > row1) {
        const int prev = atomicCAS(&st->info, old, row1);
        if (prev == old) break;
        old = prev;
    }
}

// ---- POTRF of one diagonal block (cb <= IB) in shared memory -------------
// Right-looking, two barriers per column: the rows below the pivot are scaled
// by 1 / L_jj, then the rank-1 update runs with thread (row r, group g)
// updating columns j + 1 + g, j + 5 + g, ...; the thread that updates the next
// diagonal entry (the only one to touch it) takes its square root and
// reciprocal right after its columns, so the pivot is ready at the next barrier.  The FP64
// pipe (two FMAs per clock per SM) bounds the block at cb^3 / 6 FMAs; square
// roots and divisions are taken once per column, not per thread.
__global__ void __launch_bounds__(256) k_potrf_diag(double *A, long long ld, int c0, int cb, DevStatus *st) {
    __shared__ double S[IB][IB + 1];   // S[col][row]: the block's Schur complement, then L
    __shared__ double sinv;            // 1 / L_jj of the current column
    __shared__ int fail;
    if (st->info) return;
    for (int t = threadIdx.x; t < cb * cb; t += blockDim.x) {
        const int c = t / cb, r = t % cb;
        S[c][r] = (r >= c) ? A[(long long)(c0 + c) * ld + c0 + r] : 0.0;
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    const int r = threadIdx.x % IB, g = threadIdx.x / IB;   // 4 column groups of 64 row threads
    auto pivot = [&](int j) {
        const double d = S[j][j];
        if (!(d > 0.0)) {
            fail = 1;
            set_info(st, c0 + j + 1);
        } else {
            const double l = sqrt(d);
            S[j][j] = l;
            sinv = 1.0 / l;
        }
    };
    if (threadIdx.x == 0) pivot(0);
    __syncthreads();
    for (int j = 0; j < cb; ++j) {
        if (fail) return;   // read after a barrier: uniform
        if (g == 0 && r > j && r < cb) S[j][r] *= sinv;
        __syncthreads();
        for (int c = j + 1 + g; c < cb; c += 4)
            if (r >= c && r < cb) S[c][r] -= S[j][r] * S[j][c];
        if (g == 0 && r == j + 1 && r < cb) pivot(j + 1);
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * cb; t += blockDim.x) {
        const int c = t / cb, r2 = t % cb;
        if (r2 >= c) A[(long long)(c0 + c) * ld + c0 + r2] = S[c][r2];
    }
}

// ---- TRSM: X <- X L^-T for the rows r0 .. r1-1, columns c0 .. c0+cb-1 ----
// L = A[c0:c0+cb, c0:c0+cb] (lower).  One CTA per 64 rows.
constexpr int TRSM_ROWS = 64;

__global__ void __launch_bounds__(256) k_trsm_rlt(double *A, long long ld, int c0, int cb, int r0, int r1,
                                                 const DevStatus *st) {
    extern __shared__ double smem[];
    double *Ls = smem;                       // Ls[c * IB + r]
    double *Xs = smem + IB * IB;             // Xs[c * (TRSM_ROWS + 1) + row]
    const int XLD = TRSM_ROWS + 1;
    if (st->info) return;
    const int rbase = r0 + blockIdx.x * TRSM_ROWS;
    const int nr = min(TRSM_ROWS, r1 - rbase);
    if (nr <= 0) return;
    for (int t = threadIdx.x; t < cb * cb; t += blockDim.x) {
        const int c = t / cb, r = t % cb;
        Ls[c * IB + r] = (r >= c) ? A[(long long)(c0 + c) * ld + c0 + r] : 0.0;
    }
    for (int t = threadIdx.x; t < cb * TRSM_ROWS; t += blockDim.x) {
        const int c = t / TRSM_ROWS, r = t % TRSM_ROWS;
        Xs[c * XLD + r] = (r < nr) ? A[(long long)(c0 + c) * ld + rbase + r] : 0.0;
    }
    __shared__ double dinv[IB];   // 1 / L_cc, one division per column
    __syncthreads();
    if (threadIdx.x < cb) dinv[threadIdx.x] = 1.0 / Ls[threadIdx.x * IB + threadIdx.x];
    __syncthreads();
    const int row = threadIdx.x % TRSM_ROWS, grp = threadIdx.x / TRSM_ROWS;   // 4 column groups
    for (int c = 0; c < cb; ++c) {
        if (grp == 0) Xs[c * XLD + row] *= dinv[c];
        __syncthreads();
        const double xc = Xs[c * XLD + row];
        for (int k = c + 1 + grp; k < cb; k += 4) Xs[k * XLD + row] -= xc * Ls[c * IB + k];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * TRSM_ROWS; t += blockDim.x) {
        const int c = t / TRSM_ROWS, r = t % TRSM_ROWS;
        if (r < nr) A[(long long)(c0 + c) * ld + rbase + r] = Xs[c * XLD + r];
    }
}

// ---- GEMM update: C -= A B' (FP64 FMA) -----------------------------------
// C = A[rC + i, cC + j] for i < m, j < n; A-operand rows rC.., cols kA..kA+k;
// B-operand rows cC.., same cols.  All inside the one matrix (column-major).
// CTA tiles that lie entirely above the diagonal (global row < global col
// everywhere) are skipped: those entries are never read.
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) k_dgemm_update(double *A, long long ld, int rC, int cC, int m, int n, int kA,
                                                      int k, const DevStatus *st) {
    __shared__ double As[GK][GT + 2];
    __shared__ double Bs[GK][GT + 2];
    if (st->info) return;
    const int tm = blockIdx.x * GT, tn = blockIdx.y * GT;
    if (rC + tm + GT - 1 < cC + tn) return;   // fully above the diagonal
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    const double *Ap = A + (long long)kA * ld + rC + tm;
    const double *Bp = A + (long long)kA * ld + cC + tn;
    for (int k0 = 0; k0 < k; k0 += GK) {
        for (int t = threadIdx.x; t < GK * GT; t += 256) {
            const int kk = t / GT, r = t % GT;
            const bool kin = (k0 + kk) < k;
            As[kk][r] = (kin && tm + r < m) ? Ap[(long long)(k0 + kk) * ld + r] : 0.0;
            Bs[kk][r] = (kin && tn + r < n) ? Bp[(long long)(k0 + kk) * ld + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = tn + tx + 16 * j;
        if (c >= n) continue;
        double *col = A + (long long)(cC + c) * ld + rC + tm;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = ty + 16 * i;
            if (tm + r < m) col[r] -= acc[i][j];
        }
    }
}

cudaError_t gemm_update(double *A, long long ld, int rC, int cC, int m, int n, int kA, int k, DevStatus *st,
                        cudaStream_t s) {
    if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
    dim3 grid((m + GT - 1) / GT, (n + GT - 1) / GT);
    // algorithmic work: the lower-triangle entries of C (rC == cC here), 2k flops each
    const double nn = n, mm = m;
    const double entries = (rC == cC) ? (nn * mm - nn * (nn - 1.0) / 2.0) : nn * mm;
    KScope ks(GEO_K_GEMM, s, 2.0 * k * entries, 8.0 * (2.0 * entries + (mm + nn) * k));
    k_dgemm_update<<<grid, 256, 0, s>>>(A, ld, rC, cC, m, n, kA, k, st);
    return cudaGetLastError();
}

}  // namespace

// Factor the panel of columns [j0, j0 + jb): its diagonal tile (inner 64-wide
// blocks: POTRF, TRSM, rank-64 update) and, carried through the same inner
// steps, the rows [x0, x1) below the tile (x0 >= j0 + jb; x0 == x1 = none).
// With factor_diag false the diagonal tile must already hold L and only the
// rows [x0, x1) are solved against it (X <- X L^-T).
cudaError_t chol64_panel(double *A, long long ld, int j0, int jb, int x0, int x1, DevStatus *st, cudaStream_t s,
                         bool factor_diag, const PanelUpdate *upd) {
    const size_t trsm_smem = sizeof(double) * (IB * IB + IB * (TRSM_ROWS + 1));
    cudaError_t e = cudaFuncSetAttribute(k_trsm_rlt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsm_smem);
    if (e != cudaSuccess) return e;
    const bool contiguous = factor_diag && (x0 == j0 + jb);
    for (int c0 = j0; c0 < j0 + jb; c0 += IB) {
        const int cb = min(IB, j0 + jb - c0);
        if (factor_diag) {
            KScope ks(GEO_K_POTRF, s, (double)cb * cb * cb / 3.0, 16.0 * cb * cb);
            k_potrf_diag<<<1, 256, 0, s>>>(A, ld, c0, cb, st);
        }
        const int rows0 = c0 + cb;
        // row ranges carried through this inner step
        int ra[2][2];
        int nrange = 0;
        if (!factor_diag) {
            if (x0 < x1) ra[nrange][0] = x0, ra[nrange][1] = x1, ++nrange;
        } else if (contiguous) {
            if (rows0 < x1) ra[nrange][0] = rows0, ra[nrange][1] = x1, ++nrange;
        } else {
            if (rows0 < j0 + jb) ra[nrange][0] = rows0, ra[nrange][1] = j0 + jb, ++nrange;
            if (x0 < x1) ra[nrange][0] = x0, ra[nrange][1] = x1, ++nrange;
        }
        for (int q = 0; q < nrange; ++q) {
            const int nr = ra[q][1] - ra[q][0];
            KScope ks(GEO_K_TRSM, s, (double)nr * cb * cb, 16.0 * nr * cb);
            k_trsm_rlt<<<(nr + TRSM_ROWS - 1) / TRSM_ROWS, 256, trsm_smem, s>>>(A, ld, c0, cb, ra[q][0], ra[q][1], st);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // rest of the panel: cols rows0 .. j0+jb-1
        if (rows0 < j0 + jb) {
            for (int q = 0; q < nrange; ++q) {
                e = upd ? upd->fn(upd, A, ld, ra[q][0], rows0, ra[q][1] - ra[q][0], j0 + jb - rows0, c0, cb, st, s)
                        : gemm_update(A, ld, ra[q][0], rows0, ra[q][1] - ra[q][0], j0 + jb - rows0, c0, cb, st, s);
                if (e != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}

cudaError_t chol64_gemm_update(double *A, long long ld, int rC, int cC, int m, int n, int kA, int k, DevStatus *st,
                               cudaStream_t s) {
    return gemm_update(A, ld, rC, cC, m, n, kA, k, st, s);
}

cudaError_t chol64_factor(double *A, long long ld, int N, int nrows, int nb, DevStatus *st, cudaStream_t s) {
    if (nb < IB) nb = IB;
    nb = (nb / IB) * IB;
    cudaError_t e = cudaSuccess;
    for (int j0 = 0; j0 < N; j0 += nb) {
        const int jb = min(nb, N - j0);
        e = chol64_panel(A, ld, j0, jb, j0 + jb, nrows, st, s);
        if (e != cudaSuccess) return e;
        // trailing update: rows j0+jb .. nrows-1, cols j0+jb .. N-1, rank jb
        const int t0 = j0 + jb;
        if (t0 < N) {
            e = gemm_update(A, ld, t0, t0, nrows - t0, N - t0, j0, jb, st, s);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}
