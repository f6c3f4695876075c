// Kernels of the multivariate MLOE / MMOM criteria (Eq. 5 - Eq. 8,
// Algorithm 1 of Sec. 5.4).  The cross-covariances c(s0) of the prediction
// locations ride along as extra rows of the covariance matrix through its
// factorisation (as Z does for Eq. 1), which leaves (L^-1 c)' in those rows;
// the remaining products are a right-side triangular solve X L = B and a
// product X L with the lower factor, both by 64-column blocks.
#include "geo_internal.cuh"

namespace {

constexpr int XB = 64;   // column block of the right-side solve and product

// out[(p r + j) * ld + (p q + i)] = C_ij(|s0_q - s_r|): rows = prediction
// locations (AoS), columns = observed locations (SoA, the factor's order).
__global__ void __launch_bounds__(256) k_covgen_cross(const CovParams cp, const double *__restrict__ s0, int m,
                                                      const double *__restrict__ lx, const double *__restrict__ ly,
                                                      int n, double *out, long long ld) {
    const int q = blockIdx.y * 64 + (threadIdx.x % 64);
    const int r = blockIdx.x * 4 + (threadIdx.x / 64);
    if (q >= m || r >= n) return;
    const double dx = s0[2 * q] - lx[r], dy = s0[2 * q + 1] - ly[r];
    const double x = sqrt(dx * dx + dy * dy) * cp.inv_a;
    const int p = cp.p;
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    matern_block(x, cp, v);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) out[(long long)(p * r + j) * ld + (long long)p * q + i] = v[i * GEO_PMAX_DEV + j];
}

// For rows q < R of X (column-major, ldx, N columns): s[q] = sum_c X[q, c]^2
// and, with Y, d[q] = sum_c X[q, c] Y[q, c]; one thread per row, columns in order.
__global__ void k_row_sums(const double *__restrict__ X, long long ldx, const double *__restrict__ Y, long long ldy,
                           int R, int N, double *s, double *d) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R) return;
    double a = 0.0, b = 0.0;
    for (int c = 0; c < N; ++c) {
        const double x = X[(long long)c * ldx + q];
        a = fma(x, x, a);
        if (Y) b = fma(x, Y[(long long)c * ldy + q], b);
    }
    s[q] = a;
    if (d) d[q] = b;
}

// X[:, c0 .. c0 + cb) <- X[:, c0 ..) L[c0 .., c0 ..)^-1 for the lower block
// L_JJ (cb <= 64): per row, x_c = (b_c - sum_{k > c} x_k L[k, c]) / L[c, c]
// from the last column; one thread per row.
__global__ void __launch_bounds__(128) k_trsm_right_lower_diag(double *X, long long ldx, int R, const double *L,
                                                               long long ldl, int c0, int cb) {
    __shared__ double Ls[XB][XB + 1];   // Ls[k][c] = L[c0 + k, c0 + c], k >= c
    for (int e = threadIdx.x; e < XB * XB; e += blockDim.x) {
        const int k = e / XB, c = e % XB;
        Ls[k][c] = (k < cb && c < cb && k >= c) ? L[(long long)(c0 + c) * ldl + c0 + k] : 0.0;
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R) return;
    double x[XB];
#pragma unroll
    for (int c = 0; c < XB; ++c) x[c] = (c < cb) ? X[(long long)(c0 + c) * ldx + q] : 0.0;
#pragma unroll
    for (int c = XB - 1; c >= 0; --c) {
        if (c < cb) {
            double t = x[c];
#pragma unroll
            for (int k = c + 1; k < XB; ++k) t -= x[k] * Ls[k][c];
            x[c] = t / Ls[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < XB; ++c)
        if (c < cb) X[(long long)(c0 + c) * ldx + q] = x[c];
}

// X[:, c0 .. c0 + cb) <- X[:, c0 ..) L[c0 .., c0 ..)^-T: per row,
// x_c = (b_c - sum_{k < c} x_k L[c, k]) / L[c, c] from the first column; one thread per row.
__global__ void __launch_bounds__(128) k_trsm_right_upper_diag(double *X, long long ldx, int R, const double *L,
                                                               long long ldl, int c0, int cb) {
    __shared__ double Ls[XB][XB + 1];   // Ls[c][k] = L[c0 + c, c0 + k], k <= c
    for (int e = threadIdx.x; e < XB * XB; e += blockDim.x) {
        const int k = e / XB, c = e % XB;
        Ls[c][k] = (k < cb && c < cb && k <= c) ? L[(long long)(c0 + k) * ldl + c0 + c] : 0.0;
    }
    __syncthreads();
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R) return;
    double x[XB];
#pragma unroll
    for (int c = 0; c < XB; ++c) x[c] = (c < cb) ? X[(long long)(c0 + c) * ldx + q] : 0.0;
#pragma unroll
    for (int c = 0; c < XB; ++c) {
        if (c < cb) {
            double t = x[c];
#pragma unroll
            for (int k = 0; k < c; ++k) t -= x[k] * Ls[c][k];
            x[c] = t / Ls[c][c];
        }
    }
#pragma unroll
    for (int c = 0; c < XB; ++c)
        if (c < cb) X[(long long)(c0 + c) * ldx + q] = x[c];
}

// var[q] = C_ii(0) - s[q], i = q mod p.
__global__ void k_var_finish(const double *s, int R, int p, double c0, double c1, double c2, double c3, double *var) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= R) return;
    const int i = q % p;
    const double c = (i == 0) ? c0 : (i == 1) ? c1 : (i == 2) ? c2 : c3;
    var[q] = c - s[q];
}

// Y = X' through a 32 x 32 shared-memory tile: X is R x C (column-major, ldx),
// Y is C x R (column-major, ldy); reads and writes both run along columns.
__global__ void __launch_bounds__(256) k_transpose(const double *__restrict__ X, long long ldx, int R, int C,
                                                   double *__restrict__ Y, long long ldy) {
    __shared__ double t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = r0 + threadIdx.x, c = c0 + j;
        if (r < R && c < C) t[j][threadIdx.x] = X[(long long)c * ldx + r];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = c0 + threadIdx.x, r = r0 + j;
        if (r < R && c < C) Y[(long long)r * ldy + c] = t[threadIdx.x][j];
    }
}

// s[q] = sum_{c < N} Y[q * ldy + c]^2 for q < R: one warp per column, lanes
// striding the column, then a fixed shuffle tree.
__global__ void __launch_bounds__(256) k_col_sumsq(const double *__restrict__ Y, long long ldy, int N, int R,
                                                   double *s) {
    const int q = blockIdx.x * 8 + threadIdx.x / 32, lane = threadIdx.x % 32;
    if (q >= R) return;   // uniform over the warp
    double a = 0.0;
    for (int c = lane; c < N; c += 32) {
        const double y = Y[(long long)q * ldy + c];
        a = fma(y, y, a);
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
    if (lane == 0) s[q] = a;
}

// Zero the strictly upper part of every 64 x 64 diagonal block of L (those
// entries are never part of the factor), so that block products see a lower
// triangle.
__global__ void k_zero_diag_upper(double *L, long long ld, int N) {
    const int b = blockIdx.x;
    const int c0 = b * XB;
    for (int e = threadIdx.x; e < XB * XB; e += blockDim.x) {
        const int c = e / XB, r = e % XB;
        if (r < c && c0 + c < N && c0 + r < N) L[(long long)(c0 + c) * ld + c0 + r] = 0.0;
    }
}

}  // namespace

cudaError_t launch_covgen_cross(const CovParams &cp, const double *s0, int m, const double *lx, const double *ly,
                                int n, double *out, long long ld, cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    dim3 grid((n + 3) / 4, (m + 63) / 64);
    KScope ks(GEO_K_COVGEN, s, 0.0, 8.0 * cp.p * (double)m * cp.p * (double)n);
    k_covgen_cross<<<grid, 256, 0, s>>>(cp, s0, m, lx, ly, n, out, ld);
    return cudaGetLastError();
}

cudaError_t launch_row_sums(const double *X, long long ldx, const double *Y, long long ldy, int R, int N, double *s,
                            double *d, cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    KScope ks(GEO_K_REDUCE, st, 2.0 * R * (double)N, 8.0 * R * (double)N * (Y ? 2 : 1));
    k_row_sums<<<(R + 127) / 128, 128, 0, st>>>(X, ldx, Y, ldy, R, N, s, d);
    return cudaGetLastError();
}

// X <- X L^-1 (X: R x N column-major, ldx; L lower N x N, ldl), by 64-column
// blocks from the last: X_J <- X_J L_JJ^-1, then X[:, :J] -= X_J L[J, :J].
cudaError_t trsm_right_lower(double *X, long long ldx, int R, const double *L, long long ldl, int N, void *arena_dev,
                             cudaStream_t s) {
    if (R <= 0 || N <= 0) return cudaSuccess;
    GemmDesc *gd = (GemmDesc *)arena_dev;
    const int nblk = (N + XB - 1) / XB;
    for (int J = nblk - 1; J >= 0; --J) {
        const int c0 = J * XB, cb = min(XB, N - c0);
        {
            KScope ks(GEO_K_SOLVE, s, (double)R * cb * cb, 8.0 * 2.0 * R * cb);
            k_trsm_right_lower_diag<<<(R + 127) / 128, 128, 0, s>>>(X, ldx, R, L, ldl, c0, cb);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (c0 > 0) {
            GemmDesc g{R, c0, cb, 0, 0, X + (long long)c0 * ldx, ldx, L + c0, ldl, X, ldx, -1.0, 1.0};
            // one descriptor per step, written in stream order into a ring in device memory
            GemmDesc *d = gd + (J % 64);
            if ((e = cudaMemcpyAsync(d, &g, sizeof(g), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
            if ((e = launch_bgemm(d, 1, ((R + 63) / 64) * ((c0 + 63) / 64), s, 2.0 * R * c0 * cb)) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

// X <- X L^-T (X: R x N, L lower), by 64-column blocks from the first:
// X_J <- X_J L_JJ^-T, then X[:, J+1:] -= X_J L[J+1:, J]'.
cudaError_t trsm_right_upper_t(double *X, long long ldx, int R, const double *L, long long ldl, int N,
                               void *arena_dev, cudaStream_t s) {
    if (R <= 0 || N <= 0) return cudaSuccess;
    GemmDesc *gd = (GemmDesc *)arena_dev;
    const int nblk = (N + XB - 1) / XB;
    for (int J = 0; J < nblk; ++J) {
        const int c0 = J * XB, cb = min(XB, N - c0);
        {
            KScope ks(GEO_K_SOLVE, s, (double)R * cb * cb, 8.0 * 2.0 * R * cb);
            k_trsm_right_upper_diag<<<(R + 127) / 128, 128, 0, s>>>(X, ldx, R, L, ldl, c0, cb);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int rest = N - c0 - cb;
        if (rest > 0) {
            GemmDesc g{R, rest, cb, 0, 1, X + (long long)c0 * ldx, ldx, L + (long long)c0 * ldl + c0 + cb, ldl,
                       X + (long long)(c0 + cb) * ldx, ldx, -1.0, 1.0};
            GemmDesc *d = gd + (J % 64);
            if ((e = cudaMemcpyAsync(d, &g, sizeof(g), cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
            if ((e = launch_bgemm(d, 1, ((R + 63) / 64) * ((rest + 63) / 64), s, 2.0 * R * rest * cb)) != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_transpose(const double *X, long long ldx, int R, int C, double *Y, long long ldy, cudaStream_t s) {
    if (R <= 0 || C <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    k_transpose<<<dim3((R + 31) / 32, (C + 31) / 32), dim3(32, 8), 0, s>>>(X, ldx, R, C, Y, ldy);
    return cudaGetLastError();
}

cudaError_t launch_col_sumsq(const double *Y, long long ldy, int N, int R, double *sums, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    KScope ks(GEO_K_REDUCE, s, 2.0 * N * R, 8.0 * N * R);
    k_col_sumsq<<<(R + 7) / 8, 256, 0, s>>>(Y, ldy, N, R, sums);
    return cudaGetLastError();
}

cudaError_t launch_var_finish(const double *sums, int R, int p, const double *c0diag, double *var, cudaStream_t s) {
    if (R <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    k_var_finish<<<(R + 255) / 256, 256, 0, s>>>(sums, R, p, c0diag[0], p > 1 ? c0diag[1] : 0.0,
                                                 p > 2 ? c0diag[2] : 0.0, p > 3 ? c0diag[3] : 0.0, var);
    return cudaGetLastError();
}

// V = X L (X: R x N, L lower with its diagonal blocks' upper parts zeroed
// here), by 64-column blocks: V[:, J] = X[:, J:] L[J:, J], one batched launch.
cudaError_t trmm_right_lower(const double *X, long long ldx, int R, double *L, long long ldl, int N, double *V,
                             long long ldv, void *arena_dev, void *arena_host, cudaStream_t s) {
    if (R <= 0 || N <= 0) return cudaSuccess;
    const int nblk = (N + XB - 1) / XB;
    {
        KScope ks(GEO_K_AUX, s);
        k_zero_diag_upper<<<nblk, 256, 0, s>>>(L, ldl, N);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GemmDesc *h = (GemmDesc *)arena_host;
    int tiles = 0;
    double flops = 0.0;
    for (int J = 0; J < nblk; ++J) {
        const int c0 = J * XB, cb = min(XB, N - c0);
        h[J] = GemmDesc{R, cb, N - c0, 0, 0, X + (long long)c0 * ldx, ldx, L + (long long)c0 * ldl + c0, ldl,
                        V + (long long)c0 * ldv, ldv, 1.0, 0.0};
        tiles = max(tiles, ((R + 63) / 64) * ((cb + 63) / 64));
        flops += 2.0 * R * cb * (N - c0);
    }
    GemmDesc *d = (GemmDesc *)arena_dev;
    if ((e = cudaMemcpyAsync(d, h, sizeof(GemmDesc) * nblk, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
    return launch_bgemm(d, nblk, tiles, s, flops);
}
