// FP64 iterative refinement of Sigma x = Z for the mixed-precision factor
// (Eq. 1 needs Z' Sigma^-1 Z; the reduced-precision factor L~ serves as the
// preconditioner and the residual is formed in FP64 from a stored copy of
// the lower triangle of Sigma):
//   x_0 = L~^-T L~^-1 Z,   x_{k+1} = x_k + L~^-T L~^-1 (Z - Sigma x_k).
// Then Z' Sigma^-1 Z = Z' x, and the cokriging weights of Eq. 3 are x.
// log|Sigma| is taken from the diagonal of L~ (FP64 diagonal tiles).
//
// Kernels: the one-launch triangular solves of trsv.cu, a symmetric
// matrix-vector product from the lower triangle in 256 x 256 tiles
// with per-tile partial sums reduced in a fixed order (deterministic), and
// small FP64 vector kernels.  All HBM-bound: each pass streams the lower
// triangle once.
#include "geo_internal.cuh"

namespace {

constexpr int ST = 256;   // symv tile

// Partial sums of y = S x from the lower triangle of S, tile (I, J), I >= J:
//   prow[J][r] = sum_{c in J} S[r, c] x[c] (c <= r on the diagonal tile),
//   pcol[I][c] = sum_{r in I} S[r, c] x[r] (strictly below the diagonal).
__global__ void __launch_bounds__(256) k_symv_tiles(const double *__restrict__ S, long long ld, int N,
                                                   const double *__restrict__ x, double *prow, double *pcol) {
    const int I = blockIdx.y, J = blockIdx.x;
    if (J > I) return;
    const int r0 = I * ST, c0 = J * ST;
    __shared__ double xr[ST], xc[ST];
    __shared__ double colacc[ST];
    const int tid = threadIdx.x;
    xr[tid] = (r0 + tid < N) ? x[r0 + tid] : 0.0;
    xc[tid] = (c0 + tid < N) ? x[c0 + tid] : 0.0;
    __syncthreads();
    // row sums: thread = row, loop over the tile's columns (coalesced per column)
    const int r = r0 + tid;
    double rs = 0.0;
    if (r < N) {
        const int cend = min(ST, N - c0);
        for (int cc = 0; cc < cend; ++cc) {
            const int c = c0 + cc;
            if (I == J && c > r) break;
            rs += S[(long long)c * ld + r] * xc[cc];
        }
    }
    if (r < N) prow[(long long)J * N + r] = rs;
    // column sums: warp w takes columns c = w, w + 8, ...; lanes stride rows
    const int warp = tid / 32, lane = tid % 32;
    for (int cc = warp; cc < ST; cc += 8) {
        const int c = c0 + cc;
        double t = 0.0;
        if (c < N) {
            for (int rr = lane; rr < ST; rr += 32) {
                const int rg = r0 + rr;
                if (rg >= N) break;
                if (I == J && rg <= c) continue;
                t += S[(long long)c * ld + rg] * xr[rr];
            }
        }
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) colacc[cc] = t;
    }
    __syncthreads();
    if (c0 + tid < N) pcol[(long long)I * N + c0 + tid] = colacc[tid];
}

// y[r] = sum_J prow[J][r] + sum_I pcol[I][r] over the tiles that touch r (fixed order).
__global__ void k_symv_reduce(const double *prow, const double *pcol, int N, int T, double *y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= N) return;
    const int R = r / ST;
    double t = 0.0;
    for (int J = 0; J <= R; ++J) t += prow[(long long)J * N + r];
    for (int I = R; I < T; ++I) t += pcol[(long long)I * N + r];   // I == R: the diagonal tile, rows below r
    (void)T;
    y[r] = t;
}

// r = z - y
__global__ void k_residual(const double *z, const double *y, int N, double *r) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) r[k] = z[k] - y[k];
}

// x += d
__global__ void k_axpy1(double *x, const double *d, int N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) x[k] += d[k];
}

// logdet from the diagonal of L, quad = z' x, loglik (Eq. 1); one CTA, fixed order.
__global__ void __launch_bounds__(1024) k_ir_reduce(const double *__restrict__ A, long long ld, int N,
                                                   const double *__restrict__ z, const double *__restrict__ x,
                                                   const DevStatus *st, DevResults *res) {
    __shared__ double s1[32], s2[32];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < N; k += 1024) {
        a += log(A[(long long)k * ld + k]);
        b += z[k] * x[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s1[threadIdx.x >> 5] = a;
        s2[threadIdx.x >> 5] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 32; ++w) ta += s1[w], tb += s2[w];
        if (st->info) {
            res->loglik = res->logdet = res->quad = nan("");
        } else {
            res->logdet = 2.0 * ta;
            res->quad = tb;
            res->loglik = -0.5 * (double)N * log(2.0 * 3.141592653589793) - 0.5 * res->logdet - 0.5 * tb;
        }
    }
}

}  // namespace

size_t refine_workspace_bytes(int N) {
    const size_t T = ((size_t)N + ST - 1) / ST;
    return sizeof(double) * (2 * T * (size_t)N + 4 * (size_t)N) + 1024 + 64;   // + the solves' sync words
}

// x = Sigma^-1 z by iterative refinement; S = lower triangle of Sigma (copy),
// L~ = mixed factor (both column-major, ld), y = L~^-1 z (strided row).
cudaError_t refine_solve(const double *S, const double *A, long long ld, int N, const double *z, const double *y,
                         long long ystride, int iters, double *x, void *ws, const DevStatus *st, DevResults *res,
                         cudaStream_t s) {
    const int T = (N + ST - 1) / ST;
    double *prow = (double *)ws;
    double *pcol = prow + (size_t)T * N;
    double *sy = pcol + (size_t)T * N;
    double *r = sy + N;
    int *sync = (int *)(r + N);
    int *tw = const_cast<int *>(&st->timeout);
    cudaError_t e = backward_solve(A, ld, N, y, ystride, x, sync, tw, s);
    if (e != cudaSuccess) return e;
    for (int it = 0; it < iters; ++it) {
        {
            KScope ks(GEO_K_SOLVE, s, 1.0 * N * N, 8.0 * (double)N * N / 2.0);
            k_symv_tiles<<<dim3(T, T), 256, 0, s>>>(S, ld, N, x, prow, pcol);
            k_symv_reduce<<<(N + 255) / 256, 256, 0, s>>>(prow, pcol, N, T, sy);
            k_residual<<<(N + 255) / 256, 256, 0, s>>>(z, sy, N, r);
        }
        if ((e = forward_solve(A, ld, N, r, sync, tw, s)) != cudaSuccess) return e;
        if ((e = backward_solve(A, ld, N, r, 1, r, sync, tw, s)) != cudaSuccess) return e;
        {
            KScope ks(GEO_K_AUX, s);
            k_axpy1<<<(N + 255) / 256, 256, 0, s>>>(x, r, N);
        }
    }
    KScope ks(GEO_K_REDUCE, s, 3.0 * N, 24.0 * N);
    k_ir_reduce<<<1, 1024, 0, s>>>(A, ld, N, z, x, st, res);
    return cudaGetLastError();
}
