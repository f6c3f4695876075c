// Triangular solves and the reductions of Eq. 1 (Sec. 1).
//
// * log|Sigma| = 2 sum_k log L_kk and Z' Sigma^-1 Z = y'y with y = L^-1 Z
//   (y comes out of the factorisation as an extra row), reduced in FP64 by
//   one CTA in a fixed order, so the value does not depend on timing.
// * w = L^-T y for the cokriging weights of Eq. 3: blocked backward
//   substitution, 64 x 64 diagonal solves in one CTA, and the update of the
//   remaining right-hand side by warps that each read one column segment of
//   L (contiguous in the column-major layout).
// * z = L e for the synthetic draws.
// These kernels stream L once: they are HBM-bound.
#include <math.h>

#include "geo_internal.cuh"

namespace {

constexpr int RED_THREADS = 1024;

__global__ void __launch_bounds__(RED_THREADS) k_loglik_reduce(const double *__restrict__ A, long long ld, int N,
                                                                const double *__restrict__ y, long long ystride,
                                                                const DevStatus *st, DevResults *res) {
    __shared__ double s1[RED_THREADS / 32], s2[RED_THREADS / 32];
    double ld_acc = 0.0, q_acc = 0.0;
    for (int k = threadIdx.x; k < N; k += RED_THREADS) {
        ld_acc += log(A[(long long)k * ld + k]);
        const double v = y[(long long)k * ystride];
        q_acc += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ld_acc += __shfl_down_sync(0xffffffffu, ld_acc, o);
        q_acc += __shfl_down_sync(0xffffffffu, q_acc, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        s1[wid] = ld_acc;
        s2[wid] = q_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < RED_THREADS / 32; ++w) {
            a += s1[w];
            b += s2[w];
        }
        const double logdet = 2.0 * a;
        if (st->info) {
            res->loglik = res->logdet = res->quad = nan("");
        } else {
            res->logdet = logdet;
            res->quad = b;
            res->loglik = -0.5 * (double)N * log(2.0 * 3.141592653589793) - 0.5 * logdet - 0.5 * b;
        }
    }
}

// z[i] = sum_{k <= i} L[i, k] e[k]; one thread per row, columns in chunks staged in shared memory.
__global__ void __launch_bounds__(256) k_trmv_lower(const double *__restrict__ A, long long ld, int N,
                                                   const double *__restrict__ e, double *z) {
    __shared__ double es[256];
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int imax = min(N - 1, blockIdx.x * 256 + 255);
    double t = 0.0;
    for (int k0 = 0; k0 <= imax; k0 += 256) {
        __syncthreads();
        es[threadIdx.x] = (k0 + threadIdx.x < N) ? e[k0 + threadIdx.x] : 0.0;
        __syncthreads();
        if (i < N) {
            const int kend = min(256, i - k0 + 1);
            for (int kk = 0; kk < kend; ++kk) t += A[(long long)(k0 + kk) * ld + i] * es[kk];
        }
    }
    if (i < N) z[i] = t;
}

}  // namespace

cudaError_t launch_loglik_reduce(const double *A, long long ld, int N, const double *y, long long ystride,
                                 const DevStatus *st, DevResults *res, cudaStream_t s) {
    KScope ks(GEO_K_REDUCE, s, 3.0 * N, 16.0 * N);
    k_loglik_reduce<<<1, RED_THREADS, 0, s>>>(A, ld, N, y, ystride, st, res);
    return cudaGetLastError();
}

cudaError_t launch_trmv_lower(const double *A, long long ld, int N, const double *e, double *z, cudaStream_t s) {
    if (N <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s, (double)N * N, 4.0 * (double)N * N);
    k_trmv_lower<<<(N + 255) / 256, 256, 0, s>>>(A, ld, N, e, z);
    return cudaGetLastError();
}
