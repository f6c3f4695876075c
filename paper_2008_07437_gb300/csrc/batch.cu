// Batched evaluation of many small, uneven Eq. 1 likelihoods (dense FP64).
//
// One launch per step serves the whole batch: covariance generation, the
// right-looking Cholesky in 64-wide panels (POTRF of the diagonal block, TRSM
// of the rows below with the Z row carried along, rank-64 update of the
// trailing lower triangle), and the log-determinant / quadratic-form
// reduction.  A problem whose order is below the current panel simply has no
// work in that launch.  Every per-problem quantity (matrix pointer, order,
// theta constants, input pointers) lives in a device descriptor array, so the
// launch sequence of a batch shape (count, orders) is captured once as a CUDA
// graph and replayed with new inputs and theta by refreshing the descriptors.
// Each problem's result depends only on its own data and a fixed reduction
// order: a likelihood is bit-identical alone and inside any batch.
#include <math.h>
#include <string.h>

#include <map>
#include <mutex>
#include <vector>

#include "geo_internal.cuh"

namespace {

constexpr int PB = 64;   // panel width

struct BatchDesc {
    double *A;            // column-major, ld, N columns; row N holds Z' / y'
    long long ld;
    int N, n;
    const double *locs;   // n x 2 (caller order)
    const double *z;      // N
    CovParams cp;
    DevStatus st;         // per-problem status
    DevResults res;
};

// K_nu tables of every problem's theta: block (q, k, problem).
__global__ void __launch_bounds__(32) k_b_cheb_build(BatchDesc *d) {
    __shared__ double hv[GEO_CHEB_N];
    const CovParams &cp = d[blockIdx.z].cp;
    cheb_build_block(cp, const_cast<double *>(cp.tab), blockIdx.x, blockIdx.y, hv);
}

__global__ void __launch_bounds__(256) k_b_covgen(BatchDesc *d) {
    BatchDesc &q = d[blockIdx.z];
    const int n = q.n;
    const int l0 = blockIdx.y * 64, r0 = blockIdx.x * 4;
    if (l0 >= n || r0 >= n || r0 > l0 + 63) return;
    const int l = l0 + (threadIdx.x % 64), r = r0 + (threadIdx.x / 64);
    if (l >= n || r >= n || r > l) return;
    const double dx = q.locs[2 * l] - q.locs[2 * r], dy = q.locs[2 * l + 1] - q.locs[2 * r + 1];
    const CovParams &cp = q.cp;
    const double x = (l == r) ? 0.0 : sqrt(dx * dx + dy * dy) * cp.inv_a;
    const int p = cp.p;
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    matern_block(x, cp, v);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) q.A[(long long)(p * r + j) * q.ld + p * l + i] = v[i * GEO_PMAX_DEV + j];
}

__global__ void k_b_gather(BatchDesc *d) {
    BatchDesc &q = d[blockIdx.y];
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < q.N) q.A[(long long)k * q.ld + q.N] = q.z[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) q.st.info = 0;
}

__global__ void __launch_bounds__(256) k_b_potrf(BatchDesc *d, int c0) {
    BatchDesc &q = d[blockIdx.x];
    if (c0 >= q.N || q.st.info) return;
    const int cb = min(PB, q.N - c0);
    __shared__ double S[PB][PB + 1];
    __shared__ int fail;
    double *A = q.A;
    const long long ld = q.ld;
    for (int t = threadIdx.x; t < cb * cb; t += blockDim.x) {
        const int c = t / cb, r = t % cb;
        S[c][r] = (r >= c) ? A[(long long)(c0 + c) * ld + c0 + r] : 0.0;
    }
    if (threadIdx.x == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < cb; ++j) {
        if (threadIdx.x == 0) {
            const double v = S[j][j];
            if (!(v > 0.0)) {
                fail = 1;
                q.st.info = c0 + j + 1;
            } else {
                S[j][j] = sqrt(v);
            }
        }
        __syncthreads();
        if (fail) return;
        const double inv = 1.0 / S[j][j];
        for (int r = j + 1 + threadIdx.x; r < cb; r += blockDim.x) S[j][r] *= inv;
        __syncthreads();
        const int m = cb - j - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int c = j + 1 + t / m, r = j + 1 + t % m;
            if (r >= c) S[c][r] -= S[j][r] * S[j][c];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * cb; t += blockDim.x) {
        const int c = t / cb, r = t % cb;
        if (r >= c) A[(long long)(c0 + c) * ld + c0 + r] = S[c][r];
    }
}

// rows [c0 + cb, N] (the Z row N included) <- rows L^-T, 64 rows per CTA
__global__ void __launch_bounds__(256) k_b_trsm(BatchDesc *d, int c0) {
    BatchDesc &q = d[blockIdx.y];
    if (c0 >= q.N || q.st.info) return;
    const int cb = min(PB, q.N - c0);
    const int rbase = c0 + cb + blockIdx.x * 64;
    if (rbase > q.N) return;
    const int nr = min(64, q.N + 1 - rbase);
    __shared__ double Ls[PB][PB + 1];
    __shared__ double Xs[PB][64 + 1];
    double *A = q.A;
    const long long ld = q.ld;
    for (int t = threadIdx.x; t < cb * cb; t += 256) {
        const int c = t / cb, r = t % cb;
        Ls[c][r] = (r >= c) ? A[(long long)(c0 + c) * ld + c0 + r] : 0.0;
    }
    for (int t = threadIdx.x; t < cb * 64; t += 256) {
        const int c = t / 64, r = t % 64;
        Xs[c][r] = (r < nr) ? A[(long long)(c0 + c) * ld + rbase + r] : 0.0;
    }
    __syncthreads();
    const int row = threadIdx.x % 64, grp = threadIdx.x / 64;
    for (int c = 0; c < cb; ++c) {
        if (grp == 0) Xs[c][row] *= 1.0 / Ls[c][c];
        __syncthreads();
        const double xc = Xs[c][row];
        for (int k = c + 1 + grp; k < cb; k += 4) Xs[k][row] -= xc * Ls[c][k];
        __syncthreads();
    }
    for (int t = threadIdx.x; t < cb * 64; t += 256) {
        const int c = t / 64, r = t % 64;
        if (r < nr) A[(long long)(c0 + c) * ld + rbase + r] = Xs[c][r];
    }
}

// trailing update rows [t0, N], cols [t0, N): C -= P P', P = cols [c0, c0 + cb)
__global__ void __launch_bounds__(256) k_b_update(BatchDesc *d, int c0) {
    BatchDesc &q = d[blockIdx.z];
    if (c0 >= q.N || q.st.info) return;
    const int cb = min(PB, q.N - c0);
    const int t0 = c0 + cb;
    const int m = q.N + 1 - t0, n = q.N - t0;
    const int tm = blockIdx.x * 64, tn = blockIdx.y * 64;
    if (tm >= m || tn >= n || tm + 63 < tn) return;
    __shared__ double As[16][66];
    __shared__ double Bs[16][66];
    double *A = q.A;
    const long long ld = q.ld;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < cb; k0 += 16) {
        for (int t = threadIdx.x; t < 16 * 64; t += 256) {
            const int kk = t / 64, r = t % 64;
            const bool kin = k0 + kk < cb;
            As[kk][r] = (kin && tm + r < m) ? A[(long long)(c0 + k0 + kk) * ld + t0 + tm + r] : 0.0;
            Bs[kk][r] = (kin && tn + r < n) ? A[(long long)(c0 + k0 + kk) * ld + t0 + tn + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
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
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = tm + ty + 16 * i;
            if (r < m && r >= c) A[(long long)(t0 + c) * ld + t0 + r] -= acc[i][j];   // the Z row has r > c
        }
    }
}

__global__ void __launch_bounds__(256) k_b_reduce(BatchDesc *d) {
    BatchDesc &q = d[blockIdx.x];
    __shared__ double s1[8], s2[8];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < q.N; k += 256) {
        a += log(q.A[(long long)k * q.ld + k]);
        const double v = q.A[(long long)k * q.ld + q.N];
        b += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) s1[threadIdx.x >> 5] = a, s2[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int w = 0; w < 8; ++w) ta += s1[w], tb += s2[w];
        if (q.st.info) {
            q.res.loglik = q.res.logdet = q.res.quad = nan("");
        } else {
            q.res.logdet = 2.0 * ta;
            q.res.quad = tb;
            q.res.loglik = -0.5 * (double)q.N * log(2.0 * 3.141592653589793) - 0.5 * q.res.logdet - 0.5 * tb;
        }
    }
}

}  // namespace

size_t batch_desc_bytes() { return sizeof(BatchDesc); }

// Builds the descriptors on the host (pinned staging `hdesc`), the launch
// sequence is recorded on `s` (capturable).
struct BatchPlan {
    int count = 0, nmax = 0, Nmax = 0;
};

void batch_fill_desc(void *hdesc_v, int k, double *A, long long ld, int N, int n, const double *locs,
                     const double *z, const CovParams &cp) {
    BatchDesc *h = (BatchDesc *)hdesc_v;
    memset(&h[k], 0, sizeof(BatchDesc));
    h[k].A = A;
    h[k].ld = ld;
    h[k].N = N;
    h[k].n = n;
    h[k].locs = locs;
    h[k].z = z;
    h[k].cp = cp;
}

cudaError_t batch_record(void *ddesc_v, int count, int nmax, int Nmax, cudaStream_t s) {
    BatchDesc *d = (BatchDesc *)ddesc_v;
    {
        KScope ks(GEO_K_COVGEN, s);
        k_b_cheb_build<<<dim3(GEO_PMAX_DEV * GEO_PMAX_DEV, GEO_CHEB_NI + 1, count), 32, 0, s>>>(d);
    }
    {
        KScope ks(GEO_K_COVGEN, s);
        dim3 grid((nmax + 3) / 4, (nmax + 63) / 64, count);
        k_b_covgen<<<grid, 256, 0, s>>>(d);
    }
    {
        KScope ks(GEO_K_AUX, s);
        k_b_gather<<<dim3((Nmax + 255) / 256, count), 256, 0, s>>>(d);
    }
    for (int c0 = 0; c0 < Nmax; c0 += PB) {
        {
            KScope ks(GEO_K_POTRF, s);
            k_b_potrf<<<count, 256, 0, s>>>(d, c0);
        }
        // rows below the panel, the Z row included (the last panel of a problem may be partial)
        const int rows = Nmax + 1 - (c0 + 1);
        if (rows > 0) {
            KScope ks(GEO_K_TRSM, s);
            k_b_trsm<<<dim3((rows + 63) / 64, count), 256, 0, s>>>(d, c0);
        }
        const int m = Nmax + 1 - (c0 + PB);
        if (m > 0) {
            KScope ks(GEO_K_GEMM, s);
            k_b_update<<<dim3((m + 63) / 64, (m + 63) / 64, count), 256, 0, s>>>(d, c0);
        }
    }
    {
        KScope ks(GEO_K_REDUCE, s);
        k_b_reduce<<<count, 256, 0, s>>>(d);
    }
    return cudaGetLastError();
}

// Results out of the device descriptors into host arrays (after the stream syncs).
cudaError_t batch_results(const void *ddesc_v, void *hdesc_v, int count, double *loglik, int *info, cudaStream_t s) {
    const BatchDesc *d = (const BatchDesc *)ddesc_v;
    BatchDesc *h = (BatchDesc *)hdesc_v;
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(BatchDesc) * count, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    for (int k = 0; k < count; ++k) {
        if (loglik) loglik[k] = h[k].res.loglik;
        if (info) info[k] = h[k].st.info;
    }
    return cudaSuccess;
}
