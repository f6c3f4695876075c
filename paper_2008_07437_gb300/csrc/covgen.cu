// Covariance generation (Eq. 2, Sec. 4.2) in Representation I (Sec. 5.2),
// and the fused cokriging predictor (Eq. 3 / Eq. 4, Sec. 4.3).
//
// Every matrix entry is one FP64 evaluation of Eq. 2: the work is FP64 ALU
// bound (Bessel K_nu), so the kernels map one location pair to one thread,
// evaluate the p(p+1)/2 distinct C_ij once per pair, and write the p x p block
// with column-major stores that are contiguous across a warp.
#include "geo_internal.cuh"

namespace {

constexpr int TL = 64;   // locations l (rows) per CTA
constexpr int TR = 4;    // locations r (columns) per CTA

// The p x p block of C at distance h for one location pair.
__device__ __forceinline__ void cov_block(const CovParams &cp, double h, double *v) {
    matern_block(h * cp.inv_a, cp, v);
}

// K_nu tables of one theta (cheb_build_block, matern.cuh): block (q, k).
__global__ void __launch_bounds__(32) k_cheb_build(const CovParams cp, double *tab) {
    __shared__ double hv[GEO_CHEB_N];
    cheb_build_block(cp, tab, blockIdx.x, blockIdx.y, hv);
}

// Lower triangle (location blocks l >= r) of Sigma, column-major A[c*ld + r].
__global__ void __launch_bounds__(TL *TR) k_covgen_sym(const CovParams cp, const double *__restrict__ lx,
                                                       const double *__restrict__ ly, int n, double *A,
                                                       long long ld) {
    const int l0 = blockIdx.y * TL, r0 = blockIdx.x * TR;
    if (r0 > l0 + TL - 1) return;   // tile entirely above the location diagonal
    const int l = l0 + (threadIdx.x % TL);
    const int r = r0 + (threadIdx.x / TL);
    if (l >= n || r >= n || r > l) return;
    const double dx = lx[l] - lx[r], dy = ly[l] - ly[r];
    const double h = sqrt(dx * dx + dy * dy);
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    cov_block(cp, (l == r) ? 0.0 : h, v);
    const int p = cp.p;
    for (int j = 0; j < p; ++j) {
        double *col = A + (long long)(p * r + j) * ld + (long long)p * l;
        for (int i = 0; i < p; ++i) col[i] = v[i * GEO_PMAX_DEV + j];
    }
}

// Full rectangle: rows p*n1 (locations l of set 1), cols p*n2 (set 2); AoS inputs.
__global__ void __launch_bounds__(TL *TR) k_covgen_rect(const CovParams cp, const double *__restrict__ l1, int n1,
                                                        const double *__restrict__ l2, int n2, double *out,
                                                        long long ld) {
    const int l = blockIdx.y * TL + (threadIdx.x % TL);
    const int r = blockIdx.x * TR + (threadIdx.x / TL);
    if (l >= n1 || r >= n2) return;
    const double dx = l1[2 * l] - l2[2 * r], dy = l1[2 * l + 1] - l2[2 * r + 1];
    const double h = sqrt(dx * dx + dy * dy);
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    cov_block(cp, h, v);
    const int p = cp.p;
    for (int j = 0; j < p; ++j) {
        double *col = out + (long long)(p * r + j) * ld + (long long)p * l;
        for (int i = 0; i < p; ++i) col[i] = v[i * GEO_PMAX_DEV + j];
    }
}

// One CTA per prediction location: zhat_i(s0) = sum_r sum_j C_ij(|s0 - s_r|) w_(p r + j).
// Fixed thread-to-r assignment and a fixed reduction tree: the result does not
// depend on timing.
constexpr int PRED_THREADS = 256;

__global__ void __launch_bounds__(PRED_THREADS) k_predict(const CovParams cp, const double *__restrict__ s0,
                                                          const double *__restrict__ lx,
                                                          const double *__restrict__ ly, int n,
                                                          const double *__restrict__ w, double *zhat) {
    const int l = blockIdx.x;
    const double x0 = s0[2 * l], y0 = s0[2 * l + 1];
    const int p = cp.p;
    double acc[GEO_PMAX_DEV] = {0.0, 0.0, 0.0, 0.0};
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    for (int r = threadIdx.x; r < n; r += PRED_THREADS) {
        const double dx = x0 - lx[r], dy = y0 - ly[r];
        cov_block(cp, sqrt(dx * dx + dy * dy), v);
        for (int i = 0; i < p; ++i) {
            double t = 0.0;
            for (int j = 0; j < p; ++j) t += v[i * GEO_PMAX_DEV + j] * w[(long long)p * r + j];
            acc[i] += t;
        }
    }
    __shared__ double red[GEO_PMAX_DEV][PRED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = 0; i < p; ++i) {
        double t = acc[i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[i][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < p) {
        double t = 0.0;
        for (int k = 0; k < PRED_THREADS / 32; ++k) t += red[threadIdx.x][k];
        zhat[(long long)p * l + threadIdx.x] = t;
    }
}

__global__ void k_gather_locs(const double *__restrict__ locs, const int *__restrict__ perm, int n, double *lx,
                              double *ly) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int s = perm ? perm[k] : k;
    lx[k] = locs[2 * (long long)s];
    ly[k] = locs[2 * (long long)s + 1];
}

__global__ void k_gather_vec(const double *__restrict__ in, const int *__restrict__ perm, int n, int p,
                             double *out, long long stride) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * p) return;
    const int k = (int)(t / p), i = (int)(t % p);
    const int s = perm ? perm[k] : k;
    out[t * stride] = in[(long long)p * s + i];
}

__global__ void k_scatter_vec(const double *__restrict__ in, long long stride, const int *__restrict__ perm, int n,
                              int p, double *out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)n * p) return;
    const int k = (int)(t / p), i = (int)(t % p);
    const int s = perm ? perm[k] : k;
    out[(long long)p * s + i] = in[t * stride];
}

}  // namespace

bool cov_needs_tables(const CovParams &cp) {
    for (int q = 0; q < cp.p * cp.p; ++q)
        if (cp.m[q].kind == 0 && cp.m[q].toff >= 0) return true;
    return false;
}

cudaError_t launch_cheb_build(CovParams &cp, double *tab, cudaStream_t s) {
    cp.tab = tab;
    if (!cov_needs_tables(cp)) return cudaSuccess;
    if (!tab) return cudaErrorInvalidValue;
    KScope ks(GEO_K_COVGEN, s);
    k_cheb_build<<<dim3(cp.p * cp.p, GEO_CHEB_NI + 1), 32, 0, s>>>(cp, tab);
    return cudaGetLastError();
}

cudaError_t launch_covgen_sym(const CovParams &cp, const double *lx, const double *ly, int n, double *A,
                              long long ld, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    dim3 grid((n + TR - 1) / TR, (n + TL - 1) / TL);
    const double N = (double)cp.p * n;
    KScope ks(GEO_K_COVGEN, s, 0.0, 8.0 * N * (N + cp.p) / 2.0);   // bytes: lower triangle written once
    k_covgen_sym<<<grid, TL * TR, 0, s>>>(cp, lx, ly, n, A, ld);
    return cudaGetLastError();
}

cudaError_t launch_covgen_rect(const CovParams &cp, const double *l1, int n1, const double *l2, int n2,
                               double *out, long long ld, cudaStream_t s) {
    if (n1 <= 0 || n2 <= 0) return cudaSuccess;
    dim3 grid((n2 + TR - 1) / TR, (n1 + TL - 1) / TL);
    KScope ks(GEO_K_COVGEN, s, 0.0, 8.0 * cp.p * (double)n1 * cp.p * (double)n2);
    k_covgen_rect<<<grid, TL * TR, 0, s>>>(cp, l1, n1, l2, n2, out, ld);
    return cudaGetLastError();
}

// Batched predictions: CTA g serves the new location g of the concatenation of
// every entry's locations; it finds its entry by binary search over the
// entries' first indices, copies the entry's theta constants into shared
// memory and computes exactly what k_predict computes for that location (same
// thread-to-r assignment, same reduction tree): bit-identical to one call per
// factor.
__global__ void __launch_bounds__(PRED_THREADS) k_predict_batch(const PredDesc *__restrict__ d, int count) {
    __shared__ CovParams cps;
    __shared__ int ent;
    const int g = blockIdx.x;
    if (threadIdx.x == 0) {
        int lo = 0, hi = count - 1;   // the last entry with first <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (d[mid].first <= g) lo = mid;
            else hi = mid - 1;
        }
        ent = lo;
    }
    __syncthreads();
    const PredDesc &q = d[ent];
    {
        const int words = (int)(sizeof(CovParams) / sizeof(int));
        const int *src = reinterpret_cast<const int *>(&q.cp);
        int *dst = reinterpret_cast<int *>(&cps);
        for (int t = threadIdx.x; t < words; t += PRED_THREADS) dst[t] = src[t];
    }
    __syncthreads();
    const CovParams &cp = cps;
    const int l = g - q.first, n = q.n;
    const double *lx = q.lx, *ly = q.ly, *w = q.w;
    const double x0 = q.s0[2 * l], y0 = q.s0[2 * l + 1];
    const int p = cp.p;
    double acc[GEO_PMAX_DEV] = {0.0, 0.0, 0.0, 0.0};
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    for (int r = threadIdx.x; r < n; r += PRED_THREADS) {
        const double dx = x0 - lx[r], dy = y0 - ly[r];
        cov_block(cp, sqrt(dx * dx + dy * dy), v);
        for (int i = 0; i < p; ++i) {
            double t = 0.0;
            for (int j = 0; j < p; ++j) t += v[i * GEO_PMAX_DEV + j] * w[(long long)p * r + j];
            acc[i] += t;
        }
    }
    __shared__ double red[GEO_PMAX_DEV][PRED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = 0; i < p; ++i) {
        double t = acc[i];
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[i][wid] = t;
    }
    __syncthreads();
    if (threadIdx.x < p) {
        double t = 0.0;
        for (int k = 0; k < PRED_THREADS / 32; ++k) t += red[threadIdx.x][k];
        q.zhat[(long long)p * l + threadIdx.x] = t;
    }
}

cudaError_t launch_predict(const CovParams &cp, const double *new_locs, int m, const double *lx,
                           const double *ly, int n, const double *w, double *zhat, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    KScope ks(GEO_K_PREDICT, s, 2.0 * cp.p * (double)m * cp.p * (double)n, 16.0 * n + 24.0 * m);
    k_predict<<<m, PRED_THREADS, 0, s>>>(cp, new_locs, lx, ly, n, w, zhat);
    return cudaGetLastError();
}

cudaError_t launch_gather_locs(const double *locs, const int *perm, int n, double *lx, double *ly,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    k_gather_locs<<<(n + 255) / 256, 256, 0, s>>>(locs, perm, n, lx, ly);
    return cudaGetLastError();
}

cudaError_t launch_gather_vec(const double *in, const int *perm, int n, int p, double *out, long long stride,
                              cudaStream_t s) {
    const long long t = (long long)n * p;
    if (t <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    k_gather_vec<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(in, perm, n, p, out, stride);
    return cudaGetLastError();
}

cudaError_t launch_scatter_vec(const double *in, long long stride, const int *perm, int n, int p, double *out,
                               cudaStream_t s) {
    const long long t = (long long)n * p;
    if (t <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    k_scatter_vec<<<(unsigned)((t + 255) / 256), 256, 0, s>>>(in, stride, perm, n, p, out);
    return cudaGetLastError();
}

cudaError_t launch_predict_batch(const PredDesc *d, int count, int total, double flops, cudaStream_t s) {
    if (total <= 0) return cudaSuccess;
    KScope ks(GEO_K_PREDICT, s, flops, 0.0);
    k_predict_batch<<<total, PRED_THREADS, 0, s>>>(d, count);
    return cudaGetLastError();
}
