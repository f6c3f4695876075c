// Batched FP64 building blocks of the tile-low-rank factorisation (Sec. 5.3):
// variable-size GEMMs, Householder QR of tall-skinny blocks, one-sided Jacobi
// SVD of small square blocks, and the Gaussian test matrices of the
// randomized range finder.  Every problem of a batch is independent; each
// kernel maps one problem (or one 64 x 64 tile of it) to one CTA.
#include <math.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "geo_internal.cuh"

namespace cg = cooperative_groups;

namespace {

// ---- batched GEMM: C = alpha op(A) op(B) + beta C (column-major) ----------
// One CTA per 64 x 64 output tile of one problem, 4 x 4 outputs per thread
// (rows ty + 16 i, columns tx + 16 j).  The FP64 pipe is the limit (a few DFMA
// per clock per SM), so work on padding is the waste to avoid: a tile whose
// rows (columns) end inside it runs only the IM (JM) sixteen-row (-column)
// strips that hold outputs, and the last K slice runs only its valid depth.
// Ranks and sketch widths (the skinny side of most products here) are rarely
// multiples of 64.
constexpr int BT = 64, BKK = 16;

// K range [kbeg, kend); part == NULL: C = alpha acc + beta C, else the raw
// sums go to the tile-local partial part[(c - tn) * pw + (r - tm)].
template <int IM, int JM>
__device__ __forceinline__ void bgemm_tile(const GemmDesc &g, int tm, int tn, double (*As)[BT + 2],
                                           double (*Bs)[BT + 2], int kbeg, int kend, double *part, int pw) {
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    double acc[IM][JM];
#pragma unroll
    for (int i = 0; i < IM; ++i)
#pragma unroll
        for (int j = 0; j < JM; ++j) acc[i][j] = 0.0;
    for (int k0 = kbeg; k0 < kend; k0 += BKK) {
        // consecutive threads walk the operand's contiguous index: rows for a
        // row-contiguous slice, K for a K-contiguous one (transposed A, plain B)
        for (int t = threadIdx.x; t < BKK * 16 * IM; t += 256) {
            const int kk = g.ta ? t % BKK : t / (16 * IM), r = g.ta ? t / BKK : t % (16 * IM);
            const int kg = k0 + kk;
            double a = 0.0;
            if (kg < kend && tm + r < g.m)
                a = g.ta ? g.A[(long long)(tm + r) * g.lda + kg] : g.A[(long long)kg * g.lda + tm + r];
            As[kk][r] = a;
        }
        for (int t = threadIdx.x; t < BKK * 16 * JM; t += 256) {
            const int kk = g.tb ? t / (16 * JM) : t % BKK, r = g.tb ? t % (16 * JM) : t / BKK;
            const int kg = k0 + kk;
            double b = 0.0;
            if (kg < kend && tn + r < g.n)
                b = g.tb ? g.B[(long long)kg * g.ldb + tn + r] : g.B[(long long)(tn + r) * g.ldb + kg];
            Bs[kk][r] = b;
        }
        __syncthreads();
        const int kc = min(BKK, kend - k0);   // uniform over the CTA
        if (kc == BKK) {
#pragma unroll
            for (int kk = 0; kk < BKK; ++kk) {
                double a[IM], b[JM];
#pragma unroll
                for (int i = 0; i < IM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < JM; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < IM; ++i)
#pragma unroll
                    for (int j = 0; j < JM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        } else {
            for (int kk = 0; kk < kc; ++kk) {
                double a[IM], b[JM];
#pragma unroll
                for (int i = 0; i < IM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
                for (int j = 0; j < JM; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < IM; ++i)
#pragma unroll
                    for (int j = 0; j < JM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < JM; ++j) {
        const int c = tn + tx + 16 * j;
        if (c >= g.n) continue;
#pragma unroll
        for (int i = 0; i < IM; ++i) {
            const int r = tm + ty + 16 * i;
            if (r >= g.m) continue;
            if (part) {
                part[(c - tn) * pw + (r - tm)] = acc[i][j];
                continue;
            }
            double *p = g.C + (long long)c * g.ldc + r;
            *p = g.alpha * acc[i][j] + (g.beta == 0.0 ? 0.0 : g.beta * *p);
        }
    }
}

__global__ void __launch_bounds__(256) k_bgemm(const GemmDesc *__restrict__ d, int count) {
    __shared__ double As[BKK][BT + 2];
    __shared__ double Bs[BKK][BT + 2];
    const int pi = blockIdx.y;
    if (pi >= count) return;
    const GemmDesc g = d[pi];
    const int tiles_m = (g.m + BT - 1) / BT;
    const int tiles_n = (g.n + BT - 1) / BT;
    if ((int)blockIdx.x >= tiles_m * tiles_n) return;
    const int tm = (blockIdx.x % tiles_m) * BT, tn = (blockIdx.x / tiles_m) * BT;
    const int im = min(4, (g.m - tm + 15) / 16), jm = min(4, (g.n - tn + 15) / 16);
    switch ((im - 1) * 4 + (jm - 1)) {
#define GEO_BGEMM_CASE(I, J) \
    case (I - 1) * 4 + (J - 1): bgemm_tile<I, J>(g, tm, tn, As, Bs, 0, g.k, nullptr, 0); break;
        GEO_BGEMM_CASE(1, 1) GEO_BGEMM_CASE(1, 2) GEO_BGEMM_CASE(1, 3) GEO_BGEMM_CASE(1, 4)
        GEO_BGEMM_CASE(2, 1) GEO_BGEMM_CASE(2, 2) GEO_BGEMM_CASE(2, 3) GEO_BGEMM_CASE(2, 4)
        GEO_BGEMM_CASE(3, 1) GEO_BGEMM_CASE(3, 2) GEO_BGEMM_CASE(3, 3) GEO_BGEMM_CASE(3, 4)
        GEO_BGEMM_CASE(4, 1) GEO_BGEMM_CASE(4, 2) GEO_BGEMM_CASE(4, 3) GEO_BGEMM_CASE(4, 4)
#undef GEO_BGEMM_CASE
        default: break;
    }
}

// The same strips on 32 x 32 (S = 2) or 16 x 16 (S = 1) output tiles: for
// launches whose 64 x 64 tiles would leave most SMs idle (few output tiles,
// long K, e.g. the r x r cores V_ik' V_jk with K = nb), 4x or 16x more CTAs
// share the K loops' FP64 work.  Split-K (ws != NULL): blockIdx.z takes one of
// zsplit contiguous K ranges and writes its raw sums to its own partial tile
// ws[((pi zsplit + z) tiles_cap + tile) W^2 ..]; k_bgemm_reduce adds them.
template <int S>
__global__ void __launch_bounds__(256) k_bgemm_small(const GemmDesc *__restrict__ d, int count, int zsplit,
                                                     int tiles_cap, double *ws) {
    __shared__ double As[BKK][BT + 2];
    __shared__ double Bs[BKK][BT + 2];
    const int pi = blockIdx.y;
    if (pi >= count) return;
    const GemmDesc g = d[pi];
    constexpr int W = 16 * S;
    const int tiles_m = (g.m + W - 1) / W;
    const int tiles_n = (g.n + W - 1) / W;
    if ((int)blockIdx.x >= tiles_m * tiles_n) return;
    const int tm = (blockIdx.x % tiles_m) * W, tn = (blockIdx.x / tiles_m) * W;
    const int im = min(S, (g.m - tm + 15) / 16), jm = min(S, (g.n - tn + 15) / 16);
    int kbeg = 0, kend = g.k;
    double *part = nullptr;
    if (ws) {
        const int kc = ((g.k + zsplit - 1) / zsplit + BKK - 1) / BKK * BKK;
        kbeg = min(g.k, (int)blockIdx.z * kc);
        kend = min(g.k, kbeg + kc);
        part = ws + (((long long)pi * zsplit + blockIdx.z) * tiles_cap + blockIdx.x) * (W * W);
    }
    if (S == 1 || (im == 1 && jm == 1))
        bgemm_tile<1, 1>(g, tm, tn, As, Bs, kbeg, kend, part, W);
    else if (im == 1)
        bgemm_tile<1, S == 1 ? 1 : 2>(g, tm, tn, As, Bs, kbeg, kend, part, W);
    else if (jm == 1)
        bgemm_tile<S == 1 ? 1 : 2, 1>(g, tm, tn, As, Bs, kbeg, kend, part, W);
    else
        bgemm_tile<S == 1 ? 1 : 2, S == 1 ? 1 : 2>(g, tm, tn, As, Bs, kbeg, kend, part, W);
}

// C = alpha (sum of the zsplit partial tiles, in order) + beta C: the same
// result on every run.
template <int W>
__global__ void __launch_bounds__(256) k_bgemm_reduce(const GemmDesc *__restrict__ d, int count, int zsplit,
                                                      int tiles_cap, const double *__restrict__ ws) {
    const int pi = blockIdx.y;
    if (pi >= count) return;
    const GemmDesc g = d[pi];
    const int tiles_m = (g.m + W - 1) / W;
    const int tiles_n = (g.n + W - 1) / W;
    if ((int)blockIdx.x >= tiles_m * tiles_n) return;
    const int tm = (blockIdx.x % tiles_m) * W, tn = (blockIdx.x / tiles_m) * W;
    for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
        const int i = e % W, j = e / W;
        if (tm + i >= g.m || tn + j >= g.n) continue;
        double sum = 0.0;
        for (int z = 0; z < zsplit; ++z)
            sum += ws[(((long long)pi * zsplit + z) * tiles_cap + blockIdx.x) * (W * W) + e];
        double *p = g.C + (long long)(tn + j) * g.ldc + tm + i;
        *p = g.alpha * sum + (g.beta == 0.0 ? 0.0 : g.beta * *p);
    }
}

// ---- Householder QR of an m x r block (m >= r), in place -------------------
// Column c: v = x - alpha e1 with alpha = -sign(x_0) |x|, stored below the
// diagonal (v_0 kept in tau-scaled form), R on and above the diagonal; then
// the thin Q (m x r) is formed in Qout by applying the reflectors backwards
// to [I; 0].  One CTA (32 warps) per block; warp w updates columns w, w+32, ...
__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

constexpr int LA_THREADS = 1024, LA_WARPS = LA_THREADS / 32;

__global__ void __launch_bounds__(LA_THREADS) k_house_qr(const QrDesc *__restrict__ d, int count) {
    const int pi = blockIdx.x;
    if (pi >= count) return;
    const QrDesc q = d[pi];
    double *Y = q.Y;
    const long long ld = q.ldy;
    const int m = q.m, r = q.r;
    double *tau = q.tau;   // r entries
    __shared__ double red[LA_WARPS];
    __shared__ double s_alpha, s_tau, s_v0;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int c = 0; c < r; ++c) {
        double *x = Y + (long long)c * ld;
        // norm of x[c:m]
        double s = 0.0;
        for (int i = c + threadIdx.x; i < m; i += LA_THREADS) s += x[i] * x[i];
        s = warp_sum(s);
        if (lane == 0) red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < LA_WARPS; ++w) t += red[w];
            const double nrm = sqrt(t);
            const double x0 = x[c];
            double alpha = (x0 >= 0.0) ? -nrm : nrm;
            double v0 = x0 - alpha;
            double taue;
            if (nrm == 0.0) {
                alpha = 0.0;
                v0 = 1.0;
                taue = 0.0;
            } else {
                // H = I - tau v v' with v = (v0, x[c+1:]), tau = 2 / (v'v), v'v = 2 nrm (nrm - x0 sign...)
                const double vtv = v0 * v0 + (t - x0 * x0);
                taue = (vtv > 0.0) ? 2.0 / vtv : 0.0;
            }
            s_alpha = alpha;
            s_tau = taue;
            s_v0 = v0;
        }
        __syncthreads();
        const double v0 = s_v0, tauc = s_tau;
        // apply to columns c+1 .. r-1: y -= tau (v'y) v
        for (int j = c + 1 + warp; j < r; j += LA_WARPS) {
            double *y = Y + (long long)j * ld;
            double dot = (lane == 0) ? v0 * y[c] : 0.0;
            for (int i = c + 1 + lane; i < m; i += 32) dot += x[i] * y[i];
            dot = warp_sum(dot) * tauc;
            if (lane == 0) y[c] -= dot * v0;
            for (int i = c + 1 + lane; i < m; i += 32) y[i] -= dot * x[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            x[c] = s_alpha;   // R diagonal
            tau[c] = s_tau;
            q.v0[c] = s_v0;
        }
        __syncthreads();
    }
    // thin Q: start from [I; 0] and apply H_c for c = r-1 .. 0
    double *Q = q.Q;
    const long long ldq = q.ldq;
    for (int j = warp; j < r; j += LA_WARPS)
        for (int i = lane; i < m; i += 32) Q[(long long)j * ldq + i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    for (int c = r - 1; c >= 0; --c) {
        const double *x = Y + (long long)c * ld;
        const double v0 = q.v0[c], tauc = tau[c];
        for (int j = c + warp; j < r; j += LA_WARPS) {
            double *y = Q + (long long)j * ldq;
            double dot = (lane == 0) ? v0 * y[c] : 0.0;
            for (int i = c + 1 + lane; i < m; i += 32) dot += x[i] * y[i];
            dot = warp_sum(dot) * tauc;
            if (lane == 0) y[c] -= dot * v0;
            for (int i = c + 1 + lane; i < m; i += 32) y[i] -= dot * x[i];
        }
        __syncthreads();
    }
}

// ---- the same Householder QR on a cluster of QC CTAs ------------------------
// Rows are split over the CTAs of a cluster (the block stays in global
// memory, which L2 holds); per column c the CTAs exchange partial norms, then
// partial products v'y_j for the trailing columns, through distributed shared
// memory, every CTA forming alpha, v0, tau and the dots in rank order (so all
// take the same values), and each updates its own rows.  The thin Q is
// accumulated the same way.  r <= QR_MAX.
constexpr int QC = 8, QT = 256, QR_MAX = 256;

size_t house_qr_cl_smem(int m) {
    const int rs = (m + QC - 1) / QC;
    return sizeof(double) * ((size_t)rs + 2 * (QR_MAX + 2) + 2 * QR_MAX);
}

__global__ void __launch_bounds__(QT, 1) k_house_qr_cl(const QrDesc *__restrict__ d, int count) {
    cg::cluster_group cluster = cg::this_cluster();
    const int tile = blockIdx.x / QC;
    if (tile >= count) return;   // uniform over the cluster
    const int rank = (int)cluster.block_rank();
    const QrDesc q = d[tile];
    double *Y = q.Y;
    const long long ld = q.ldy;
    const int m = q.m, r = q.r;
    const int rs = (m + QC - 1) / QC;
    const int row0 = rank * rs, row1 = min(m, row0 + rs);
    extern __shared__ double qsm[];
    double *vloc = qsm;                       // reflector on this CTA's rows (row c holds v0)
    double *P = vloc + rs;                    // [2][QR_MAX + 2]: partial dots, then norm, x_c
    double *taus = P + 2 * (QR_MAX + 2);      // [QR_MAX]
    double *v0s = taus + QR_MAX;              // [QR_MAX]
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32, nw = QT / 32;
    int buf = 0;
    for (int c = 0; c < r; ++c) {
        double *Pb = P + buf * (QR_MAX + 2);
        const double *x = Y + (long long)c * ld;
        // (a) partial |x[c:]|^2 over this CTA's rows; the owner of row c also passes x_c
        const int i0 = max(c, row0);
        double t = 0.0;
        for (int i = i0 + threadIdx.x; i < row1; i += QT) t = fma(x[i], x[i], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        __shared__ double red[QT / 32];
        if (lane == 0) red[warp] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0;
            for (int w = 0; w < nw; ++w) a += red[w];
            Pb[QR_MAX] = a;
            Pb[QR_MAX + 1] = (c >= row0 && c < row1) ? x[c] : 0.0;
        }
        cluster.sync();
        // (b) alpha, v0, tau (the same in every CTA)
        double nrm2 = 0.0;
        for (int k = 0; k < QC; ++k) nrm2 += cluster.map_shared_rank(Pb, k)[QR_MAX];
        const double x0 = cluster.map_shared_rank(Pb, c / rs)[QR_MAX + 1];
        const double nrm = sqrt(nrm2);
        double alpha = (x0 >= 0.0) ? -nrm : nrm;
        double v0 = x0 - alpha, tauc;
        if (nrm == 0.0) {
            alpha = 0.0;
            v0 = 1.0;
            tauc = 0.0;
        } else {
            const double vtv = v0 * v0 + (nrm2 - x0 * x0);
            tauc = (vtv > 0.0) ? 2.0 / vtv : 0.0;
        }
        // the reflector on this CTA's rows
        for (int i = i0 + threadIdx.x; i < row1; i += QT) vloc[i - row0] = (i == c) ? v0 : x[i];
        __syncthreads();
        // (c) partial v'y_j for j > c: a warp per pair of columns, lanes over rows
        for (int j = c + 1 + warp; j < r; j += 2 * nw) {
            const int j2 = j + nw;
            const double *y = Y + (long long)j * ld, *y2 = Y + (long long)(j2 < r ? j2 : j) * ld;
            double dot = 0.0, dot2 = 0.0;
#pragma unroll 4
            for (int i = i0 + lane; i < row1; i += 32) {
                const double v = vloc[i - row0];
                dot = fma(v, y[i], dot);
                dot2 = fma(v, y2[i], dot2);
            }
            for (int o = 16; o > 0; o >>= 1) {
                dot += __shfl_down_sync(0xffffffffu, dot, o);
                dot2 += __shfl_down_sync(0xffffffffu, dot2, o);
            }
            if (lane == 0) {
                Pb[j] = dot;
                if (j2 < r) Pb[j2] = dot2;
            }
        }
        cluster.sync();
        // (d) y_j -= tau (v'y_j) v on this CTA's rows
        for (int j = c + 1 + warp; j < r; j += nw) {
            double dot = 0.0;
            for (int k = 0; k < QC; ++k) dot += cluster.map_shared_rank(Pb, k)[j];
            dot *= tauc;
            double *y = Y + (long long)j * ld;
            for (int i = i0 + lane; i < row1; i += 32) y[i] -= dot * vloc[i - row0];
        }
        if (threadIdx.x == 0) {
            taus[c] = tauc;
            v0s[c] = v0;
            if (c >= row0 && c < row1) {
                Y[(long long)c * ld + c] = alpha;   // R diagonal
                q.tau[c] = tauc;
                q.v0[c] = v0;
            }
        }
        __syncthreads();
        buf ^= 1;
    }
    // thin Q: [I; 0] on this CTA's rows, then H_c for c = r-1 .. 0
    double *Q = q.Q;
    const long long ldq = q.ldq;
    for (int j = warp; j < r; j += nw)
        for (int i = row0 + lane; i < row1; i += 32) Q[(long long)j * ldq + i] = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    for (int c = r - 1; c >= 0; --c) {
        double *Pb = P + buf * (QR_MAX + 2);
        const double *x = Y + (long long)c * ld;
        const int i0 = max(c, row0);
        const double v0 = v0s[c], tauc = taus[c];
        for (int j = c + warp; j < r; j += 2 * nw) {
            const int j2 = j + nw;
            const double *y = Q + (long long)j * ldq, *y2 = Q + (long long)(j2 < r ? j2 : j) * ldq;
            double dot = 0.0, dot2 = 0.0;
#pragma unroll 4
            for (int i = i0 + lane; i < row1; i += 32) {
                const double v = (i == c) ? v0 : x[i];
                dot = fma(v, y[i], dot);
                dot2 = fma(v, y2[i], dot2);
            }
            for (int o = 16; o > 0; o >>= 1) {
                dot += __shfl_down_sync(0xffffffffu, dot, o);
                dot2 += __shfl_down_sync(0xffffffffu, dot2, o);
            }
            if (lane == 0) {
                Pb[j] = dot;
                if (j2 < r) Pb[j2] = dot2;
            }
        }
        cluster.sync();
        for (int j = c + warp; j < r; j += nw) {
            double dot = 0.0;
            for (int k = 0; k < QC; ++k) dot += cluster.map_shared_rank(Pb, k)[j];
            dot *= tauc;
            double *y = Q + (long long)j * ldq;
            for (int i = i0 + lane; i < row1; i += 32) y[i] -= dot * ((i == c) ? v0 : x[i]);
        }
        __syncthreads();
        buf ^= 1;
    }
    cluster.sync();   // no CTA leaves while another still reads its shared memory
}

// ---- one-sided Jacobi SVD of an r x r block M (Hestenes) --------------------
// Rotates column pairs of M (and accumulates V) until every pair is
// orthogonal to relative 1e-13 or the sweep budget is spent (pairs whose
// columns both have norms below `skip` are not rotated); on exit the
// column norms of M are the singular values (unsorted), M = U S V' with
// U = M_col / norm.  Pairs are processed in round-robin order, r/2 disjoint
// pairs per round, one warp per pair.
__global__ void __launch_bounds__(LA_THREADS) k_jacobi_svd(const SvdDesc *__restrict__ d, int count, int max_sweeps) {
    const int pi = blockIdx.x;
    if (pi >= count) return;
    const SvdDesc s = d[pi];
    const int r = s.r;
    double *M = s.M, *V = s.V;
    const long long ld = s.ld;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    for (int j = warp; j < r; j += LA_WARPS)
        for (int i = lane; i < r; i += 32) V[(long long)j * ld + i] = (i == j) ? 1.0 : 0.0;
    __shared__ int rotated;
    const int rr = r + (r & 1);   // round-robin over an even count (index r = dummy)
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int round = 0; round < rr - 1; ++round) {
            for (int pr = warp; pr < rr / 2; pr += LA_WARPS) {
                // pairing of the circle method: position 0 fixed, others rotate
                int a = (pr == 0) ? 0 : 1 + (pr - 1 + round) % (rr - 1);
                int b = 1 + (rr - 2 - pr + round) % (rr - 1);
                if (a >= r || b >= r || a == b) continue;
                if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                double *ma = M + (long long)a * ld, *mb = M + (long long)b * ld;
                double al = 0.0, be = 0.0, ga = 0.0;
                for (int i = lane; i < r; i += 32) {
                    const double x = ma[i], y = mb[i];
                    al += x * x;
                    be += y * y;
                    ga += x * y;
                }
                al = warp_sum(al);
                be = warp_sum(be);
                ga = warp_sum(ga);
                // both columns far below the truncation threshold: they are dropped anyway,
                // and any combination of them stays below sqrt(r) * skip
                if (al < s.skip * s.skip && be < s.skip * s.skip) continue;
                if (fabs(ga) <= 1e-13 * sqrt(al * be) || ga == 0.0) continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int i = lane; i < r; i += 32) {
                    const double x = ma[i], y = mb[i];
                    ma[i] = cs * x - sn * y;
                    mb[i] = sn * x + cs * y;
                }
                double *va = V + (long long)a * ld, *vb = V + (long long)b * ld;
                for (int i = lane; i < r; i += 32) {
                    const double x = va[i], y = vb[i];
                    va[i] = cs * x - sn * y;
                    vb[i] = sn * x + cs * y;
                }
                if (lane == 0) rotated = 1;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // singular values = column norms
    for (int j = warp; j < r; j += LA_WARPS) {
        double t = 0.0;
        for (int i = lane; i < r; i += 32) t += M[(long long)j * ld + i] * M[(long long)j * ld + i];
        t = warp_sum(t);
        if (lane == 0) s.sigma[j] = sqrt(t);
    }
}

// ---- the same one-sided Jacobi SVD on a cluster of JC CTAs ------------------
// One FP64 SM needs ~13 ms per sweep at r = 232, so the SVD of a tile is
// spread over a thread-block cluster: CTA c holds rows [c rs, (c+1) rs) of M
// and V in shared memory.  Each round (r/2 disjoint pairs, the same circle
// order), two threads per pair form partial (alpha, beta, gamma) over the
// CTA's rows, the partials are exchanged through distributed shared memory
// (one cluster barrier, double-buffered), every CTA sums them in rank order
// (so every CTA takes the same rotation decisions, bit for bit) and rotates
// its own rows.  Column norms are reduced the same way at the end.  r <= 256.
constexpr int JC = 8, JT = 256, JR_MAX = 256, JLD = JR_MAX / JC + 1;

size_t jacobi_cl_smem(int r) {
    return sizeof(double) * (2 * (size_t)r * JLD + 2 * 3 * (JR_MAX / 2) + JR_MAX);
}

__global__ void __launch_bounds__(JT, 1) k_jacobi_svd_cl(const SvdDesc *__restrict__ d, int count, int max_sweeps) {
    cg::cluster_group cluster = cg::this_cluster();
    const int tile = blockIdx.x / JC;
    if (tile >= count) return;   // uniform over the cluster
    const int rank = (int)cluster.block_rank();
    extern __shared__ double sm[];
    const SvdDesc s = d[tile];
    const int r = s.r;
    const long long ld = s.ld;
    const int rs = (r + JC - 1) / JC;
    const int row0 = rank * rs, nrow = max(0, min(rs, r - row0));
    double *Ms = sm;                          // [r][JLD], rows of this CTA
    double *Vs = Ms + (size_t)r * JLD;
    double *P = Vs + (size_t)r * JLD;         // [2][3][JR_MAX / 2]
    double *nrm = P + 2 * 3 * (JR_MAX / 2);   // [JR_MAX]
    for (int e = threadIdx.x; e < r * rs; e += JT) {
        const int c = e / rs, i = e % rs;
        Ms[c * JLD + i] = (i < nrow) ? s.M[(long long)c * ld + row0 + i] : 0.0;
        Vs[c * JLD + i] = (i < nrow && row0 + i == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int rr = r + (r & 1), npairs = rr / 2;
    const int p = threadIdx.x >> 1, half = threadIdx.x & 1;
    const double skip2 = s.skip * s.skip;
    int buf = 0;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        int rotated = 0;
        for (int round = 0; round < rr - 1; ++round) {
            int a = -1, b = -1;
            double al = 0.0, be = 0.0, ga = 0.0;
            if (p < npairs) {
                a = (p == 0) ? 0 : 1 + (p - 1 + round) % (rr - 1);
                b = 1 + (rr - 2 - p + round) % (rr - 1);
                if (a >= r || b >= r || a == b) {
                    a = -1;
                } else if (a > b) {
                    const int t = a;
                    a = b;
                    b = t;
                }
                if (a >= 0)
                    for (int i = half; i < nrow; i += 2) {
                        const double x = Ms[a * JLD + i], y = Ms[b * JLD + i];
                        al = fma(x, x, al);
                        be = fma(y, y, be);
                        ga = fma(x, y, ga);
                    }
            }
            al += __shfl_xor_sync(0xffffffffu, al, 1);
            be += __shfl_xor_sync(0xffffffffu, be, 1);
            ga += __shfl_xor_sync(0xffffffffu, ga, 1);
            double *Pb = P + buf * 3 * (JR_MAX / 2);
            if (half == 0 && p < npairs) {
                Pb[p] = al;
                Pb[JR_MAX / 2 + p] = be;
                Pb[JR_MAX + p] = ga;
            }
            cluster.sync();
            if (a >= 0) {
                double A = 0.0, B = 0.0, G = 0.0;
                for (int c = 0; c < JC; ++c) {
                    const double *rp = cluster.map_shared_rank(Pb, c);
                    A += rp[p];
                    B += rp[JR_MAX / 2 + p];
                    G += rp[JR_MAX + p];
                }
                if (!(A < skip2 && B < skip2) && !(fabs(G) <= 1e-13 * sqrt(A * B) || G == 0.0)) {
                    const double zeta = (B - A) / (2.0 * G);
                    const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                    const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                    for (int i = half; i < nrow; i += 2) {
                        const double x = Ms[a * JLD + i], y = Ms[b * JLD + i];
                        Ms[a * JLD + i] = cs * x - sn * y;
                        Ms[b * JLD + i] = sn * x + cs * y;
                        const double u = Vs[a * JLD + i], v = Vs[b * JLD + i];
                        Vs[a * JLD + i] = cs * u - sn * v;
                        Vs[b * JLD + i] = sn * u + cs * v;
                    }
                    rotated = 1;
                }
            }
            __syncthreads();   // rotated columns before the next round's partials
            buf ^= 1;          // the other partial buffer: free since this round's barrier
        }
        if (!__syncthreads_or(rotated)) break;   // the same decision in every CTA
    }
    // singular values = column norms
    for (int c = threadIdx.x; c < r; c += JT) {
        double t = 0.0;
        for (int i = 0; i < nrow; ++i) t = fma(Ms[c * JLD + i], Ms[c * JLD + i], t);
        nrm[c] = t;
    }
    cluster.sync();
    if (rank == 0)
        for (int c = threadIdx.x; c < r; c += JT) {
            double t = 0.0;
            for (int q = 0; q < JC; ++q) t += cluster.map_shared_rank(nrm, q)[c];
            s.sigma[c] = sqrt(t);
        }
    for (int e = threadIdx.x; e < r * rs; e += JT) {
        const int c = e / rs, i = e % rs;
        if (i < nrow) {
            s.M[(long long)c * ld + row0 + i] = Ms[c * JLD + i];
            s.V[(long long)c * ld + row0 + i] = Vs[c * JLD + i];
        }
    }
    cluster.sync();   // no CTA leaves while another still reads its shared memory
}

// ---- Gaussian test matrices: counter-based SplitMix64 -> Box-Muller ---------
__device__ __forceinline__ unsigned long long splitmix(unsigned long long z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_gaussian(double *O, long long n, unsigned long long seed) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (n + 1) / 2) return;
    const unsigned long long h1 = splitmix(seed ^ (2ull * t)), h2 = splitmix(seed ^ (2ull * t + 1));
    const double u1 = 1.0 - (double)(h1 >> 11) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    O[2 * t] = rad * cos(6.283185307179586 * u2);
    if (2 * t + 1 < n) O[2 * t + 1] = rad * sin(6.283185307179586 * u2);
}

}  // namespace

static int device_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        n <= 0)
        return 1;
    return n;
}

thread_local double *t_splitk_ws = nullptr;
thread_local size_t t_splitk_doubles = 0;

void bgemm_splitk_scratch(double *ws, size_t bytes) {
    t_splitk_ws = ws;
    t_splitk_doubles = ws ? bytes / sizeof(double) : 0;
}

// max_tiles: the largest number of 64 x 64 output tiles of one problem.  A
// problem has at most 4x (16x) as many 32 x 32 (16 x 16) tiles; the surplus
// CTAs of the smaller-tile grids return at once.  With fewer than two CTAs
// per SM on the small tiles, a K of at least 512 and a split-K scratch
// registered on this thread, the K loop is split over up to 16 CTAs per tile.
cudaError_t launch_bgemm(const GemmDesc *d_desc, int count, int max_tiles, cudaStream_t s, double flops, int kmax) {
    if (count <= 0 || max_tiles <= 0) return cudaSuccess;
    KScope ks(GEO_K_GEMM, s, flops, 0.0);
    const long long ctas = (long long)max_tiles * count;
    const long long sms = device_sms();
    if (ctas >= sms) {
        k_bgemm<<<dim3(max_tiles, count), 256, 0, s>>>(d_desc, count);
        return cudaGetLastError();
    }
    const int S = (4 * ctas >= sms) ? 2 : 1;
    const int W = 16 * S;
    const long long tiles_cap = (long long)(64 / W) * (64 / W) * max_tiles;
    int z = 1;
    if (kmax >= 512 && t_splitk_ws && tiles_cap * count < 2 * sms) {
        const long long want = (2 * sms + tiles_cap * count - 1) / (tiles_cap * count);
        z = (int)std::min<long long>(std::min<long long>(want, 16), kmax / 128);
        while (z >= 2 && (size_t)z * count * tiles_cap * W * W > t_splitk_doubles) --z;
    }
    double *ws = z >= 2 ? t_splitk_ws : nullptr;
    if (z < 2) z = 1;
    const dim3 grid((unsigned)tiles_cap, count, z);
    if (S == 2)
        k_bgemm_small<2><<<grid, 256, 0, s>>>(d_desc, count, z, (int)tiles_cap, ws);
    else
        k_bgemm_small<1><<<grid, 256, 0, s>>>(d_desc, count, z, (int)tiles_cap, ws);
    if (ws) {
        if (S == 2)
            k_bgemm_reduce<32><<<dim3((unsigned)tiles_cap, count), 256, 0, s>>>(d_desc, count, z, (int)tiles_cap, ws);
        else
            k_bgemm_reduce<16><<<dim3((unsigned)tiles_cap, count), 256, 0, s>>>(d_desc, count, z, (int)tiles_cap, ws);
    }
    return cudaGetLastError();
}

cudaError_t launch_house_qr(const QrDesc *d_desc, int count, int mmax, int rmax, cudaStream_t s, double flops) {
    if (count <= 0) return cudaSuccess;
    KScope ks(GEO_K_TLR, s, flops, 0.0);
    if (rmax > QR_MAX) {
        k_house_qr<<<count, LA_THREADS, 0, s>>>(d_desc, count);
        return cudaGetLastError();
    }
    const size_t smem = house_qr_cl_smem(mmax);
    cudaError_t e = cudaFuncSetAttribute(k_house_qr_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)count * QC);
    cfg.blockDim = dim3(QT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = QC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_house_qr_cl, d_desc, count);
}

cudaError_t launch_jacobi_svd(const SvdDesc *d_desc, int count, int max_sweeps, int rmax, cudaStream_t s,
                              double flops) {
    if (count <= 0) return cudaSuccess;
    KScope ks(GEO_K_TLR, s, flops, 0.0);
    if (rmax > JR_MAX) {
        k_jacobi_svd<<<count, LA_THREADS, 0, s>>>(d_desc, count, max_sweeps);
        return cudaGetLastError();
    }
    const size_t smem = jacobi_cl_smem(rmax);
    cudaError_t e = cudaFuncSetAttribute(k_jacobi_svd_cl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)count * JC);
    cfg.blockDim = dim3(JT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = JC;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_jacobi_svd_cl, d_desc, count, max_sweeps);
}

cudaError_t launch_gaussian(double *O, long long n, unsigned long long seed, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    KScope ks(GEO_K_AUX, s);
    const long long pairs = (n + 1) / 2;
    k_gaussian<<<(unsigned)((pairs + 255) / 256), 256, 0, s>>>(O, n, seed);
    return cudaGetLastError();
}
