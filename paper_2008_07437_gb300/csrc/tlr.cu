// Tile-low-rank (TLR) Cholesky factorisation (Sec. 5.3): diagonal tiles
// dense, every off-diagonal tile of the factor held as U V' with a rank
// chosen so that the dropped singular values of the tile lie below an
// absolute accuracy tol (at most kmax; Fig. 5 / TLR5-9 accuracy levels).
//
// Schedule (left-looking over tile columns j, one GPU):
//   1. regenerate the dense column panel W = Sigma[j.., j] from Eq. 2 (covgen);
//   2. apply the updates of the finished columns k < j in low-rank form:
//        W_ij -= sum_k U_ik (V_ik' V_jk) U_jk'
//      as batched FP64 GEMMs (cores M = V_ik' V_jk, P_i = [U_ik M], then one
//      W_i -= P_i [U_jk]' per tile, in chunks of the stacked rank);
//   3. factor the diagonal tile in FP64 (the dense POTRF of the tile algorithm);
//   4. compress each W_ij, i > j, by a randomized SVD: Y = W Omega (Gaussian
//      sketch), Q = qr(Y), B' = W' Q, Q2 R2 = qr(B'), R2' = X S Yj' (one-sided
//      Jacobi), keep the singular values above tol: U = Q X S, V = Q2 Yj; a tile
//      whose sketch is too narrow is redone with the widest sketch;
//   5. V_ij <- L_jj^-1 V_ij (the TRSM of the tile algorithm on the V factor only).
// The paper's own TLR kernels (HiCMA) update in low-rank form and recompress
// after every product; regenerating and updating the dense panel keeps every
// heavy step a plain GEMM and compresses each tile once, at its final value.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "geo_internal.cuh"

namespace {

// Sigma block: rows = locations [l0, l0 + nl), cols = locations [r0, r0 + nr), SoA locations, Rep. I.
__global__ void __launch_bounds__(256) k_covgen_block(const CovParams cp, const double *__restrict__ lx,
                                                     const double *__restrict__ ly, int l0, int nl, int r0, int nr,
                                                     double *out, long long ld) {
    const int l = l0 + blockIdx.y * 64 + (threadIdx.x % 64);
    const int r = r0 + blockIdx.x * 4 + (threadIdx.x / 64);
    if (l >= l0 + nl || r >= r0 + nr) return;
    const double dx = lx[l] - lx[r], dy = ly[l] - ly[r];
    const double x = (l == r) ? 0.0 : sqrt(dx * dx + dy * dy) * cp.inv_a;
    const int p = cp.p;
    double v[GEO_PMAX_DEV * GEO_PMAX_DEV];
    matern_block(x, cp, v);
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) out[(long long)(p * (r - r0) + j) * ld + p * (l - l0) + i] = v[i * GEO_PMAX_DEV + j];
}

// M (r x r) = transpose of the upper triangle of B (r x r leading block, ld ldb).
__global__ void k_copy_r2t(const TlrR2Desc *__restrict__ d, int count) {
    if ((int)blockIdx.y >= count) return;
    const TlrR2Desc q = d[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= q.r * q.r) return;
    const int c = t / q.r, rr = t % q.r;   // M[rr, c] = B[c, rr] if c <= rr
    q.M[(long long)c * q.ldm + rr] = (c <= rr) ? q.B[(long long)rr * q.ldb + c] : 0.0;
}

// Gather the selected columns: Msel[:, c] = M[:, sel[c]], Vsel[:, c] = Vj[:, sel[c]].
__global__ void k_gather_sel(const TlrSelDesc *__restrict__ d, int count) {
    if ((int)blockIdx.y >= count) return;
    const TlrSelDesc q = d[blockIdx.y];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= q.r * q.k) return;
    const int c = t / q.r, rr = t % q.r;
    const int src = q.sel[c];
    q.Msel[(long long)c * q.ld + rr] = q.M[(long long)src * q.ld + rr];
    q.Vsel[(long long)c * q.ld + rr] = q.Vj[(long long)src * q.ld + rr];
}

// Left lower triangular solve on a 64-row block: X = L[c0:c0+cb, c0:c0+cb]^-1 X, for
// 64 columns of one problem per CTA (blockIdx.x = column chunk, blockIdx.y = problem).
__global__ void __launch_bounds__(256) k_trsm_left_diag(const TlrTrsmDesc *__restrict__ d, int count, int c0,
                                                       int cb) {
    if ((int)blockIdx.y >= count) return;
    const TlrTrsmDesc q = d[blockIdx.y];
    const int col0 = blockIdx.x * 64;
    if (col0 >= q.ncols) return;
    const int nc = min(64, q.ncols - col0);
    __shared__ double Ls[64][65];   // Ls[c][r] = L[c0 + r, c0 + c]
    __shared__ double Xs[64][65];   // Xs[c][r] = X[c0 + r, col0 + c]
    for (int t = threadIdx.x; t < cb * cb; t += 256) {
        const int c = t / cb, r = t % cb;
        Ls[c][r] = q.L[(long long)(c0 + c) * q.ldl + c0 + r];
    }
    for (int t = threadIdx.x; t < nc * cb; t += 256) {
        const int c = t / cb, r = t % cb;
        Xs[c][r] = q.X[(long long)(col0 + c) * q.ldx + c0 + r];
    }
    __syncthreads();
    // column-parallel forward substitution: thread (c, part) owns column c
    const int c = threadIdx.x % 64, part = threadIdx.x / 64;
    for (int r = 0; r < cb; ++r) {
        if (part == 0 && c < nc) Xs[c][r] /= Ls[r][r];
        __syncthreads();
        if (c < nc) {
            const double xr = Xs[c][r];
            for (int rr = r + 1 + part; rr < cb; rr += 4) Xs[c][rr] -= Ls[r][rr] * xr;
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < nc * cb; t += 256) {
        const int c2 = t / cb, r = t % cb;
        q.X[(long long)(col0 + c2) * q.ldx + c0 + r] = Xs[c2][r];
    }
}

// V = I (m x m, ld ld)
__global__ void k_identity(double *V, long long ld, int m) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= ld * m) return;
    const long long c = t / ld, r = t % ld;
    V[t] = (r == c) ? 1.0 : 0.0;
}

// r -= sum_c buf[:, c] (c < ncols) for m entries (fixed order)
__global__ void k_sub_cols(double *r, const double *buf, long long ldb, int m, int ncols) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double t = 0.0;
    for (int c = 0; c < ncols; ++c) t += buf[(long long)c * ldb + i];
    r[i] -= t;
}

// logdet over the diagonal tiles, y'y, Eq. 1
__global__ void __launch_bounds__(1024) k_tlr_reduce(const double *D, int nb, int T, int N, const double *y,
                                                    const DevStatus *st, DevResults *res) {
    __shared__ double s1[32], s2[32];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < N; k += 1024) {
        const int t = k / nb, o = k % nb;
        a += log(D[(long long)t * nb * nb + (long long)o * nb + o]);
        b += y[k] * y[k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) s1[threadIdx.x >> 5] = a, s2[threadIdx.x >> 5] = b;
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
    (void)T;
}

// ---- descriptor arenas (host pinned staging -> device), reset at sync points ----
struct Arena {
    uint8_t *host = nullptr, *dev = nullptr;
    size_t cap = 0, used = 0;
};

template <typename T>
T *push(Arena &a, const std::vector<T> &v, cudaStream_t s, cudaError_t *err) {
    const size_t bytes = sizeof(T) * v.size();
    const size_t off = (a.used + 255) & ~(size_t)255;
    if (off + bytes > a.cap) {
        // the arena is reset only at stream synchronisation points between columns
        *err = cudaErrorMemoryAllocation;
        return nullptr;
    }
    memcpy(a.host + off, v.data(), bytes);
    *err = cudaMemcpyAsync(a.dev + off, a.host + off, bytes, cudaMemcpyHostToDevice, s);
    a.used = off + bytes;
    return (T *)(a.dev + off);
}

int gemm_tiles(const std::vector<GemmDesc> &v) {
    int mx = 0;
    for (const GemmDesc &g : v) mx = std::max(mx, ((g.m + 63) / 64) * ((g.n + 63) / 64));
    return mx;
}

int gemm_kmax(const std::vector<GemmDesc> &v) {
    int k = 0;
    for (const GemmDesc &g : v) k = std::max(k, g.k);
    return k;
}

double gemm_flops(const std::vector<GemmDesc> &v) {
    double f = 0.0;
    for (const GemmDesc &g : v) f += 2.0 * g.m * g.n * g.k;
    return f;
}

}  // namespace

// The diagonal tiles; U and V are allocated in segments as the ranks are found.
size_t tlr_factor_bytes(int N, int nb, int kmax) {
    (void)kmax;
    const size_t T = ((size_t)N + nb - 1) / nb;
    return sizeof(double) * (T * (size_t)nb * nb);
}

size_t tlr_workspace_bytes(int N, int nb, int kmax) {
    const size_t T = ((size_t)N + nb - 1) / nb;
    const size_t rmax = std::min((size_t)kmax + 16, (size_t)nb);
    const size_t per_tile = (5 * (size_t)nb * rmax + 4 * rmax * rmax + 4 * rmax) * sizeof(double);
    return sizeof(double) * ((size_t)N * nb                   // column panel W
                             + (size_t)nb * rmax                // Omega
                             + (size_t)nb * TLR_KCHUNK          // stacked U_jk chunk
                             + T * (size_t)nb * TLR_KCHUNK      // P_i per tile
                             + T * TLR_MAXK_PER_CHUNK * (size_t)kmax * kmax   // cores
                             + (size_t)TLR_KCHUNK * rmax        // Qc' Omega
                             + T * (size_t)TLR_KCHUNK * rmax)   // P_i' Q_i per tile
           + T * per_tile + 2 * TLR_ARENA_BYTES + (size_t)N * 2 * sizeof(double) + 16 * 256 + 4096 +
           TLR_SPLITK_BYTES + 256;
}

namespace {
// Registers the split-K scratch of the batched GEMMs for the calls on this thread.
struct SplitKScope {
    SplitKScope(void *ws, size_t bytes) { bgemm_splitk_scratch((double *)ws, bytes); }
    ~SplitKScope() { bgemm_splitk_scratch(nullptr, 0); }
};
}  // namespace

cudaError_t tlr_factor(TlrFactor &F, const CovParams &cp, const double *lx, const double *ly, void *ws,
                       size_t ws_bytes, void *arena_host, DevStatus *st, DevStatus *h_st, cudaStream_t s) {
    const int N = F.N, nb = F.nb, T = F.T, kmax = F.kmax, p = cp.p;
    const int rmax = std::min(kmax + 16, nb);
    if (nb % p) return cudaErrorInvalidValue;
    if (ws_bytes < tlr_workspace_bytes(N, nb, kmax)) return cudaErrorInvalidValue;
    auto mt = [&](int t) { return std::min(nb, N - t * nb); };
    // carve the workspace
    uint8_t *w = (uint8_t *)ws;
    auto take = [&](size_t bytes) {
        uint8_t *q = w;
        w += (bytes + 255) & ~(size_t)255;
        return q;
    };
    double *W = (double *)take(sizeof(double) * (size_t)N * nb);
    double *Om = (double *)take(sizeof(double) * (size_t)nb * rmax);
    double *Qc = (double *)take(sizeof(double) * (size_t)nb * TLR_KCHUNK);
    double *Pb = (double *)take(sizeof(double) * (size_t)T * nb * TLR_KCHUNK);
    double *Mb = (double *)take(sizeof(double) * (size_t)T * TLR_MAXK_PER_CHUNK * kmax * kmax);
    double *Zb = (double *)take(sizeof(double) * (size_t)TLR_KCHUNK * rmax);
    double *Tb = (double *)take(sizeof(double) * (size_t)T * TLR_KCHUNK * rmax);
    // per tile: Y, Q, B', Q2 (nb x rmax), M, Vj, Ms, Vs (rmax^2), sigma, tau, v0, spare (rmax), saved Y (nb x rmax)
    const size_t per_tile = 5 * (size_t)nb * rmax + 4 * (size_t)rmax * rmax + 4 * (size_t)rmax;
    double *TW = (double *)take(sizeof(double) * (size_t)T * per_tile);
    SplitKScope splitk(take(TLR_SPLITK_BYTES), TLR_SPLITK_BYTES);
    Arena arena;
    arena.dev = take(TLR_ARENA_BYTES);
    arena.host = (uint8_t *)arena_host;
    arena.cap = TLR_ARENA_BYTES;
    double *h_sigma = (double *)((uint8_t *)arena_host + TLR_ARENA_BYTES);   // pinned, T * rmax doubles
    cudaError_t e = cudaSuccess;
#define TCK(x)                                  \
    do {                                        \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    const size_t nslots = (size_t)T * (T - 1) / 2;
    F.rank.assign(nslots, 0);
    F.uptr.assign(nslots, nullptr);
    F.vptr.assign(nslots, nullptr);
    F.dense.assign(nslots, 0);
    F.capped = 0;
    F.max_rank = 0;
    auto slot = [&](int i, int j) { return (size_t)i * (i - 1) / 2 + j; };
    auto Uof = [&](int i, int j) { return F.Uof(slot(i, j)); };
    auto Vof = [&](int i, int j) { return F.Vof(slot(i, j)); };
    // per-tile compression buffers (tile index i - j - 1 within the column)
    auto tb = [&](int q) { return TW + (size_t)q * per_tile; };
    std::vector<int> rank_hint;   // rank by distance from the diagonal in the previous column

    for (int j = 0; j < T; ++j) {
        const int mj = mt(j);
        const int Rj = N - j * nb;
        const long long ldw = Rj;
        // 1. dense column panel
        {
            const int l0 = j * nb / p, nl = Rj / p, r0 = j * nb / p, nr = mj / p;
            dim3 grid((nr + 3) / 4, (nl + 63) / 64);
            KScope ks(GEO_K_COVGEN, s, 0.0, 8.0 * (double)Rj * mj);
            k_covgen_block<<<grid, 256, 0, s>>>(cp, lx, ly, l0, nl, r0, nr, W, ldw);
            TCK(cudaGetLastError());
        }
        // 2. the updates of the finished columns k < j, applied implicitly:
        //    W_ij = Sigma_ij - P_i Qc'  with  Qc = [U_jk]_k and P_i = [U_ik (V_ik' V_jk)]_k
        //    (stacked over k in chunks).  Only the diagonal tile and the tiles
        //    stored dense are formed; the others enter the randomized SVD through
        //    Y_i = Sigma_ij Omega - P_i (Qc' Omega) and B_i' = Sigma_ij' Q_i - Qc (P_i' Q_i).
        const int nt = T - j - 1;
        std::vector<int> rk(nt, 0), rused(nt, 0), rwant(nt);
        std::vector<char> dense_now(nt, 0);   // tiles formed densely with the diagonal tile (none)
        for (int q = 0; q < nt; ++q) {
            const int d = q + 1;
            const int hint = (j > 0 && d < (int)rank_hint.size()) ? rank_hint[d] : 16;
            // sketch width: the rank at the same distance in the previous column plus
            // oversampling, rounded up to 32 (the widest sketch after a dense tile); the
            // widest sketch if that fails.  Whether a tile is stored dense is decided by
            // its own compression only (a forecast from the previous column would feed
            // on itself and spread the dense band).
            rwant[q] = std::min(rmax, std::max(32, (hint + 16 + 31) / 32 * 32));
        }
        auto Ysave = [&](int q) { return tb(q) + 4 * (size_t)nb * rmax + 4 * (size_t)rmax * rmax + 4 * (size_t)rmax; };
        // for each chunk of row j's finished columns: Qc, and P_i for the tiles i in `rows`
        // (i - j in 0 .. nt), then apply(Kc, has) with has[i - j] = some rank of the chunk in row i
        auto chunk_loop = [&](const std::vector<int> &rows, auto &&apply) -> cudaError_t {
            cudaError_t ce = cudaSuccess;
            std::vector<int> ks;
            for (int k = 0; k < j; ++k)
                if (F.rank[slot(j, k)] > 0) ks.push_back(k);
            size_t pos = 0;
            while (pos < ks.size()) {
                std::vector<int> chunk;
                int Kc = 0;
                while (pos < ks.size() && (int)chunk.size() < TLR_MAXK_PER_CHUNK &&
                       Kc + F.rank[slot(j, ks[pos])] <= TLR_KCHUNK) {
                    Kc += F.rank[slot(j, ks[pos])];
                    chunk.push_back(ks[pos]);
                    ++pos;
                }
                std::vector<GemmDesc> dm, dp;
                std::vector<char> has(nt + 1, 0);
                int off = 0;
                size_t mused = 0;
                const size_t mcap = (size_t)T * TLR_MAXK_PER_CHUNK * kmax * kmax;
                for (size_t ci = 0; ci < chunk.size(); ++ci) {
                    const int k = chunk[ci];
                    const size_t sjk = slot(j, k);
                    const int rjk = F.rank[sjk];
                    if ((ce = cudaMemcpyAsync(Qc + (size_t)off * nb, Uof(j, k), sizeof(double) * (size_t)nb * rjk,
                                              cudaMemcpyDeviceToDevice, s)))
                        return ce;
                    for (int i : rows) {
                        // P_ik = U_ik (V_ik' V_jk), the block of columns [off, off + rjk) of P_i
                        const size_t sik = slot(i, k);
                        const int rik = F.rank[sik];
                        if (rik == 0) continue;
                        has[i - j] = 1;
                        double *P = Pb + (size_t)(i - j) * nb * TLR_KCHUNK + (size_t)off * nb;
                        if (F.dense[sjk]) {
                            // V_jk = I: P = U_ik V_ik' (= U_ik itself when (i, k) is dense too)
                            if (F.dense[sik]) {
                                if ((ce = cudaMemcpyAsync(P, Uof(i, k), sizeof(double) * (size_t)nb * rjk,
                                                          cudaMemcpyDeviceToDevice, s)))
                                    return ce;
                            } else {
                                dp.push_back({mt(i), rjk, rik, 0, 1, Uof(i, k), nb, Vof(i, k), nb, P, nb, 1.0, 0.0});
                            }
                        } else if (F.dense[sik]) {
                            // V_ik = I: P = U_ik V_jk
                            dp.push_back({mt(i), rjk, mt(k), 0, 0, Uof(i, k), nb, Vof(j, k), nb, P, nb, 1.0, 0.0});
                        } else {
                            double *M = Mb + mused;
                            mused += (size_t)kmax * kmax;
                            if (mused > mcap) return cudaErrorMemoryAllocation;
                            dm.push_back({rik, rjk, nb, 1, 0, Vof(i, k), nb, Vof(j, k), nb, M, kmax, 1.0, 0.0});
                            dp.push_back({mt(i), rjk, rik, 0, 0, Uof(i, k), nb, M, kmax, P, nb, 1.0, 0.0});
                        }
                    }
                    off += rjk;
                }
                // rows with something in this chunk: zero the P blocks of the k with rank 0 there
                for (int i : rows) {
                    if (!has[i - j]) continue;
                    int o2 = 0;
                    for (int k : chunk) {
                        const int rjk = F.rank[slot(j, k)];
                        if (F.rank[slot(i, k)] == 0 &&
                            (ce = cudaMemsetAsync(Pb + (size_t)(i - j) * nb * TLR_KCHUNK + (size_t)o2 * nb, 0,
                                                  sizeof(double) * (size_t)nb * rjk, s)))
                            return ce;
                        o2 += rjk;
                    }
                }
                if (!dm.empty()) {
                    GemmDesc *d1 = push(arena, dm, s, &ce);
                    if (ce) return ce;
                    if ((ce = launch_bgemm(d1, (int)dm.size(), gemm_tiles(dm), s, gemm_flops(dm), gemm_kmax(dm)))) return ce;
                }
                if (!dp.empty()) {
                    GemmDesc *d2 = push(arena, dp, s, &ce);
                    if (ce) return ce;
                    if ((ce = launch_bgemm(d2, (int)dp.size(), gemm_tiles(dp), s, gemm_flops(dp), gemm_kmax(dp)))) return ce;
                }
                if ((ce = apply(Kc, has))) return ce;
            }
            return ce;
        };
        auto Pof = [&](int i) { return Pb + (size_t)(i - j) * nb * TLR_KCHUNK; };
        // dense update W_i -= P_i Qc' for the listed tiles
        auto dense_update = [&](const std::vector<int> &rows, int Kc, const std::vector<char> &has) -> cudaError_t {
            std::vector<GemmDesc> dw;
            for (int i : rows)
                if (has[i - j])
                    dw.push_back({mt(i), mj, Kc, 0, 1, Pof(i), nb, Qc, nb, W + (size_t)(i - j) * nb, ldw, -1.0, 1.0});
            if (dw.empty()) return cudaSuccess;
            cudaError_t ce;
            GemmDesc *d3 = push(arena, dw, s, &ce);
            if (ce) return ce;
            return launch_bgemm(d3, (int)dw.size(), gemm_tiles(dw), s, gemm_flops(dw), gemm_kmax(dw));
        };
        // the Gaussian test matrix of this column and the raw sketches Y_i = Sigma_ij Omega
        TCK(launch_gaussian(Om, (long long)nb * rmax, 0x5EEDull * (j + 1), s));
        std::vector<int> all_rows{j}, dense_rows{j}, lr_rows;
        for (int q = 0; q < nt; ++q) {
            all_rows.push_back(j + 1 + q);
            if (F.dst > 0) {
                // Diagonal Super Tile: the tiles within the band are formed densely, the others dropped
                if (q + 1 < F.dst) dense_rows.push_back(j + 1 + q);
            } else {
                (dense_now[q] ? dense_rows : lr_rows).push_back(j + 1 + q);
            }
        }
        if (!lr_rows.empty()) {
            std::vector<GemmDesc> dy0;
            for (int i : lr_rows)
                dy0.push_back({mt(i), rmax, mj, 0, 0, W + (size_t)(i - j) * nb, ldw, Om, nb, Ysave(i - j - 1), nb,
                               1.0, 0.0});
            GemmDesc *g0 = push(arena, dy0, s, &e);
            TCK(e);
            TCK(launch_bgemm(g0, (int)dy0.size(), gemm_tiles(dy0), s, gemm_flops(dy0), gemm_kmax(dy0)));
        }
        TCK(chunk_loop(all_rows, [&](int Kc, const std::vector<char> &has) -> cudaError_t {
            cudaError_t ce = dense_update(dense_rows, Kc, has);
            if (ce || lr_rows.empty()) return ce;
            // Z = Qc' Omega, then Y_i -= P_i Z
            std::vector<GemmDesc> dz{{Kc, rmax, mj, 1, 0, Qc, nb, Om, nb, Zb, TLR_KCHUNK, 1.0, 0.0}};
            std::vector<GemmDesc> dy;
            for (int i : lr_rows)
                if (has[i - j])
                    dy.push_back({mt(i), rmax, Kc, 0, 0, Pof(i), nb, Zb, TLR_KCHUNK, Ysave(i - j - 1), nb, -1.0, 1.0});
            GemmDesc *gz = push(arena, dz, s, &ce);
            if (ce) return ce;
            if ((ce = launch_bgemm(gz, 1, gemm_tiles(dz), s, gemm_flops(dz), gemm_kmax(dz)))) return ce;
            if (dy.empty()) return cudaSuccess;
            GemmDesc *gy = push(arena, dy, s, &ce);
            if (ce) return ce;
            return launch_bgemm(gy, (int)dy.size(), gemm_tiles(dy), s, gemm_flops(dy), gemm_kmax(dy));
        }));
        // 3. diagonal tile in FP64
        TCK(chol64_panel(W, ldw, 0, mj, mj, mj, st, s));
        TCK(cudaMemcpy2DAsync(F.D + (size_t)j * nb * nb, sizeof(double) * nb, W, sizeof(double) * ldw,
                              sizeof(double) * mj, mj, cudaMemcpyDeviceToDevice, s));
        if (j == T - 1) break;
        // 4. compress the tiles below: first with a narrow sketch, then the widest one where needed
        std::vector<int> todo;
        for (int q = 0; q < nt; ++q) {
            if (F.dst > 0)
                rk[q] = (q + 1 < F.dst) ? -1 : 0;   // dense within the band, rank 0 beyond
            else if (dense_now[q])
                rk[q] = -1;
            else
                todo.push_back(q);
        }
        std::vector<std::vector<int>> sel(nt);
        for (int pass = 0; pass < 2 && !todo.empty(); ++pass) {
            std::vector<GemmDesc> db;
            std::vector<QrDesc> dq1, dq2;
            std::vector<TlrR2Desc> dr;
            std::vector<SvdDesc> dsv;
            std::vector<int> rows_b;
            int r = 0;
            for (int q : todo) r = std::max(r, std::min(std::min(pass == 0 ? rwant[q] : rmax, mj), mt(j + 1 + q)));
            for (int q : todo) {
                const int i = j + 1 + q;
                const int mi = mt(i);
                const int rr = std::min(std::min(pass == 0 ? rwant[q] : rmax, mj), mi);
                double *b = tb(q);
                double *Y = b, *Q = b + (size_t)nb * rmax, *Bt = Q + (size_t)nb * rmax, *Q2 = Bt + (size_t)nb * rmax;
                double *M = Q2 + (size_t)nb * rmax, *Vj = M + (size_t)rmax * rmax, *Ms = Vj + (size_t)rmax * rmax;
                double *Vs = Ms + (size_t)rmax * rmax, *sig = Vs + (size_t)rmax * rmax, *tau = sig + rmax;
                double *v0 = tau + rmax;
                double *Wi = W + (size_t)(i - j) * nb;
                // the first rr columns of the saved sketch (the QR works in place)
                TCK(cudaMemcpyAsync(Y, Ysave(q), sizeof(double) * (size_t)nb * rr, cudaMemcpyDeviceToDevice, s));
                dq1.push_back({mi, rr, Y, nb, Q, nb, tau, v0});
                db.push_back({mj, rr, mi, 1, 0, Wi, ldw, Q, nb, Bt, nb, 1.0, 0.0});
                dq2.push_back({mj, rr, Bt, nb, Q2, nb, tau, v0});
                dr.push_back({rr, Bt, nb, M, rmax});
                dsv.push_back({rr, M, Vj, rmax, sig, F.tol / 16.0});
                rused[q] = rr;
                rows_b.push_back(i);
            }
            QrDesc *q1 = push(arena, dq1, s, &e);
            TCK(e);
            TCK(launch_house_qr(q1, (int)dq1.size(), nb, r, s, 4.0 * (double)dq1.size() * nb * r * r));
            GemmDesc *g2 = push(arena, db, s, &e);
            TCK(e);
            TCK(launch_bgemm(g2, (int)db.size(), gemm_tiles(db), s, gemm_flops(db), gemm_kmax(db)));
            // B_i' -= Qc (P_i' Q_i)
            TCK(chunk_loop(rows_b, [&](int Kc, const std::vector<char> &has) -> cudaError_t {
                std::vector<GemmDesc> dt1, dt2;
                for (int i : rows_b) {
                    if (!has[i - j]) continue;
                    const int q = i - j - 1;
                    double *Q = tb(q) + (size_t)nb * rmax, *Bt = Q + (size_t)nb * rmax;
                    double *Tq = Tb + (size_t)q * TLR_KCHUNK * rmax;
                    dt1.push_back({Kc, rused[q], mt(i), 1, 0, Pof(i), nb, Q, nb, Tq, TLR_KCHUNK, 1.0, 0.0});
                    dt2.push_back({mj, rused[q], Kc, 0, 0, Qc, nb, Tq, TLR_KCHUNK, Bt, nb, -1.0, 1.0});
                }
                if (dt1.empty()) return cudaSuccess;
                cudaError_t ce;
                GemmDesc *h1 = push(arena, dt1, s, &ce);
                if (ce) return ce;
                if ((ce = launch_bgemm(h1, (int)dt1.size(), gemm_tiles(dt1), s, gemm_flops(dt1), gemm_kmax(dt1)))) return ce;
                GemmDesc *h2 = push(arena, dt2, s, &ce);
                if (ce) return ce;
                return launch_bgemm(h2, (int)dt2.size(), gemm_tiles(dt2), s, gemm_flops(dt2), gemm_kmax(dt2));
            }));
            QrDesc *q2 = push(arena, dq2, s, &e);
            TCK(e);
            TCK(launch_house_qr(q2, (int)dq2.size(), nb, r, s, 4.0 * (double)dq2.size() * nb * r * r));
            TlrR2Desc *r2 = push(arena, dr, s, &e);
            TCK(e);
            {
                KScope kk(GEO_K_AUX, s);
                k_copy_r2t<<<dim3((r * r + 255) / 256, (unsigned)dr.size()), 256, 0, s>>>(r2, (int)dr.size());
                TCK(cudaGetLastError());
            }
            SvdDesc *sv = push(arena, dsv, s, &e);
            TCK(e);
            TCK(launch_jacobi_svd(sv, (int)dsv.size(), 30, r, s, 3.0 * 12.0 * (double)dsv.size() * r * r * r));
            // singular values to the host
            for (size_t t = 0; t < todo.size(); ++t) {
                const int q = todo[t];
                double *sig = tb(q) + 4 * (size_t)nb * rmax + 4 * (size_t)rmax * rmax;
                TCK(cudaMemcpyAsync(h_sigma + (size_t)t * rmax, sig, sizeof(double) * rused[q], cudaMemcpyDeviceToHost,
                                    s));
            }
            TCK(cudaStreamSynchronize(s));
            arena.used = 0;
            if (h_st) {
                TCK(cudaMemcpy(h_st, st, sizeof(DevStatus), cudaMemcpyDeviceToHost));
                if (h_st->info) return cudaSuccess;   // not SPD: the caller reports it
            }
            std::vector<int> next;
            for (size_t t = 0; t < todo.size(); ++t) {
                const int q = todo[t];
                const int rr = rused[q];
                std::vector<int> idx(rr);
                std::iota(idx.begin(), idx.end(), 0);
                const double *sg = h_sigma + (size_t)t * rmax;
                std::stable_sort(idx.begin(), idx.end(), [&](int a, int b2) { return sg[a] > sg[b2]; });
                int k = 0;
                while (k < rr && sg[idx[k]] > F.tol) ++k;
                // the sketch must exceed the kept rank by 8 columns (oversampling) unless it spans the tile
                const bool full = (k + 8 > rr) && rr < std::min(mt(j + 1 + q), mj);
                if (full && pass == 0 && rr < std::min(std::min(rmax, mj), mt(j + 1 + q))) {
                    next.push_back(q);   // too narrow: redo with the widest sketch
                    continue;
                }
                if (k > kmax || full) {
                    // rank above kmax, or beyond the widest sketch: the tile is stored dense
                    rk[q] = -1;
                    continue;
                }
                rk[q] = k;
                sel[q].assign(idx.begin(), idx.begin() + k);
            }
            todo = next;
        }
        // tiles found dense during the compression: form them (W_i -= P_i Qc') before their TRSM
        {
            std::vector<int> late;
            for (int q = 0; q < nt; ++q)
                if (rk[q] < 0 && !dense_now[q] && F.dst == 0) late.push_back(j + 1 + q);
            if (!late.empty())
                TCK(chunk_loop(late, [&](int Kc, const std::vector<char> &has) -> cudaError_t {
                    return dense_update(late, Kc, has);
                }));
        }
        // U = Q (M Vj)[:, sel], V = Q2 Vj[:, sel]
        {
            std::vector<int> hsel;
            std::vector<size_t> selpos(nt);
            for (int q = 0; q < nt; ++q) {
                selpos[q] = hsel.size();
                hsel.insert(hsel.end(), sel[q].begin(), sel[q].end());
            }
            int *dsel = nullptr;
            if (!hsel.empty()) {
                dsel = push(arena, hsel, s, &e);
                TCK(e);
            }
            std::vector<TlrSelDesc> dg;
            std::vector<GemmDesc> du, dv;
            // pool space for every tile of the column, then the dense tiles (U = W_ij, V = I)
            for (int q = 0; q < nt; ++q) {
                const int i = j + 1 + q;
                const size_t sl = slot(i, j);
                if (rk[q] < 0) {
                    rk[q] = mj;
                    F.dense[sl] = 1;
                    F.capped += 1;
                }
                if (rk[q] > 0) {
                    F.uptr[sl] = F.take((size_t)nb * rk[q]);
                    F.vptr[sl] = F.take((size_t)nb * rk[q]);
                    if (!F.uptr[sl] || !F.vptr[sl]) return cudaErrorMemoryAllocation;
                }
                F.rank[sl] = rk[q];
                F.max_rank = std::max(F.max_rank, F.dense[sl] ? 0 : rk[q]);
                if (F.dense[sl]) {
                    // L_ij = W_ij L_jj^-T in FP64 (the panel TRSM on these rows), U = L_ij, V = I
                    TCK(chol64_panel(W, ldw, 0, mj, (i - j) * nb, (i - j) * nb + mt(i), st, s, false));
                    TCK(cudaMemcpy2DAsync(Uof(i, j), sizeof(double) * nb, W + (size_t)(i - j) * nb, sizeof(double) * ldw,
                                          sizeof(double) * mt(i), mj, cudaMemcpyDeviceToDevice, s));
                    KScope kk(GEO_K_AUX, s);
                    k_identity<<<(unsigned)(((size_t)nb * mj + 255) / 256), 256, 0, s>>>(Vof(i, j), nb, mj);
                    TCK(cudaGetLastError());
                }
            }
            for (int q = 0; q < nt; ++q) {
                const int i = j + 1 + q, k = rk[q];
                if (k == 0 || F.dense[slot(i, j)]) continue;
                double *b = tb(q);
                double *Q = b + (size_t)nb * rmax, *Q2 = Q + 2 * (size_t)nb * rmax;
                double *M = Q2 + (size_t)nb * rmax, *Vj = M + (size_t)rmax * rmax, *Ms = Vj + (size_t)rmax * rmax;
                double *Vs = Ms + (size_t)rmax * rmax;
                dg.push_back({rused[q], k, M, Vj, Ms, Vs, rmax, dsel + selpos[q]});
                du.push_back({mt(i), k, rused[q], 0, 0, Q, nb, Ms, rmax, Uof(i, j), nb, 1.0, 0.0});
                dv.push_back({mj, k, rused[q], 0, 0, Q2, nb, Vs, rmax, Vof(i, j), nb, 1.0, 0.0});
            }
            if (!dg.empty()) {
                TlrSelDesc *g = push(arena, dg, s, &e);
                TCK(e);
                int mx = 0;
                for (auto &x : dg) mx = std::max(mx, x.r * x.k);
                {
                    KScope kk(GEO_K_AUX, s);
                    k_gather_sel<<<dim3((mx + 255) / 256, (unsigned)dg.size()), 256, 0, s>>>(g, (int)dg.size());
                    TCK(cudaGetLastError());
                }
                GemmDesc *g1 = push(arena, du, s, &e);
                TCK(e);
                TCK(launch_bgemm(g1, (int)du.size(), gemm_tiles(du), s, gemm_flops(du), gemm_kmax(du)));
                GemmDesc *g2 = push(arena, dv, s, &e);
                TCK(e);
                TCK(launch_bgemm(g2, (int)dv.size(), gemm_tiles(dv), s, gemm_flops(dv), gemm_kmax(dv)));
                // 5. V_ij <- L_jj^-1 V_ij, 64-row blocks
                const double *Ljj = F.D + (size_t)j * nb * nb;
                std::vector<TlrTrsmDesc> dt;
                int maxc = 0;
                for (int q = 0; q < nt; ++q)
                    if (rk[q] > 0 && !F.dense[slot(j + 1 + q, j)]) {
                        dt.push_back({Ljj, nb, Vof(j + 1 + q, j), nb, rk[q]});
                        maxc = std::max(maxc, rk[q]);
                    }
                TlrTrsmDesc *gt = push(arena, dt, s, &e);
                TCK(e);
                for (int c0 = 0; c0 < mj; c0 += 64) {
                    const int cb = std::min(64, mj - c0);
                    {
                        KScope kk(GEO_K_TRSM, s, (double)cb * cb * 0.5 * maxc * dt.size(), 0.0);
                        k_trsm_left_diag<<<dim3((maxc + 63) / 64, (unsigned)dt.size()), 256, 0, s>>>(gt, (int)dt.size(),
                                                                                                 c0, cb);
                        TCK(cudaGetLastError());
                    }
                    if (c0 + cb < mj) {
                        std::vector<GemmDesc> du2;
                        for (auto &x : dt)
                            du2.push_back({mj - c0 - cb, x.ncols, cb, 0, 0, Ljj + (size_t)c0 * nb + c0 + cb, nb,
                                           x.X + c0, nb, x.X + c0 + cb, nb, -1.0, 1.0});
                        GemmDesc *g3 = push(arena, du2, s, &e);
                        TCK(e);
                        TCK(launch_bgemm(g3, (int)du2.size(), gemm_tiles(du2), s, gemm_flops(du2), gemm_kmax(du2)));
                    }
                }
            }
        }
        rank_hint.assign(nt + 1, 0);
        for (int q = 0; q < nt; ++q) rank_hint[q + 1] = F.dense[slot(j + 1 + q, j)] ? rmax : rk[q];
        TCK(cudaStreamSynchronize(s));
        arena.used = 0;
    }
#undef TCK
    return cudaSuccess;
}

// y = L^-1 z (forward) or w = L^-T y (backward) with the TLR factor; x in place.
cudaError_t tlr_solve(const TlrFactor &F, double *x, bool transpose, void *ws, void *arena_host, cudaStream_t s) {
    const int N = F.N, nb = F.nb, T = F.T;
    auto mt = [&](int t) { return std::min(nb, N - t * nb); };
    auto slot = [&](int i, int j) { return (size_t)i * (i - 1) / 2 + j; };
    uint8_t *w = (uint8_t *)ws;
    double *tbuf = (double *)w;                       // T x nb     (V' y_k or U' w_k; dense tiles have rank nb)
    double *cbuf = tbuf + (size_t)T * nb;             // nb x T     (contributions)
    Arena arena;
    arena.dev = (uint8_t *)(cbuf + (size_t)nb * T);
    arena.dev = (uint8_t *)(((uintptr_t)arena.dev + 255) & ~(uintptr_t)255);
    arena.host = (uint8_t *)arena_host;
    arena.cap = TLR_ARENA_BYTES;
    int *sync = (int *)(arena.dev + TLR_ARENA_BYTES);   // the diagonal solves' sync words
    SplitKScope splitk((void *)(((uintptr_t)sync + 512 + 255) & ~(uintptr_t)255), TLR_SPLITK_BYTES);
    cudaError_t e = cudaSuccess;
    for (int step = 0; step < T; ++step) {
        const int i = transpose ? T - 1 - step : step;
        std::vector<GemmDesc> d1, d2;
        int nc = 0;
        const int others = transpose ? T - 1 - i : i;
        for (int o = 0; o < others; ++o) {
            const int k = transpose ? i + 1 + o : o;
            const size_t sl = transpose ? slot(k, i) : slot(i, k);
            const int r = F.rank[sl];
            if (r == 0) continue;
            const double *U = F.Uof(sl), *V = F.Vof(sl);
            // forward: t = V_ik' y_k, c = U_ik t;  backward: t = U_ki' w_k, c = V_ki t
            const double *A1 = transpose ? U : V, *A2 = transpose ? V : U;
            const int m1 = transpose ? mt(k) : mt(k);
            d1.push_back({r, 1, m1, 1, 0, A1, nb, x + (size_t)k * nb, nb, tbuf + (size_t)nc * nb, nb, 1.0, 0.0});
            d2.push_back({mt(i), 1, r, 0, 0, A2, nb, tbuf + (size_t)nc * nb, nb, cbuf + (size_t)nc * nb, nb, 1.0,
                          0.0});
            ++nc;
        }
        if (nc > 0) {
            GemmDesc *g1 = push(arena, d1, s, &e);
            if (e) return e;
            if ((e = launch_bgemm(g1, nc, gemm_tiles(d1), s, gemm_flops(d1), gemm_kmax(d1)))) return e;
            GemmDesc *g2 = push(arena, d2, s, &e);
            if (e) return e;
            if ((e = launch_bgemm(g2, nc, gemm_tiles(d2), s, gemm_flops(d2), gemm_kmax(d2)))) return e;
            KScope ks(GEO_K_SOLVE, s);
            k_sub_cols<<<(mt(i) + 255) / 256, 256, 0, s>>>(x + (size_t)i * nb, cbuf, nb, mt(i), nc);
            if ((e = cudaGetLastError())) return e;
        }
        const double *Dii = F.D + (size_t)i * nb * nb;
        if (transpose) {
            if ((e = backward_solve(Dii, nb, mt(i), x + (size_t)i * nb, 1, x + (size_t)i * nb, sync, nullptr, s)))
                return e;
        } else {
            if ((e = forward_solve(Dii, nb, mt(i), x + (size_t)i * nb, sync, nullptr, s))) return e;
        }
        if (arena.used > TLR_ARENA_BYTES / 2) {
            if ((e = cudaStreamSynchronize(s))) return e;
            arena.used = 0;
        }
    }
    return cudaSuccess;
}

size_t tlr_solve_workspace_bytes(int N, int nb, int kmax) {
    (void)kmax;
    const size_t T = ((size_t)N + nb - 1) / nb;
    return sizeof(double) * (T * (size_t)nb + (size_t)nb * T) + TLR_ARENA_BYTES + 512 + 64 + TLR_SPLITK_BYTES + 512;
}

cudaError_t tlr_reduce(const TlrFactor &F, const double *y, const DevStatus *st, DevResults *res, cudaStream_t s) {
    KScope ks(GEO_K_REDUCE, s, 3.0 * F.N, 16.0 * F.N);
    k_tlr_reduce<<<1, 1024, 0, s>>>(F.D, F.nb, F.T, F.N, y, st, res);
    return cudaGetLastError();
}
