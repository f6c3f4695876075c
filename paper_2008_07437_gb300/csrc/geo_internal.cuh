// Internal declarations shared by the translation units of libgeo.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <utility>
#include <vector>

#include "geo.h"
#include "matern.cuh"

// Status words the kernels write (device memory of the context).
struct DevStatus {
    int info;      // 0, or 1-based row of the first non-positive pivot
    int timeout;   // a bounded wait expired (code of the wait site)
    int pad[2];
};

// Device scalars of one likelihood evaluation.
struct DevResults {
    double loglik, logdet, quad, pad;
};

// Matrix view: column-major, A[c * ld + r].
struct MatView {
    double *a;
    long long ld;
};

// ---- per-launch profiling (api.cu) ---------------------------------------
// The API entry points point t_prof at their context's profiler; every
// launch site opens a KScope, which counts the launch and, when recording is
// on, brackets it with CUDA events on the launching stream.
struct Profiler {
    bool enabled = false;
    long long launches[GEO_K_COUNT] = {};
    long long timed[GEO_K_COUNT] = {};
    double flops[GEO_K_COUNT] = {};
    double bytes[GEO_K_COUNT] = {};
    double ms[GEO_K_COUNT] = {};
    unsigned long long *d_tc_flops = nullptr;   // device counter: tensor-core flops of the emulated products
    struct Rec {
        int cls;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    cudaEvent_t take();
    void resolve();
    void clear();
};
extern thread_local Profiler *t_prof;

struct KScope {
    Profiler *p;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    KScope(int cls_, cudaStream_t s_, double flops = 0.0, double bytes = 0.0);
    ~KScope();
};

// ---- covgen.cu ----------------------------------------------------------
// Build the K_nu tables of theta into tab (GEO_TAB_DOUBLES device doubles) on
// stream s and point cp.tab at them; every covariance kernel launched with cp
// afterwards reads them.  Nothing is launched when theta has no tabulated order.
cudaError_t launch_cheb_build(CovParams &cp, double *tab, cudaStream_t s);
bool cov_needs_tables(const CovParams &cp);
// Lower triangle of Sigma (order p*n) into A (column-major, ld), from
// SoA locations; the full p x p block on the location diagonal.
cudaError_t launch_covgen_sym(const CovParams &cp, const double *lx, const double *ly, int n, double *A,
                              long long ld, cudaStream_t s);
// Full rectangular cross-covariance, rows p*n1 (locations 1), cols p*n2.
cudaError_t launch_covgen_rect(const CovParams &cp, const double *l1, int n1, const double *l2, int n2,
                               double *out, long long ld, cudaStream_t s);
// zhat[p*l + i] = sum_{r,j} C_ij(|s0_l - s_r|) w[p*r + j]; s0 interleaved (x,y), s SoA.
cudaError_t launch_predict(const CovParams &cp, const double *new_locs, int m, const double *lx,
                           const double *ly, int n, const double *w, double *zhat, cudaStream_t s);
// One entry of a batched prediction: a factor's theta constants, locations (SoA, n), weights w
// (p n), its m new locations s0 (AoS) and outputs zhat (p m); first = the entry's first global index.
struct PredDesc {
    CovParams cp;
    const double *lx, *ly, *w;
    const double *s0;
    double *zhat;
    int n, m, first;
};
// d: count device entries whose m sum to total; one CTA per new location.
cudaError_t launch_predict_batch(const PredDesc *d, int count, int total, double flops, cudaStream_t s);
// AoS (x, y) -> SoA gathered by perm (device ints).
cudaError_t launch_gather_locs(const double *locs, const int *perm, int n, double *lx, double *ly,
                               cudaStream_t s);
// out[k] = in[perm-ordered Rep. I]: out[p*k + i] = in[p*perm[k] + i], strided store (stride for out).
cudaError_t launch_gather_vec(const double *in, const int *perm, int n, int p, double *out, long long stride,
                              cudaStream_t s);
cudaError_t launch_scatter_vec(const double *in, long long stride, const int *perm, int n, int p, double *out,
                               cudaStream_t s);

// ---- chol64.cu ----------------------------------------------------------
// In-place lower Cholesky of the leading N x N block of A; rows N..nrows-1
// are extra right-hand-side rows carried through the factorisation (row N
// receives (L^-1 z)' when it holds z').  nb = outer tile size.
cudaError_t chol64_factor(double *A, long long ld, int N, int nrows, int nb, DevStatus *st, cudaStream_t s);
// The rank-64 updates inside a panel, C[rC.., cC..] (m x n) -= A[rC.., kA..kA+k] A[cC.., kA..kA+k]'
// (lower part when rC == cC), when they should not run on the FP64 pipe.
struct PanelUpdate {
    cudaError_t (*fn)(const PanelUpdate *u, double *A, long long ld, int rC, int cC, int m, int n, int kA, int k,
                      DevStatus *st, cudaStream_t s);
    void *ctx;
};
// One panel [j0, j0+jb): diagonal tile plus extra rows [x0, x1) carried along.
cudaError_t chol64_panel(double *A, long long ld, int j0, int jb, int x0, int x1, DevStatus *st, cudaStream_t s,
                         bool factor_diag = true, const PanelUpdate *upd = nullptr);
// C[rC.., cC..] (m x n) -= A[rC.., kA..kA+k] A[cC.., kA..kA+k]' in FP64.
cudaError_t chol64_gemm_update(double *A, long long ld, int rC, int cC, int m, int n, int kA, int k, DevStatus *st,
                               cudaStream_t s);

// ---- chol_mixed.cu --------------------------------------------------------
size_t mixed_workspace_bytes(int N, int nb);
cudaError_t chol_mixed_factor(double *A, long long ld, int N, int nrows, int nb, int band, int lowp, void *ws,
                              size_t ws_bytes, DevStatus *st, cudaStream_t s);


// ---- ozaki.cu -------------------------------------------------------------
// FP64-accurate products on the BF16 tensor cores: the rows of an operand
// as S BF16 digit slices with a power-of-two exponent per row and K chunk.
struct OzSlices {
    void *d;                  // S slices of rows x Kp BF16 digits (row-major, K contiguous)
    int *e;                   // row exponents, nchunk x rows
    int S, K, Kp, kchunk, nchunk;
    long long rows;           // capacity: row stride of the exponent array
    long long valid;          // rows holding data (extent of the tensor maps)
    long long slice_stride;   // elements between slices
    int *be;                  // per 32-row block exponent maxima: 2 nchunk x bstride (all rows, reference rows)
    long long bstride;
    long long ref_rows;       // rows that set the level cut's reference scale (-1: every sliced row)
};
// Depth of one exact-accumulation launch: S * kmax * 2^12 <= 2^24.
int oz_kmax(int S);
size_t oz_slices_bytes(long long rows, int K, int S);
OzSlices oz_slices_carve(void *ws, long long rows, int K, int S);
// Slices of rows [0, R) of the column-major panel P (ld), columns [0, o.K).
cudaError_t oz_slice(const double *P, long long ld, int R, const OzSlices &o, const DevStatus *st, cudaStream_t s);
// C[r0 + i, c0 + j] -= sum_k A[a_off + i, k] B[b_off + j, k] for i < rows, j < cols, written only
// where the global row < m_end and col < n_end (and row >= col when tri); grid_cap persistent CTAs.
// overwrite = 1: C = -sum (C is not read).  cut = 1: each output tile keeps only the digit levels
// its operands' magnitudes need against the launch's largest rows (not with overwrite).
cudaError_t oz_update(const OzSlices &A, const OzSlices &B, double *C, long long ldc, int r0, int c0, int rows,
                      int cols, int m_end, int n_end, int a_off, int b_off, int tri, int grid_cap, DevStatus *st,
                      cudaStream_t s, int overwrite, int cut);
size_t oz_chol_workspace_bytes(int nrows, int nb, int S);
// Dense Cholesky as chol64_factor, trailing updates and panel solves on the
// tensor cores with S slices (nb <= 1024); cut = 1: the trailing updates use the level cut.
cudaError_t chol_oz_factor(double *A, long long ld, int N, int nrows, int nb, int S, int cut, void *ws,
                           size_t ws_bytes, DevStatus *st, cudaStream_t s);
size_t oz_gemm_workspace_bytes(int m, int n, int k, int S);
// C (m x n) -= A (m x k) B (n x k)', column-major FP64, S slices.
cudaError_t oz_gemm(int m, int n, int k, const double *A, long long lda, const double *B, long long ldb, double *C,
                    long long ldc, int S, void *ws, DevStatus *st, cudaStream_t s);

// ---- mloe.cu --------------------------------------------------------------
// Rows = prediction locations (AoS s0, m), cols = observed locations (SoA, n):
// out[(p r + j) * ld + (p q + i)] = C_ij(|s0_q - s_r|).
cudaError_t launch_covgen_cross(const CovParams &cp, const double *s0, int m, const double *lx, const double *ly,
                                int n, double *out, long long ld, cudaStream_t s);
// s[q] = sum_c X[q, c]^2, d[q] = sum_c X[q, c] Y[q, c] (Y, d may be NULL), q < R, c < N.
cudaError_t launch_row_sums(const double *X, long long ldx, const double *Y, long long ldy, int R, int N, double *s,
                            double *d, cudaStream_t st);
// X <- X L^-1 (X: R x N, L lower); arena_dev: 64 GemmDesc of device scratch.
cudaError_t trsm_right_lower(double *X, long long ldx, int R, const double *L, long long ldl, int N, void *arena_dev,
                             cudaStream_t s);
// X <- X L^-T (X: R x N, L lower); arena_dev: 64 GemmDesc of device scratch.
cudaError_t trsm_right_upper_t(double *X, long long ldx, int R, const double *L, long long ldl, int N,
                               void *arena_dev, cudaStream_t s);
// Y = X' (X: R x C column-major, ldx; Y: C x R column-major, ldy).
cudaError_t launch_transpose(const double *X, long long ldx, int R, int C, double *Y, long long ldy, cudaStream_t s);
// sums[q] = sum_{c < N} Y[q * ldy + c]^2, q < R (columns of a column-major Y).
cudaError_t launch_col_sumsq(const double *Y, long long ldy, int N, int R, double *sums, cudaStream_t s);
// var[q] = c0diag[q mod p] - sums[q] (device arrays of R doubles).
cudaError_t launch_var_finish(const double *sums, int R, int p, const double *c0diag, double *var, cudaStream_t s);
// V = X L (L lower; the upper parts of its 64 x 64 diagonal blocks are zeroed);
// arena_dev / arena_host (pinned): ceil(N / 64) GemmDesc each.
cudaError_t trmm_right_lower(const double *X, long long ldx, int R, double *L, long long ldl, int N, double *V,
                             long long ldv, void *arena_dev, void *arena_host, cudaStream_t s);

// ---- api.cu (for the request server) ---------------------------------------
// Device bytes a context holds (cached workspaces and kept factors).
size_t ctx_device_bytes(const geo_ctx *ctx);
// Free the context's cached workspaces (after synchronising s); kept factors stay.
size_t ctx_trim(geo_ctx *ctx, cudaStream_t s);
// Upper bound of the device bytes one geo_loglik call with these options may
// add to a context that holds no cached workspace.
size_t loglik_device_bytes(int device, int n, int p, const geo_opts *opts);

// ---- solve.cu -----------------------------------------------------------
// logdet = 2 sum log L_kk, quad = sum y_k^2 (y = row N of A), loglik = Eq. 1.
cudaError_t launch_loglik_reduce(const double *A, long long ld, int N, const double *y, long long ystride,
                                 const DevStatus *st, DevResults *res, cudaStream_t s);
// ---- trsv.cu --------------------------------------------------------------
// One-launch triangular solves with the column-major lower factor in A.
// sync: 4 device ints of scratch (zeroed here); timeout_word: NULL or the int
// that records a bounded wait that expired (the solve is then unfinished).
// x <- L^-1 x.
cudaError_t forward_solve(const double *A, long long ld, int N, double *x, int *sync, int *timeout_word,
                          cudaStream_t s);
// Forward solve with block 0 withheld (a dependency nothing satisfies) and a
// wait budget of wait_limit cycles: the bounded waits give up, record code 3
// in *timeout_word and the launch returns (self-test of the waits).
cudaError_t forward_solve_withheld(const double *A, long long ld, int N, double *x, int *sync, int *timeout_word,
                                   long long wait_limit, cudaStream_t s);
// w = L^-T y (y strided; w may be y's storage when ystride == 1).
cudaError_t backward_solve(const double *A, long long ld, int N, const double *y, long long ystride, double *w,
                           int *sync, int *timeout_word, cudaStream_t s);
// z = L e (lower-triangular matrix-vector product).
cudaError_t launch_trmv_lower(const double *A, long long ld, int N, const double *e, double *z, cudaStream_t s);

// ---- refine.cu ------------------------------------------------------------
size_t refine_workspace_bytes(int N);
// x = Sigma^-1 z by FP64 iterative refinement with the factor in A and the
// lower triangle of Sigma in S; writes l, log|Sigma|, z'x to res.
cudaError_t refine_solve(const double *S, const double *A, long long ld, int N, const double *z, const double *y,
                         long long ystride, int iters, double *x, void *ws, const DevStatus *st, DevResults *res,
                         cudaStream_t s);

// ---- batched.cu -----------------------------------------------------------
struct GemmDesc {           // C = alpha op(A) op(B) + beta C, column-major
    int m, n, k, ta, tb;
    const double *A;
    long long lda;
    const double *B;
    long long ldb;
    double *C;
    long long ldc;
    double alpha, beta;
};
struct QrDesc {             // in-place Householder QR of Y (m x r), thin Q out
    int m, r;
    double *Y;
    long long ldy;
    double *Q;
    long long ldq;
    double *tau, *v0;       // r entries each
};
struct SvdDesc {            // one-sided Jacobi SVD of M (r x r): M <- M V, V, sigma
    int r;
    double *M, *V;
    long long ld;
    double *sigma;
    double skip;            // pairs of columns both below this norm are left alone (0 = none)
};
// kmax: the largest K of the batch (0: no split-K).
cudaError_t launch_bgemm(const GemmDesc *d_desc, int count, int max_tiles, cudaStream_t s, double flops,
                         int kmax = 0);
// Scratch for the split-K partial tiles of this thread's launch_bgemm calls (NULL: none).
void bgemm_splitk_scratch(double *ws, size_t bytes);
constexpr size_t TLR_SPLITK_BYTES = 8u << 20;
// mmax, rmax: the largest m and r of the batch (the cluster kernel serves r <= 256).
cudaError_t launch_house_qr(const QrDesc *d_desc, int count, int mmax, int rmax, cudaStream_t s, double flops);
// rmax: the largest r of the batch (the cluster kernel serves r <= 256).
cudaError_t launch_jacobi_svd(const SvdDesc *d_desc, int count, int max_sweeps, int rmax, cudaStream_t s,
                              double flops);
cudaError_t launch_gaussian(double *O, long long n, unsigned long long seed, cudaStream_t s);

// ---- tlr.cu ---------------------------------------------------------------
constexpr int TLR_KCHUNK = 2048;            // stacked rank per update chunk
constexpr int TLR_MAXK_PER_CHUNK = 16;      // column tiles per update chunk
constexpr size_t TLR_ARENA_BYTES = 16u << 20;
struct TlrFactor {
    int dst = 0;               // > 0: keep only the dst tile diagonals nearest the diagonal, dense
    int N = 0, nb = 0, T = 0, kmax = 0;
    double tol = 0.0;
    double *D = nullptr;                    // T diagonal tiles nb x nb (ld nb), lower = L_tt
    // U and V of every off-diagonal tile live in pool segments (nb x rank each, ld nb);
    // a new segment is requested through grow() when the current one is full
    std::vector<std::pair<double *, size_t>> segs;   // (pointer, capacity in doubles)
    size_t seg_used = 0;                              // doubles used in the last segment
    std::function<double *(size_t)> grow;             // returns a segment of >= n doubles or nullptr
    std::vector<int> rank;                  // per slot(i, j) = i (i - 1) / 2 + j
    std::vector<double *> uptr, vptr;       // per slot
    std::vector<char> dense;                // per slot: stored dense (U = L_ij, V = I; rank = tile width)
    int capped = 0, max_rank = 0;           // capped = tiles stored dense (rank above kmax)
    double *Uof(size_t sl) const { return uptr[sl]; }
    double *Vof(size_t sl) const { return vptr[sl]; }
    double *take(size_t n) {
        if (segs.empty() || seg_used + n > segs.back().second) {
            double *p = grow ? grow(n) : nullptr;
            if (!p) return nullptr;
            seg_used = 0;
        }
        double *p = segs.back().first + seg_used;
        seg_used += (n + 31) / 32 * 32;
        return p;
    }
};
struct TlrR2Desc {
    int r;
    const double *B;
    long long ldb;
    double *M;
    long long ldm;
};
struct TlrSelDesc {
    int r, k;
    const double *M, *Vj;
    double *Msel, *Vsel;
    long long ld;
    const int *sel;
};
struct TlrTrsmDesc {
    const double *L;
    long long ldl;
    double *X;
    long long ldx;
    int ncols;
};
size_t tlr_factor_bytes(int N, int nb, int kmax);
size_t tlr_workspace_bytes(int N, int nb, int kmax);
size_t tlr_solve_workspace_bytes(int N, int nb, int kmax);
cudaError_t tlr_factor(TlrFactor &F, const CovParams &cp, const double *lx, const double *ly, void *ws,
                       size_t ws_bytes, void *arena_host, DevStatus *st, DevStatus *h_st, cudaStream_t s);
cudaError_t tlr_solve(const TlrFactor &F, double *x, bool transpose, void *ws, void *arena_host, cudaStream_t s);
cudaError_t tlr_reduce(const TlrFactor &F, const double *y, const DevStatus *st, DevResults *res, cudaStream_t s);

// ---- batch.cu -------------------------------------------------------------
size_t batch_desc_bytes();
void batch_fill_desc(void *hdesc, int k, double *A, long long ld, int N, int n, const double *locs, const double *z,
                     const CovParams &cp);
// Ticket table of the persistent launch (16 bytes per unit) for problems of orders N[0..count) and
// n[0..count) locations,
// ordered by a list-scheduling simulation on `workers` CTAs; returns the unit count, or minus it when
// out is NULL or cap (units) is too small.
int batch_units(const int *N, const int *n, int count, int workers, void *out, size_t cap);
// CTAs of the persistent launch.
int batch_workers();
// units: device ticket table, nunits: device int holding its length (read by the launch, so a captured
// sequence serves any table); counters: 4 + count device ints (zeroed by the sequence itself).
cudaError_t batch_record(void *ddesc, const void *units, const int *nunits, int *counters, int count, int nmax,
                         int Nmax, cudaStream_t s);
cudaError_t batch_results(const void *ddesc, void *hdesc, int count, double *loglik, int *info, cudaStream_t s);

// ---- host helpers (api.cu) ------------------------------------------------
int theta_to_params(const geo_theta *th, CovParams *cp, std::string *err);
void morton_perm_host(const double *locs, int n, int *perm);
