/*
 * geo.h -- C ABI of the GB300 library for the multivariate Matern Gaussian
 * log-likelihood and cokriging of arxiv 2008.07437, "High Performance
 * Multivariate Geospatial Statistics on Manycore Systems".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an int status (GEO_OK = 0 or a GEO_E* code).
 *   Nothing throws across the ABI and no kernel traps; the context keeps a
 *   human-readable message for the last failure (geo_last_error).
 * - "_dev" pointers are device memory owned by the caller (for example the
 *   data_ptr() of a torch tensor on the context's device); the library never
 *   frees them.  "_host" pointers are host memory owned by the caller.
 * - Locations are n x 2 row-major doubles (x_0, y_0, x_1, y_1, ...): points
 *   of [0, 1]^2 or of any bounded planar domain, Euclidean distance (d = 2).
 * - Vectors of observations use Representation I (Sec. 5.2): entry p*l + i is
 *   variable i at location l ("location-major, variable-minor").
 * - All device work is enqueued on the given stream (a cudaStream_t passed
 *   as void*, NULL = legacy default stream).  Functions that return a host
 *   scalar synchronise that stream before returning.
 * - Objects returned through out-pointers (geo_ctx, geo_factor) are owned by
 *   the library and released with geo_destroy / geo_factor_free.
 */
#ifndef GEO_H
#define GEO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
enum {
    GEO_OK = 0,
    GEO_EINVAL = 1,      /* bad argument: sizes, theta outside its domain, NULL pointer */
    GEO_ENOTSPD = 2,     /* Sigma(theta) not positive definite; *info = 1-based failing row */
    GEO_ENOMEM = 3,      /* the context's HBM budget (or the device) cannot hold the request */
    GEO_ETIMEOUT = 4,    /* a bounded device-side wait expired; the context stays usable */
    GEO_ECUDA = 5,       /* a CUDA runtime call failed; see geo_last_error */
    GEO_EUNSUPPORTED = 6, /* option combination not implemented */
    GEO_ESCRATCH = 7      /* geo_loglik_noalloc: p*n exceeds GEO_NOALLOC_MAX_N */
};

/* ---- factorisation forms (Sec. 5.2 exact, Sec. 5.3 TLR) ----------------- */
enum {
    GEO_PREC_FP64 = 0,   /* dense FP64 tiled Cholesky (exact computation) */
    GEO_PREC_MIXED = 1,  /* FP64 diagonal tiles, FP32 band, FP16/BF16 beyond (per-tile scale) */
    GEO_PREC_TLR = 2     /* tile low-rank off-diagonal tiles at accuracy tlr_tol */
};

#define GEO_PMAX 4       /* largest number of variables p */

/*
 * theta = (sigma^2_11..pp, a, nu_11..pp, beta) of the parsimonious
 * multivariate Matern model, Eq. 2 (Sec. 4.2).  All arrays are host memory.
 *   p       number of variables, 1 <= p <= GEO_PMAX
 *   sigma2  p marginal variances sigma^2_ii > 0
 *   nu      p marginal smoothness nu_ii > 0 (nu_ij = (nu_ii + nu_jj) / 2)
 *   beta    p*p row-major symmetric positive definite correlation matrix
 *           (its diagonal is read as 1); NULL is allowed when p == 1
 *   a       spatial range a > 0
 * rho_ij follows Sec. 4.2 with d = 2, reading the square roots as applying to
 * the marginal Gamma ratios, which gives rho_ii = 1.
 */
typedef struct {
    int p;
    const double *sigma2;
    const double *nu;
    const double *beta;
    double a;
} geo_theta;

/* Options of a likelihood evaluation.  geo_opts_default fills the defaults. */
typedef struct {
    int nb;             /* tile size of the tiled Cholesky (default 960) */
    int prec;           /* GEO_PREC_* (default GEO_PREC_FP64) */
    int band;           /* MIXED: tiles with 0 < |i - j| <= band stay FP32 (default 4) */
    int lowp;           /* MIXED: 0 = FP16 operands with a per-tile power-of-two scale, 1 = BF16 */
    int refine_iters;   /* MIXED: FP64 iterative-refinement sweeps on Sigma x = Z (default 2) */
    double tlr_tol;     /* TLR: absolute accuracy of each compressed tile (default 1e-9) */
    int tlr_kmax;       /* TLR: maximum tile rank (default 200) */
    int morton;         /* 1 = reorder locations by Morton (Z-order) key internally (default 1) */
    int fp64_gemm;      /* FP64 form, trailing updates (the SYRK / GEMM tasks of Sec. 5.1):
                           0 = native FP64 FMA (default); 1 = emulated on the BF16 tensor cores
                           (Ozaki scheme: each panel row split into oz_slices 7-bit integer digits
                           with a power-of-two row scale, digit products accumulated exactly in
                           FP32, recombined in 64-bit integers and FP64).  The rows below each
                           diagonal tile are solved the same way, as the product with the inverse
                           of the diagonal tile; POTRF and the inversion of the diagonal tiles, the
                           last panel and every other step stay native FP64.  nb must be a
                           multiple of 64 and at most 1024 (default 512). */
    int dst;            /* TLR form: > 0 = Diagonal Super Tile (Sec. 3.4), keep the dst tile diagonals
                           nearest the diagonal (1 = diagonal tiles only) dense and zero the other
                           tiles (of the Morton-ordered matrix); 0 = off (default) */
    int oz_slices;      /* fp64_gemm = 1: digits per operand, 3..8 (0 = 8).  An update then carries a
                           relative error of about 2^(-7 oz_slices) of max|a_r| max|b_c| per product
                           term (8 slices: below FP64's 2^-53 rounding; 5 slices: ~2^-35) */
    int oz_cut;         /* fp64_gemm = 1: 1 = magnitude-aware level cut in the trailing updates: an
                           output tile keeps only the digit levels whose products reach
                           2^-(7 oz_slices) of the update's largest products (from the per-row
                           exponents), so tiles of small entries (far from the diagonal) cost less
                           or nothing; every entry's error stays within that of the largest
                           products.  0 = every tile keeps all levels (default) */
    int reserved[4];
} geo_opts;

typedef struct geo_ctx geo_ctx;
typedef struct geo_factor geo_factor;

/* Fill *opts with the defaults listed above. */
void geo_opts_default(geo_opts *opts);

/*
 * Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context allocates for its own workspaces and factors (0 = no cap
 * beyond the device).  The context owns its workspaces; geo_destroy frees
 * them and every factor still alive.
 */
int geo_create(geo_ctx **ctx, int device, size_t hbm_budget_bytes);
int geo_destroy(geo_ctx *ctx);

/* Message of the last failed call on this context ("" if none); owned by the context. */
const char *geo_last_error(const geo_ctx *ctx);

/*
 * Cross-covariance matrix of Eq. 2 in Representation I (Sec. 5.2, Eq. 4):
 *   out[(p*r + j) * ld + (p*l + i)] = C_ij(|s1_l - s2_r|; theta)
 * i.e. column-major (p*n1) x (p*n2) with leading dimension ld >= p*n1.
 * locs2_dev == NULL means locs2 = locs1 (then Sigma itself, all entries).
 * h = 0 uses the limit rho_ij sigma_ii sigma_jj (no nugget).  The Bessel
 * function K_nu is evaluated in FP64 on the device.  No reordering.  The
 * call first builds the per-theta K_nu tables in a buffer of the context on
 * `stream`: calls on one context must not overlap on different streams.
 */
int geo_covgen(geo_ctx *ctx, const double *locs1_dev, int n1, const double *locs2_dev, int n2,
               const geo_theta *theta, double *out_dev, long long ld, void *stream);

/*
 * Gaussian log-likelihood, Eq. 1 (Sec. 1):
 *   l(theta) = -(N/2) log(2 pi) - 1/2 log|Sigma(theta)| - 1/2 Z' Sigma(theta)^-1 Z,  N = p n,
 * by covariance generation, tiled Cholesky, triangular solve and
 * log-determinant, all on the device.
 *   locs_dev     n x 2 locations (device)
 *   z_dev        N observations in Representation I (device)
 *   opts         NULL = defaults
 *   loglik_host  receives l (host); may be NULL
 *   keep         if non-NULL, receives a factor (L, L^-1 Z and the reordered
 *                locations) kept on the device for geo_predict; free with
 *                geo_factor_free.  NULL = discard.
 *   info         if non-NULL, receives 0 or, on GEO_ENOTSPD, the 1-based row
 *                (in the library's internal location order) of the first
 *                non-positive pivot.
 * Synchronises `stream`.
 */
int geo_loglik(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
               const geo_opts *opts, double *loglik_host, geo_factor **keep, int *info, void *stream);

/*
 * Marginal variances of the profile likelihood (Sec. 4.2):
 *   sigma2_host[i] = n^-1 Z_i' R_ii^-1 Z_i,  i = 0 .. p-1,
 * Z_i the n values of variable i (z_dev[l*p + i], Representation I) and R_ii
 * the correlation matrix of variable i alone (Eq. 2 with i = j,
 * sigma^2_ii = 1, smoothness nu_ii, range a).  theta->sigma2 and theta->beta
 * are not read.  Each R_ii is factored in the form opts selects (as
 * geo_loglik with p = 1); in the tile-low-rank form (and its DST variant) with
 * tiles of nb / p rows, so that they cover the same blocks of locations as the
 * tiles of Sigma.  sigma2_host: p doubles (host).  info as in
 * geo_loglik, for the first R_ii that is not positive definite.
 * Synchronises `stream`.
 */
int geo_sigma2_hat(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                   const geo_opts *opts, double *sigma2_host, int *info, void *stream);

/*
 * Profile log-likelihood (Sec. 4.2): Eq. 1 at theta with its marginal
 * variances replaced by geo_sigma2_hat.  The cost is one likelihood of size
 * p n and p of size n.  loglik_host, sigma2_host (p doubles): host, either may
 * be NULL.  Errors as geo_loglik.  Synchronises `stream`.
 */
int geo_loglik_profile(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                       const geo_opts *opts, double *loglik_host, double *sigma2_host, int *info, void *stream);

/*
 * Cokriging predictor, Eq. 3 / Eq. 4 (Sec. 4.3): for each of the m new
 * locations s0, Zhat(s0) = c0' Sigma^-1 Z, c0 the (p n) x p cross-covariance
 * between Z(s0) and the observed locations.  Every new location misses all p
 * variables.  Uses the factor kept by geo_loglik (its theta, L and L^-1 Z).
 *   new_locs_dev  m x 2 (device)
 *   zhat_dev      p*m outputs in Representation I, in the caller's order of
 *                 new locations (device)
 */
int geo_predict(geo_ctx *ctx, const geo_factor *factor, const double *new_locs_dev, int m, double *zhat_dev,
                void *stream);

/*
 * Batched cokriging (Eq. 3 / Eq. 4) on many factors kept by this context, in one launch: entry k
 * predicts the m[k] new locations new_locs_dev[k] (m[k] x 2, device) on
 * factors[k] into zhat_dev[k] (p m[k] doubles, device, Representation I),
 * exactly as geo_predict would (bit-identical).  Factors of any forms, sizes
 * and theta may be mixed; each factor's weights Sigma^-1 Z are computed on its
 * first prediction, as in geo_predict.  The work is enqueued on `stream`
 * (the descriptors are staged in pinned memory of the context: the call waits
 * for the stream's previous work before reusing them).  The zhat_dev buffers
 * must not overlap.  GEO_EINVAL for a bad entry (named in geo_last_error).
 */
int geo_predict_batch(geo_ctx *ctx, int count, const geo_factor *const *factors, const double *const *new_locs_dev,
                      const int *m, double *const *zhat_dev, void *stream);

/*
 * Synthetic draw Z = L e with L L' = Sigma(theta) (Sec. 6.4.1 synthetic data;
 * the paper does not state its generator): e_dev holds N standard normals
 * (device), z_dev receives N values in Representation I in the caller's
 * location order.  With opts->prec = GEO_PREC_MIXED, L is the mixed-precision
 * factor (a draw from N(0, L L') with L L' close to Sigma).  With the default
 * Morton reordering the draw differs from the one of the caller's order
 * (Cholesky factors of permuted matrices are not permutations of each other);
 * opts->morton = 0 reproduces L e in the caller's order.  Synchronises `stream`.
 */
int geo_simulate(geo_ctx *ctx, const double *locs_dev, int n, const double *e_dev, const geo_theta *theta,
                 const geo_opts *opts, double *z_dev, int *info, void *stream);

/* Summary of a kept factor. */
typedef struct {
    int n, p, N, nb, prec;
    double loglik, logdet, quad;   /* Eq. 1 and its two data-dependent terms */
    long long device_bytes;        /* device memory the factor holds */
    double tlr_bytes_ratio;        /* TLR: bytes of the compressed factor / dense bytes; else 1 */
    int tlr_max_rank, tlr_dense_tiles;
} geo_factor_stats;

int geo_factor_stats_get(const geo_factor *factor, geo_factor_stats *out);

/*
 * Copy part of a kept factor to host memory, in the library's internal
 * (reordered) index space:
 *   what = 0: the block L[r0:r1, c0:c1] of the Cholesky factor (row-major
 *             out, (r1-r0)*(c1-c0) doubles; entries above the diagonal are 0)
 *   what = 1: y = L^-1 Z, entries r0..r1-1
 *   what = 2: the location permutation, entries r0..r1-1 as doubles
 *             (internal location k is caller location perm[k])
 * Tile-low-rank factors (tiles of nb rows; tile (i, j), i > j, is U V'):
 *   what = 3: ranks of tiles (i, c0) for i = r0 .. r1-1 (-1 where i <= c0)
 *   what = 4: U of tile (r0, c0), rows of tile r0 x rank, column-major
 *   what = 5: V of tile (r0, c0), rows of tile c0 x rank, column-major
 *   what = 6: diagonal tile r0 of L, column-major (zeros above the diagonal)
 */
int geo_factor_read(const geo_factor *factor, int what, long long r0, long long r1, long long c0, long long c1,
                    double *host_out);

void geo_factor_free(geo_factor *factor);

/*
 * Morton (Z-order) permutation of n locations (Sec. 5.3): keys interleave the
 * two coordinates quantised to 16 bits over the square bounding box
 * [xmin, xmin + span]^2 (span = the larger extent), x on the even bits;
 * locations are sorted by (key, index).  Host memory in and out; perm_host
 * receives n indices (internal position k holds caller location perm[k]).
 */
int geo_morton_order(const double *locs_host, int n, int *perm_host);

/*
 * Layout check for bindings (host only, no device): writes up to n values to
 * out (host): the sizes in bytes of geo_theta, geo_opts, geo_factor_stats,
 * geo_mle_state, geo_batch_item, geo_request, geo_result and geo_kstat, then
 * the offsets of geo_opts.oz_slices, geo_opts.oz_cut and
 * geo_kstat.tensor_flops.  Returns the number of values the library has
 * (11), or GEO_EINVAL for a NULL out with n > 0.
 */
int geo_abi_layout(long long *out, int n);

/*
 * Maximum likelihood by the Nelder-Mead simplex method (the paper maximises
 * Eq. 1 with NLopt, Sec. 5.1; the algorithm is not named).  The state is a
 * plain host struct owned by the caller: it can be copied, saved and
 * restored, and geo_mle_step resumes from it.  Coordinates are
 * x = (log sigma^2_i, log a, log nu_i, beta_ij for i < j); a vertex whose
 * beta is not positive definite, or whose Sigma is not, scores +inf.
 */
#define GEO_MLE_QMAX 16
typedef struct {
    int p, q;                                  /* variables, coordinates */
    int iter, evals;                           /* iterations done, likelihood evaluations */
    int initialized;                           /* simplex values computed */
    double step;                               /* initial simplex step */
    double x[GEO_MLE_QMAX + 1][GEO_MLE_QMAX];  /* vertices, ordered best first once initialized */
    double f[GEO_MLE_QMAX + 1];                /* -l at each vertex */
    double last_f;                             /* -l of the last evaluation */
    int profile;                               /* 1 = profile likelihood (geo_mle_init_profile) */
    double s2[GEO_MLE_QMAX + 1][GEO_PMAX];     /* profile: sigma^2 estimate at each vertex */
} geo_mle_state;

/* Start a simplex at theta0 (host) with x0 + step * e_k as the other vertices. */
int geo_mle_init(geo_mle_state *state, const geo_theta *theta0, double step);

/*
 * The same over the profile likelihood (Sec. 4.2): coordinates
 * x = (log a, log nu_i, beta_ij for i < j), every evaluation is
 * geo_loglik_profile, and the marginal variances of a vertex are the
 * geo_sigma2_hat values at it (theta0->sigma2 is not read; it may be NULL).
 */
int geo_mle_init_profile(geo_mle_state *state, const geo_theta *theta0, double step);

/*
 * One unit of work: the q + 1 initial evaluations on the first call, one
 * Nelder-Mead iteration (reflection, expansion, contraction or shrink, with
 * coefficients 1, 2, 1/2, 1/2; vertices ordered by (value, index)) after.
 */
int geo_mle_step(geo_ctx *ctx, geo_mle_state *state, const double *locs_dev, int n, const double *z_dev,
                 const geo_opts *opts, void *stream);

/* Best vertex as theta: sigma2[p], a, nu[p], beta[p*p] (host; beta may be NULL).  For a
   profile run sigma2 is the sigma^2 estimate at the best vertex (NaN before the first
   geo_mle_step); loglik is NaN before the first step. */
int geo_mle_best(const geo_mle_state *state, double *sigma2, double *a, double *nu, double *beta,
                 double *loglik);

/*
 * Batched log-likelihoods of many small, uneven problems (Eq. 1 for each),
 * dense FP64, in the callers' location order.  One launch builds the K_nu
 * tables of every theta; one persistent launch does the rest for the whole
 * batch: its CTAs walk a table of units (a 64 x 64 block of location pairs of
 * Eq. 2, the POTRF of a 64-wide diagonal block, the TRSM of 128 rows below
 * it, a 128 x 64 tile of the trailing update, the reduction), each unit
 * waiting (bounded) on its problem's progress counter.  The table's order
 * comes from a list-scheduling simulation on the host (cached while the
 * problem sizes stay the same).  The launch sequence of a batch shape (count
 * and largest order) is captured once as a CUDA graph and replayed, with the
 * per-problem inputs, theta and units refreshed in device memory.  A
 * problem's result depends only on its own inputs: it is bit-identical alone
 * and in any batch.  GEO_ETIMEOUT if a bounded wait expired.
 *   items        count entries (host array); each names device inputs and a
 *                host theta, as for geo_loglik
 *   loglik_host  count results (host); NaN where Sigma is not positive definite
 *   info_host    NULL or count ints: 0 or the 1-based failing row
 * Synchronises `stream`.  Returns GEO_EINVAL for bad items (the first one is
 * named in geo_last_error), GEO_ENOMEM beyond the context's budget.
 */
typedef struct {
    const double *locs_dev;   /* n x 2 */
    int n;
    const double *z_dev;      /* p n, Representation I */
    geo_theta theta;
} geo_batch_item;

int geo_loglik_batch(geo_ctx *ctx, int count, const geo_batch_item *items, double *loglik_host, int *info_host,
                     void *stream);

/*
 * Prediction (cokriging) variances on a kept factor: the diagonal of
 * C(0) - c0' Sigma^-1 c0 at each new location s0, i.e. the mean square error
 * of the Eq. 3 predictor under the model (the E_t term of Eq. 5).
 *   new_locs_dev  m x 2 (device);  var_dev  p m doubles (device), Representation I
 * Dense FP64 or mixed factors: N^2 p m flops (a right-side triangular solve
 * of the m cross-covariances).  Tile-low-rank factors (and their DST form): one
 * TLR forward solve per column of c0, p m in all, with a stream synchronisation
 * after each.  Synchronises `stream`.
 */
int geo_predict_var(geo_ctx *ctx, const geo_factor *factor, const double *new_locs_dev, int m, double *var_dev,
                    void *stream);

/*
 * Multivariate MLOE / MMOM (Eq. 5 - Eq. 8, Algorithm 1 of Sec. 5.4): how much
 * cokriging with theta_a instead of the true theta_t loses in prediction
 * efficiency (LOE) and misstates the mean square prediction error (MOM),
 * averaged over m prediction locations s0:
 *   E_t  = tr{C(0; t) - c_t' S_t^-1 c_t}
 *   E_ta = tr{C(0; t) - 2 c_t' S_a^-1 c_a + c_a' S_a^-1 S_t S_a^-1 c_a}
 *   E_a  = tr{C(0; a) - c_a' S_a^-1 c_a}
 *   LOE = E_ta / E_t - 1,  MOM = E_a / E_ta - 1,  MLOE / MMOM = their means,
 * with S = Sigma(theta) at the observed locations and c the p n x p
 * cross-covariance with s0.  Dense FP64: both matrices are factored with the
 * cross-covariances of all m locations riding along as extra rows.
 *   locs_dev  n x 2, pred_dev m x 2 (device, caller-owned)
 *   theta_t, theta_a  host structs with the same p
 *   opts      NULL or options (nb, morton; the form is always FP64)
 *   mloe, mmom  host scalars; loe_host, mom_host  NULL or m doubles (host)
 * Synchronises `stream`.  GEO_ENOTSPD if either matrix is not positive
 * definite; GEO_ENOMEM beyond the budget (two N x (N + 2 p m) matrices).
 */
int geo_mloe_mmom(geo_ctx *ctx, const double *locs_dev, int n, const double *pred_dev, int m,
                  const geo_theta *theta_t, const geo_theta *theta_a, const geo_opts *opts, double *mloe,
                  double *mmom, double *loe_host, double *mom_host, void *stream);

/*
 * Request server: likelihood and cokriging requests of different sizes on one
 * GPU, admitted continuously (no paper counterpart: the paper evaluates one
 * likelihood at a time).  `slots` worker threads each own a context and a
 * CUDA stream, so concurrent requests overlap on the device.
 * Admission by device memory (hbm_budget_bytes, 0 = no budget): each worker's
 * footprint is what its context holds (cached workspaces, kept factors) plus
 * its staging buffers, and while it runs a request, plus an upper bound of
 * what the request may allocate.  A free worker takes the oldest queued
 * request for which the sum of the footprints stays within the budget,
 * dropping its own cached workspaces first if that makes it fit; idle workers
 * drop theirs while a request waits for memory.  A likelihood request whose
 * bound alone exceeds the budget is refused at submission with GEO_ENOMEM.
 * A likelihood request with keep = 1 leaves its factor on the device under
 * `dataset`; prediction requests for that key run on the worker that owns
 * the factor (after the likelihood has finished), and one with release = 1
 * frees it.  If that likelihood failed, its predictions finish with
 * GEO_EINVAL.  With escalate = 1, a mixed-precision or TLR likelihood that
 * finds its reduced-precision Sigma not positive definite is run again in
 * FP64 on the same worker; geo_result.prec gives the form that produced the
 * result.  Inputs are host memory and are copied at submission.
 * geo_server_pending reports the queued and running requests and the summed
 * footprint in bytes.
 */
enum { GEO_REQ_LOGLIK = 0, GEO_REQ_PREDICT = 1 };

typedef struct {
    int kind;                      /* GEO_REQ_LOGLIK or GEO_REQ_PREDICT */
    long long dataset;             /* key of a kept factor */
    int keep;                      /* LOGLIK: keep the factor under `dataset` */
    int release;                   /* PREDICT: free the factor after this request */
    int n;                         /* LOGLIK: locations */
    const double *locs_host;       /* LOGLIK: n x 2 */
    const double *z_host;          /* LOGLIK: p n, Representation I */
    geo_theta theta;               /* LOGLIK */
    const geo_opts *opts;          /* LOGLIK: NULL = defaults */
    int m;                         /* PREDICT: new locations */
    const double *new_locs_host;   /* PREDICT: m x 2 */
    int escalate;                  /* LOGLIK: on GEO_ENOTSPD in a reduced form, run again in FP64 */
} geo_request;

typedef struct {
    long long id, dataset;
    int kind, status;              /* status: GEO_OK or the error of the call */
    double loglik;                 /* LOGLIK */
    double t_submit, t_start, t_end;   /* seconds, steady clock */
    int prec;                      /* LOGLIK: GEO_PREC_* of the evaluation that produced the result */
} geo_result;

typedef struct geo_server geo_server;

int geo_server_create(geo_server **server, int device, size_t hbm_budget_bytes, int slots);
/* zhat_host: PREDICT output (p m doubles, host, caller-owned, valid until the result is polled) */
int geo_server_submit(geo_server *server, const geo_request *request, double *zhat_host, long long *id);
/* Up to max finished results; waits up to wait_ms for the first one. */
int geo_server_poll(geo_server *server, geo_result *out, int max, int *nout, int wait_ms);
int geo_server_pending(geo_server *server, int *queued, int *inflight, long long *reserved_bytes);
/* Drops queued requests, waits for running ones, frees everything. */
int geo_server_destroy(geo_server *server);

/*
 * Autotuner (no paper counterpart: the paper fixes its tile sizes by hand,
 * Sec. 6): times geo_loglik on the caller's problem for every candidate tile
 * size nb and, in the mixed form (opts->prec = GEO_PREC_MIXED), every
 * candidate FP32 band, and keeps the fastest.  Each candidate gets one
 * warm-up and `samples` timed evaluations (CUDA events on `stream`; 0 = 3);
 * its time is their median.  Candidates that are not valid for the form are
 * skipped.  The choice is cached for the whole process, per device, form
 * (FP64, FP64 with tensor-core updates, mixed, TLR) and order bucket (powers
 * of two of N): geo_loglik with opts->nb = 0 on any context of that device
 * takes the tuned nb and, in the mixed form, the tuned band (defaults when
 * nothing is cached: nb 960 FP64, 512 FP64 with tensor-core updates, 1024
 * mixed).  best_band receives -1 when the band was not tuned.
 */
int geo_autotune(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                 const geo_opts *base, const int *nb_candidates, int n_nb, const int *band_candidates, int n_band,
                 int samples, int *best_nb, int *best_band, double *best_ms, void *stream);
/* geo_autotune over tile sizes only, 3 samples per candidate. */
int geo_autotune_nb(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                    const geo_opts *base, const int *candidates, int ncand, int *best_nb, double *best_ms,
                    void *stream);

/*
 * FP64-accurate matrix product on the tensor cores (the emulated trailing
 * update of fp64_gemm = 1 as a standalone operation; the paper's GEMM tile task
 * of Sec. 5.1 computes C -= A B' in FP64):
 *   C -= A B',  A m x k, B n x k, C m x n, all column-major FP64 device memory
 *   (caller-owned; lda >= m, ldb >= n, ldc >= m).
 * Each row of A and of B is split into `slices` (3..8, 0 = 8) BF16 digits of 7
 * bits under a power-of-two row scale; digit products are accumulated without
 * rounding on the tensor cores in chunks of k <= 4096 / slices and recombined
 * exactly in 64-bit integers, then added to C in FP64.  The error of each
 * entry is at most about (k + 1) 2^(1 - 7 slices) max_i |A[r, i]| max_i |B[c, i]|
 * (2^-53-class for 8 slices) plus the rounding of the FP64 additions to C.
 * Uses a workspace of the context (S (m + n) k 2 bytes).  Synchronises `stream`.
 * GEO_EINVAL for bad sizes or slices, GEO_ETIMEOUT if a bounded device wait
 * expired.
 */
int geo_gemm_f64e(geo_ctx *ctx, int m, int n, int k, const double *A_dev, long long lda, const double *B_dev,
                  long long ldb, double *C_dev, long long ldc, int slices, void *stream);

/*
 * Self-test of the bounded device waits (no paper counterpart; failure
 * handling).  Every spin-wait of the library's kernels on another block's
 * progress is bounded: when its clock budget runs out the kernel records the
 * wait site in the context's status word, raises an abort word so that the
 * other waiters give up too, and returns, leaving the context usable.  This
 * entry point makes that happen on purpose: it runs the one-launch forward
 * triangular solve on an identity factor of order 64 n_blocks with the first
 * block withheld (the ticket counter starts past it, so the completion the
 * second block waits for is never published) and a wait budget of
 * wait_cycles clock cycles (1 .. 4e9).  Returns GEO_ETIMEOUT with *site = 3
 * (the forward solve's wait) when the waits gave up as designed, GEO_OK if no
 * wait expired (which would mean the dependency was not withheld).  The
 * context's status words are cleared afterwards.  Synchronises `stream`.
 */
int geo_selftest_bounded_wait(geo_ctx *ctx, int n_blocks, long long wait_cycles, int *site, void *stream);

/*
 * Device-time profile per kernel class, measured with CUDA events recorded
 * on the stream each kernel is launched on (no paper counterpart: the
 * paper's timing is wall-clock per phase, Sec. 6.1 / Sec. 6.3).
 *   geo_profile_enable(ctx, 1) clears the counters and starts recording events
 *   around every launch; 0 stops recording (launch counting never stops).
 *   geo_profile_read synchronises the device, resolves the recorded events
 *   and fills out[0 .. GEO_K_COUNT-1]; flops / bytes are the algorithmic
 *   work of the launches (lower-triangle flops for the Cholesky updates).
 */
enum {
    GEO_K_COVGEN = 0,   /* Eq. 2 matrix generation */
    GEO_K_POTRF = 1,    /* diagonal-block Cholesky */
    GEO_K_TRSM = 2,     /* panel triangular solves */
    GEO_K_GEMM = 3,     /* trailing / panel updates (SYRK + GEMM) */
    GEO_K_REDUCE = 4,   /* log-determinant and quadratic form */
    GEO_K_SOLVE = 5,    /* backward substitution L' w = y */
    GEO_K_PREDICT = 6,  /* fused cross-covariance + GEMV of Eq. 3 */
    GEO_K_AUX = 7,      /* gathers, scatters, conversions */
    GEO_K_TCGEMM = 8,   /* tensor-core (tcgen05) updates: far tiles of the mixed form, and every
                           trailing update of the emulated FP64 form (flops counted as FP64 flops) */
    GEO_K_SGEMM = 9,    /* FP32 SIMT updates (mixed precision: diagonal and band tiles, panel) */
    GEO_K_TLR = 10,     /* TLR compression: Householder QR and Jacobi SVD of sketched tiles */
    GEO_K_COUNT = 11
};
typedef struct {
    long long launches;
    double ms;        /* summed device time of the launches that were timed */
    double flops;     /* algorithmic floating-point operations */
    double bytes;     /* algorithmic HBM bytes */
    long long timed;  /* launches with events */
    double tensor_flops; /* GEO_K_TCGEMM: BF16 tensor-core flops the emulated products issued (counted
                            on the device; the level cut lowers it), 0 for the other classes */
} geo_kstat;

int geo_profile_enable(geo_ctx *ctx, int enable);
int geo_profile_read(geo_ctx *ctx, geo_kstat *out);
/* Kernel counters summed over a server's worker contexts (launch counts
 * always; times only where profiling was on).  out: GEO_K_COUNT entries.
 * GEO_EINVAL while requests are queued or running. */
int geo_server_profile_read(geo_server *server, geo_kstat *out);

/*
 * geo_loglik_noalloc -- the log-likelihood of geo_loglik for small problems,
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; this is a deployment variant.
 *
 * Some callers cannot call cudaMalloc: a host application or framework that
 * reserved the GPU's memory for its own allocator up front (a cudaMalloc from
 * this library would then fail or fragment that pool), or a latency-critical
 * loop that cannot afford cudaMalloc / cudaFree, which may synchronise the
 * device and may fail at unpredictable times.  This entry point allocates
 * nothing and needs no context: every intermediate (the covariance matrix and
 * its factor, the locations in SoA form in the caller's order, the K_nu tables
 * of theta, the status words) lives in one fixed-size array in device global memory owned by the
 * library, about GEO_NOALLOC_SCRATCH_DOUBLES * 8 bytes (34 MB), which every
 * GPU that loads the library holds until the process exits.
 *
 *   locs_dev  n x 2 locations (device, caller-owned); used in the caller's order
 *   z_dev     N = p*n observations in Representation I (device)
 *   theta     host struct as for geo_loglik
 *   nb        tile size (>= 64)
 *   out_dev   3 doubles (device, caller-owned): l(theta), log|Sigma|, Z' Sigma^-1 Z;
 *             l is NaN when Sigma is not positive definite
 *   info_dev  NULL or one int (device): 0, or the 1-based failing row
 * Every buffer must be device memory of the current device (the call has no
 * context of its own and does not switch devices); other pointers are refused
 * with GEO_EINVAL before anything is enqueued.
 * The work is only enqueued on `stream`: synchronise it before reading the
 * outputs.  Returns GEO_ESCRATCH when p*n > GEO_NOALLOC_MAX_N (the scratch is
 * too small), GEO_EINVAL for other bad arguments, GEO_ECUDA if a launch or the
 * scratch set-up fails.  The first call on each device looks up the device
 * address of the scratch array (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  All calls share
 * the one array, which keeps the previous call's contents (the status words are
 * cleared at the start of each call): calls that overlap on the GPU race, so
 * serialise them (one stream, one thread).  The address is cached for the
 * life of the process: a call after cudaDeviceReset on that device is not
 * supported.
 */
#define GEO_NOALLOC_MAX_N 2048
#define GEO_NOALLOC_SCRATCH_DOUBLES 4267778LL
int geo_loglik_noalloc(const double *locs_dev, int n, const double *z_dev, const geo_theta *theta, int nb,
                       double *out_dev, int *info_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GEO_H */
