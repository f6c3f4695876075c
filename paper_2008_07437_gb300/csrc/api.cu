// C ABI of libgeo.so (declared in include/geo.h): argument checking, theta
// constants, Morton ordering, memory under the context's HBM budget, and the
// stream-ordered pipelines of geo_loglik / geo_predict / geo_simulate /
// geo_mle_step.  All arithmetic of the likelihood runs in the CUDA kernels;
// this file only prepares per-theta constants (p(p+1)/2 triples) and moves
// scalars.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <cstdio>
#include <map>
#include <mutex>
#include <tuple>
#include <numeric>
#include <stdexcept>
#include <string>
#include <vector>

#include "geo_internal.cuh"

// ---------------------------------------------------------------------------
// Context, factor
// ---------------------------------------------------------------------------
struct geo_ctx {
    int device = 0;
    size_t budget = 0;      // 0 = no cap
    size_t used = 0;
    std::string err;
    DevStatus *st = nullptr;
    DevResults *res = nullptr;
    int *sync = nullptr;          // 4 ints: sync words of the one-launch triangular solves
    DevStatus *h_st = nullptr;    // pinned
    DevResults *h_res = nullptr;  // pinned
    // reusable workspace for the matrix of a discarded evaluation
    double *ws = nullptr;
    size_t ws_bytes = 0;
    // workspace of the mixed-precision factorisation (panel copies)
    void *mws = nullptr;
    size_t mws_bytes = 0;
    // digit slices of the tensor-core FP64 emulation (fp64_gemm = 1)
    void *ows = nullptr;
    size_t ows_bytes = 0;
    // iterative refinement: copy of Sigma, sorted Z, partial sums
    void *sws = nullptr, *zws = nullptr, *rws = nullptr;
    size_t sws_bytes = 0, zws_bytes = 0, rws_bytes = 0;
    // TLR workspace (device) and descriptor staging (pinned host)
    void *tws = nullptr, *tarena = nullptr;
    size_t tws_bytes = 0, tarena_bytes = 0;
    // batched likelihoods: matrices, descriptors (device + pinned host), captured graphs
    void *bws = nullptr, *bdesc_d = nullptr, *bdesc_h = nullptr;
    size_t bws_bytes = 0, bdesc_cap = 0;
    std::map<std::tuple<int, int, int>, std::pair<cudaGraphExec_t, long long>> graphs;   // -> (exec, kernel nodes)
    std::vector<int> border;            // problem orders of the cached ticket table
    // batched predictions: descriptors (device + pinned staging)
    void *pdesc_d = nullptr, *pdesc_h = nullptr;
    size_t pdesc_cap = 0;
    std::vector<unsigned char> bunits;  // cached ticket table (16 bytes per unit)
    cudaStream_t cap_stream = nullptr;   // private stream for graph capture (the legacy stream cannot capture)
    std::vector<geo_factor *> factors;
    // K_nu tables of the theta of the last geo_covgen call
    double *ctab = nullptr;
    Profiler prof;
};

struct geo_factor {
    geo_ctx *ctx = nullptr;
    int n = 0, p = 0, N = 0, nb = 0, prec = GEO_PREC_FP64;
    long long ld = 0;
    double *A = nullptr;    // L (lower) with y' in row N
    size_t A_bytes = 0;
    double *lx = nullptr, *ly = nullptr;   // locations in internal order (SoA)
    double *w = nullptr;                   // L^-T y (lazy)
    std::vector<int> perm;                 // internal k -> caller location perm[k]
    CovParams cp;
    double loglik = 0, logdet = 0, quad = 0;
    // tile-low-rank form
    TlrFactor *tlr = nullptr;
    size_t tlr_bytes = 0;
    double *ybuf = nullptr;                // L^-1 Z (TLR form)
};

thread_local Profiler *t_prof = nullptr;

cudaEvent_t Profiler::take() {
    if (pool_used == pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        pool.push_back(e);
    }
    return pool[pool_used++];
}

void Profiler::resolve() {
    for (const Rec &r : recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.cls] += t;
            timed[r.cls] += 1;
        }
    }
    recs.clear();
    pool_used = 0;
}

void Profiler::clear() {
    recs.clear();
    pool_used = 0;
    for (int k = 0; k < GEO_K_COUNT; ++k) launches[k] = timed[k] = 0, flops[k] = bytes[k] = ms[k] = 0.0;
}

KScope::KScope(int cls_, cudaStream_t s_, double fl, double by) : p(t_prof), cls(cls_), s(s_) {
    if (!p) return;
    p->launches[cls] += 1;
    p->flops[cls] += fl;
    p->bytes[cls] += by;
    if (p->enabled) {
        a = p->take();
        if (a) cudaEventRecord(a, s);
    }
}

KScope::~KScope() {
    if (!p || !a) return;
    cudaEvent_t b = p->take();
    if (!b) return;
    cudaEventRecord(b, s);
    p->recs.push_back({cls, a, b});
}

// Points t_prof at a context's profiler for the duration of an API call.
struct ProfBind {
    Profiler *prev;
    explicit ProfBind(Profiler *p) : prev(t_prof) { t_prof = p; }
    ~ProfBind() { t_prof = prev; }
};

namespace {

int fail(geo_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

int cuda_fail(geo_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, GEO_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return cuda_fail(ctx, _e, #call);   \
    } while (0)

int dev_alloc(geo_ctx *ctx, void **ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return GEO_OK;
    if (ctx->budget && ctx->used + bytes > ctx->budget)
        return fail(ctx, GEO_ENOMEM, "HBM budget exceeded: need " + std::to_string(bytes) + " bytes, " +
                                         std::to_string(ctx->budget - ctx->used) + " left");
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return fail(ctx, GEO_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    ctx->used += bytes;
    return GEO_OK;
}

void dev_free(geo_ctx *ctx, void *ptr, size_t bytes) {
    if (!ptr) return;
    cudaFree(ptr);
    ctx->used -= bytes;
}

struct SetDevice {
    int prev = -1;
    explicit SetDevice(int d) {
        cudaGetDevice(&prev);
        if (prev != d) cudaSetDevice(d);
    }
    ~SetDevice() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

// Tile sizes (and, for the mixed form, FP32 bands) picked by the autotuner,
// shared by every context of the process: (device, form, floor(log2 N)) ->
// (nb, band); band < 0 when it was not tuned.
struct Tuned {
    int nb, band;
};
std::mutex g_tuned_mu;
std::map<std::tuple<int, int, int>, Tuned> g_tuned;

int order_bucket(int N) {
    int b = 0;
    while ((1 << (b + 1)) <= N) ++b;
    return b;
}

// Form key of the tuned-tile cache: the precision mode, or FORM_F64E for the
// FP64 form with tensor-core emulated updates (a different best tile size).
constexpr int FORM_F64E = 16;
int form_of(const geo_opts &o) { return (o.prec == GEO_PREC_FP64 && o.fp64_gemm == 1) ? FORM_F64E : o.prec; }

int resolve_nb(int device, int form, int N) {
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(std::make_tuple(device, form, order_bucket(N)));
    if (it != g_tuned.end()) return it->second.nb;
    return form == GEO_PREC_MIXED ? 1024 : form == FORM_F64E ? 512 : 960;
}

// nb = 0 in the options: the tuned tile size, and for the mixed form the tuned band.
void resolve_tuned(int device, int N, geo_opts *o) {
    const int form = form_of(*o);
    o->nb = resolve_nb(device, form, N);
    if (o->prec != GEO_PREC_MIXED) return;
    std::lock_guard<std::mutex> lk(g_tuned_mu);
    auto it = g_tuned.find(std::make_tuple(device, form, order_bucket(N)));
    if (it != g_tuned.end() && it->second.band >= 0) o->band = it->second.band;
}

int oz_slices_of(const geo_opts &o) { return o.oz_slices > 0 ? o.oz_slices : 8; }

// Grow a context-cached device buffer to at least `need` bytes.
int ensure_buffer(geo_ctx *ctx, void **buf, size_t *have, size_t need, cudaStream_t s) {
    if (*have >= need) return GEO_OK;
    if (*buf) {
        cudaStreamSynchronize(s);
        dev_free(ctx, *buf, *have);
        *buf = nullptr;
        *have = 0;
    }
    int rc = dev_alloc(ctx, buf, need);
    if (rc) return rc;
    *have = need;
    return GEO_OK;
}

// G1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu), G2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2.
// Near mu = 0 the difference cancels: G1 is even in mu and equals
// -(a2 + a4 mu^2 + a6 mu^4 + ...), a_k the Taylor coefficients of 1/Gamma(z).
void temme_gammas(double mu, double *g1, double *g2, double *gp, double *gm, double *fact) {
    const long double m = mu;
    const long double rp = 1.0L / tgammal(1.0L + m), rm = 1.0L / tgammal(1.0L - m);
    *gp = (double)tgammal(1.0L + m);
    *gm = (double)tgammal(1.0L - m);
    *g2 = (double)(0.5L * (rm + rp));
    if (fabsl(m) < 1e-3L) {
        const double u = mu * mu;
        // a2 = Euler's constant; a4, a6 of the series of 1/Gamma(z)
        *g1 = -(0.5772156649015328606 + u * (-0.042002635034095235529 + u * (-0.04219773455554433675)));
    } else {
        *g1 = (double)((rm - rp) / (2.0L * m));
    }
    const long double pi = 3.141592653589793238462643383279502884L;
    *fact = (mu == 0.0) ? 1.0 : (double)(m * pi / sinl(m * pi));
}

}  // namespace

// theta -> per-(i, j) constants of Eq. 2.  rho_ij (Sec. 4.2, d = 2):
//   rho_ij = beta_ij sqrt(G(nu_i + 1)/G(nu_i)) sqrt(G(nu_j + 1)/G(nu_j)) G(nu_ij)/G(nu_ij + 1).
int theta_to_params(const geo_theta *th, CovParams *cp, std::string *err) {
    if (!th) {
        *err = "theta is NULL";
        return GEO_EINVAL;
    }
    const int p = th->p;
    if (p < 1 || p > GEO_PMAX) {
        *err = "theta.p must be in 1.." + std::to_string(GEO_PMAX);
        return GEO_EINVAL;
    }
    if (!th->sigma2 || !th->nu || (p > 1 && !th->beta)) {
        *err = "theta arrays must not be NULL";
        return GEO_EINVAL;
    }
    if (!(th->a > 0.0) || !isfinite(th->a)) {
        *err = "theta.a must be > 0";
        return GEO_EINVAL;
    }
    for (int i = 0; i < p; ++i) {
        if (!(th->sigma2[i] > 0.0) || !isfinite(th->sigma2[i])) {
            *err = "theta.sigma2 must be > 0";
            return GEO_EINVAL;
        }
        if (!(th->nu[i] > 0.0) || !(th->nu[i] < 50.0)) {
            *err = "theta.nu must be in (0, 50)";
            return GEO_EINVAL;
        }
    }
    // beta: symmetric, unit diagonal (implied), positive definite
    double B[GEO_PMAX][GEO_PMAX];
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) {
            if (i == j) {
                B[i][j] = 1.0;
                continue;
            }
            const double b = th->beta[i * p + j];
            if (!isfinite(b) || b != th->beta[j * p + i]) {
                *err = "theta.beta must be finite and symmetric";
                return GEO_EINVAL;
            }
            B[i][j] = b;
        }
    {
        double L[GEO_PMAX][GEO_PMAX] = {};
        for (int j = 0; j < p; ++j) {
            double s = B[j][j];
            for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
            if (!(s > 0.0)) {
                *err = "theta.beta is not positive definite";
                return GEO_EINVAL;
            }
            L[j][j] = sqrt(s);
            for (int i = j + 1; i < p; ++i) {
                double t = B[i][j];
                for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
                L[i][j] = t / L[j][j];
            }
        }
    }
    memset(cp, 0, sizeof(*cp));
    cp->p = p;
    cp->inv_a = 1.0 / th->a;
    for (int i = 0; i < p; ++i) {
        for (int j = 0; j < p; ++j) {
            MaternConst &c = cp->m[i * p + j];
            const double nui = th->nu[i], nuj = th->nu[j];
            const double nij = 0.5 * (nui + nuj);
            const long double ri = tgammal((long double)nui + 1.0L) / tgammal((long double)nui);
            const long double rj = tgammal((long double)nuj + 1.0L) / tgammal((long double)nuj);
            const long double rho = (long double)B[i][j] * sqrtl(ri) * sqrtl(rj) * tgammal((long double)nij) /
                                    tgammal((long double)nij + 1.0L);
            const long double c0 = rho * sqrtl((long double)th->sigma2[i]) * sqrtl((long double)th->sigma2[j]);
            c.nu = nij;
            c.c0 = (double)c0;
            c.pre = (double)(c0 / (powl(2.0L, (long double)nij - 1.0L) * tgammal((long double)nij)));
            const int nl = (int)floor(nij + 0.5);
            c.nl = nl;
            c.mu = nij - nl;
            temme_gammas(c.mu, &c.g1, &c.g2, &c.gp, &c.gm, &c.fact);
            c.kind = (nij == 0.5) ? 1 : (nij == 1.5) ? 2 : (nij == 2.5) ? 3 : 0;
            c.toff = -1;
        }
    }
    // K_nu tables for the general orders nu_ij <= GEO_CHEB_NU_MAX, one per i <= j
    int g = 0;
    for (int i = 0; i < p; ++i)
        for (int j = i; j < p; ++j) {
            MaternConst &c = cp->m[i * p + j];
            if (c.kind == 0 && c.nu <= GEO_CHEB_NU_MAX) c.toff = (g++) * GEO_TAB_PER_PAIR;
            cp->m[j * p + i].toff = c.toff;
        }
    cp->tab = nullptr;
    return GEO_OK;
}

// Morton order: 16-bit quantisation over the square bounding box, x bits on
// the even positions, sort by (key, index).
void morton_perm_host(const double *locs, int n, int *perm) {
    if (n <= 0) return;
    double xmin = locs[0], xmax = locs[0], ymin = locs[1], ymax = locs[1];
    for (int k = 1; k < n; ++k) {
        xmin = std::min(xmin, locs[2 * k]);
        xmax = std::max(xmax, locs[2 * k]);
        ymin = std::min(ymin, locs[2 * k + 1]);
        ymax = std::max(ymax, locs[2 * k + 1]);
    }
    const double span = std::max(xmax - xmin, ymax - ymin);
    auto spread = [](uint32_t v) {
        uint32_t out = 0;
        for (int b = 0; b < 16; ++b) out |= ((v >> b) & 1u) << (2 * b);
        return out;
    };
    std::vector<uint32_t> key(n);
    for (int k = 0; k < n; ++k) {
        long long qx = 0, qy = 0;
        if (span > 0.0) {
            qx = (long long)floor((locs[2 * k] - xmin) / span * 65536.0);
            qy = (long long)floor((locs[2 * k + 1] - ymin) / span * 65536.0);
        }
        qx = std::min(std::max(qx, 0LL), 65535LL);
        qy = std::min(std::max(qy, 0LL), 65535LL);
        key[k] = spread((uint32_t)qx) | (spread((uint32_t)qy) << 1);
    }
    std::iota(perm, perm + n, 0);
    std::stable_sort(perm, perm + n, [&](int a, int b) { return key[a] < key[b]; });
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void geo_opts_default(geo_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->nb = 960;
    o->prec = GEO_PREC_FP64;
    o->band = 4;
    o->lowp = 0;
    o->refine_iters = 2;
    o->tlr_tol = 1e-9;
    o->tlr_kmax = 200;
    o->morton = 1;
    o->fp64_gemm = 0;
}

int geo_create(geo_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return GEO_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return GEO_ECUDA;
    }
    if (device < 0 || device >= ndev) return GEO_EINVAL;
    geo_ctx *ctx = new geo_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    SetDevice sd(device);
    if (cudaMalloc(&ctx->st, sizeof(DevStatus)) != cudaSuccess ||
        cudaMalloc(&ctx->res, sizeof(DevResults)) != cudaSuccess ||
        cudaMalloc(&ctx->sync, 4 * sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_st, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_res, sizeof(DevResults)) != cudaSuccess ||
        cudaMalloc(&ctx->prof.d_tc_flops, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(ctx->prof.d_tc_flops, 0, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        geo_destroy(ctx);
        return GEO_ECUDA;
    }
    *out = ctx;
    return GEO_OK;
}

int geo_destroy(geo_ctx *ctx) {
    if (!ctx) return GEO_OK;
    SetDevice sd(ctx->device);
    cudaDeviceSynchronize();
    while (!ctx->factors.empty()) geo_factor_free(ctx->factors.back());
    for (cudaEvent_t e : ctx->prof.pool) cudaEventDestroy(e);
    if (ctx->prof.d_tc_flops) cudaFree(ctx->prof.d_tc_flops);
    if (ctx->ws) dev_free(ctx, ctx->ws, ctx->ws_bytes);
    if (ctx->mws) dev_free(ctx, ctx->mws, ctx->mws_bytes);
    if (ctx->ows) dev_free(ctx, ctx->ows, ctx->ows_bytes);
    if (ctx->sws) dev_free(ctx, ctx->sws, ctx->sws_bytes);
    if (ctx->zws) dev_free(ctx, ctx->zws, ctx->zws_bytes);
    if (ctx->rws) dev_free(ctx, ctx->rws, ctx->rws_bytes);
    if (ctx->tws) dev_free(ctx, ctx->tws, ctx->tws_bytes);
    if (ctx->tarena) cudaFreeHost(ctx->tarena);
    if (ctx->ctab) dev_free(ctx, ctx->ctab, sizeof(double) * GEO_TAB_DOUBLES);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second.first);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->bws) dev_free(ctx, ctx->bws, ctx->bws_bytes);
    if (ctx->bdesc_d) cudaFree(ctx->bdesc_d);
    if (ctx->bdesc_h) cudaFreeHost(ctx->bdesc_h);
    if (ctx->pdesc_d) cudaFree(ctx->pdesc_d);
    if (ctx->pdesc_h) cudaFreeHost(ctx->pdesc_h);
    if (ctx->st) cudaFree(ctx->st);
    if (ctx->res) cudaFree(ctx->res);
    if (ctx->sync) cudaFree(ctx->sync);
    if (ctx->h_st) cudaFreeHost(ctx->h_st);
    if (ctx->h_res) cudaFreeHost(ctx->h_res);
    delete ctx;
    return GEO_OK;
}

const char *geo_last_error(const geo_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int geo_covgen(geo_ctx *ctx, const double *locs1_dev, int n1, const double *locs2_dev, int n2,
               const geo_theta *theta, double *out_dev, long long ld, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    CovParams cp;
    std::string err;
    int rc = theta_to_params(theta, &cp, &err);
    if (rc) return fail(ctx, rc, err);
    if (n1 < 0 || (locs2_dev && n2 < 0)) return fail(ctx, GEO_EINVAL, "negative size");
    if (!locs2_dev) n2 = n1;
    if (ld < (long long)cp.p * n1) return fail(ctx, GEO_EINVAL, "ld < p * n1");
    if ((n1 > 0 && (!locs1_dev || !out_dev))) return fail(ctx, GEO_EINVAL, "NULL pointer");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n1 == 0 || n2 == 0) return GEO_OK;
    if (!ctx->ctab && cov_needs_tables(cp)) {
        void *pt;
        if ((rc = dev_alloc(ctx, &pt, sizeof(double) * GEO_TAB_DOUBLES))) return rc;
        ctx->ctab = (double *)pt;
    }
    CK(launch_cheb_build(cp, ctx->ctab, s));
    CK(launch_covgen_rect(cp, locs1_dev, n1, locs2_dev ? locs2_dev : locs1_dev, n2, out_dev, ld, s));
    return GEO_OK;
}

// Shared front half of loglik / simulate: order locations, generate Sigma.
// Checks of the dense-form options shared by the entry points.
static int check_dense_opts(geo_ctx *ctx, const geo_opts &o) {
    if (o.fp64_gemm != 0 && o.fp64_gemm != 1) return fail(ctx, GEO_EINVAL, "fp64_gemm must be 0 or 1");
    if (o.fp64_gemm == 1 && (o.oz_slices != 0 && (o.oz_slices < 3 || o.oz_slices > 8)))
        return fail(ctx, GEO_EINVAL, "oz_slices must be 0 (default 8) or 3..8");
    if (o.oz_cut != 0 && o.oz_cut != 1) return fail(ctx, GEO_EINVAL, "oz_cut must be 0 or 1");
    if (o.fp64_gemm == 1 && (o.nb % 64 != 0 || o.nb > 1024))
        return fail(ctx, GEO_EINVAL, "fp64_gemm = 1 needs nb a multiple of 64, at most 1024");
    return GEO_OK;
}

// Dense FP64 factorisation in the form the options select: native FP64 FMA
// updates (chol64_factor) or tensor-core emulated ones (chol_oz_factor, with
// the context's slice workspace grown as needed).
static int dense_factor(geo_ctx *ctx, double *A, long long ld, int N, int nrows, const geo_opts &o, cudaStream_t s,
                        cudaError_t *err) {
    *err = cudaSuccess;
    if (o.fp64_gemm != 1) {
        *err = chol64_factor(A, ld, N, nrows, o.nb, ctx->st, s);
        return GEO_OK;
    }
    const int S = oz_slices_of(o);
    int rc = ensure_buffer(ctx, &ctx->ows, &ctx->ows_bytes, oz_chol_workspace_bytes(nrows, o.nb, S), s);
    if (rc) return rc;
    *err = chol_oz_factor(A, ld, N, nrows, o.nb, S, o.oz_cut, ctx->ows, ctx->ows_bytes, ctx->st, s);
    return GEO_OK;
}

static int prepare_matrix(geo_ctx *ctx, const double *locs_dev, int n, const geo_theta *theta,
                          const geo_opts *o, int extra_rows, geo_factor *f, cudaStream_t s, bool with_matrix = true) {
    std::string err;
    int rc = theta_to_params(theta, &f->cp, &err);
    if (rc) return fail(ctx, rc, err);
    const int p = theta->p;
    f->n = n;
    f->p = p;
    f->N = p * n;
    f->nb = o->nb;
    f->prec = o->prec;
    f->ld = round_up((long long)f->N + extra_rows, 32);
    // location order
    std::vector<double> h_locs((size_t)2 * n);
    CK(cudaMemcpyAsync(h_locs.data(), locs_dev, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < 2 * n; ++k)
        if (!isfinite(h_locs[k])) return fail(ctx, GEO_EINVAL, "non-finite location");
    f->perm.resize(n);
    if (o->morton)
        morton_perm_host(h_locs.data(), n, f->perm.data());
    else
        std::iota(f->perm.begin(), f->perm.end(), 0);
    // device buffers: locations (SoA) + permutation
    void *p1, *p2;
    if ((rc = dev_alloc(ctx, &p1, sizeof(double) * (2 * (size_t)n + GEO_TAB_DOUBLES)))) return rc;
    f->lx = (double *)p1;
    f->ly = f->lx + n;
    CK(launch_cheb_build(f->cp, f->lx + 2 * (size_t)n, s));   // K_nu tables after the locations
    if ((rc = dev_alloc(ctx, &p2, sizeof(int) * n))) return rc;
    int *d_perm = (int *)p2;
    CK(cudaMemcpyAsync(d_perm, f->perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s));
    CK(launch_gather_locs(locs_dev, d_perm, n, f->lx, f->ly, s));
    if (!with_matrix) {
        CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s));
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, d_perm, sizeof(int) * n);
        return GEO_OK;
    }
    // matrix
    const size_t bytes = sizeof(double) * (size_t)f->ld * (size_t)f->N;
    if (ctx->ws && ctx->ws_bytes >= bytes) {
        f->A = ctx->ws;
        f->A_bytes = ctx->ws_bytes;
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    } else {
        if (ctx->ws) {
            CK(cudaStreamSynchronize(s));
            dev_free(ctx, ctx->ws, ctx->ws_bytes);
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
        }
        void *pa;
        if ((rc = dev_alloc(ctx, &pa, bytes))) {
            dev_free(ctx, d_perm, sizeof(int) * n);
            return rc;
        }
        f->A = (double *)pa;
        f->A_bytes = bytes;
    }
    CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s));
    CK(launch_covgen_sym(f->cp, f->lx, f->ly, n, f->A, f->ld, s));
    // keep d_perm alive until the stream has used it
    CK(cudaStreamSynchronize(s));
    dev_free(ctx, d_perm, sizeof(int) * n);
    return GEO_OK;
}

static void release_factor_buffers(geo_ctx *ctx, geo_factor *f, bool keep_matrix_as_ws) {
    if (f->A) {
        if (keep_matrix_as_ws && !ctx->ws) {
            ctx->ws = f->A;
            ctx->ws_bytes = f->A_bytes;
        } else {
            dev_free(ctx, f->A, f->A_bytes);
        }
        f->A = nullptr;
    }
    if (f->lx) dev_free(ctx, f->lx, sizeof(double) * (2 * (size_t)f->n + GEO_TAB_DOUBLES));
    if (f->w) dev_free(ctx, f->w, sizeof(double) * f->N);
    f->lx = f->ly = f->w = nullptr;
    if (f->ybuf) dev_free(ctx, f->ybuf, sizeof(double) * f->N);
    f->ybuf = nullptr;
    if (f->tlr) {
        if (f->tlr->D) dev_free(ctx, f->tlr->D, f->tlr_bytes);
        for (auto &sg : f->tlr->segs) dev_free(ctx, sg.first, sizeof(double) * sg.second);
        delete f->tlr;
        f->tlr = nullptr;
    }
}

// Tile-low-rank evaluation of Eq. 1 (Sec. 5.3).
static int loglik_tlr(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                      const geo_opts &o, double *loglik_host, geo_factor **keep, int *info, cudaStream_t s) {
    geo_factor *f = new geo_factor();
    f->ctx = ctx;
    int rc = prepare_matrix(ctx, locs_dev, n, theta, &o, 0, f, s, false);
    auto bail = [&](int code) {
        release_factor_buffers(ctx, f, false);
        delete f;
        return code;
    };
    if (rc) return bail(rc);
    const int N = f->N, p = f->p, nb = o.nb;
    if (nb % p != 0) return bail(fail(ctx, GEO_EINVAL, "TLR needs nb to be a multiple of p"));
    if (!(o.tlr_tol > 0.0) || o.tlr_kmax < 1) return bail(fail(ctx, GEO_EINVAL, "TLR needs tol > 0 and kmax >= 1"));
    if (o.dst < 0) return bail(fail(ctx, GEO_EINVAL, "dst must be >= 0"));
    TlrFactor *F = new TlrFactor();
    f->tlr = F;
    F->N = N;
    F->nb = nb;
    F->T = (N + nb - 1) / nb;
    F->kmax = std::min(o.tlr_kmax, nb);
    F->tol = o.tlr_tol;
    F->dst = o.dst;
    const size_t fbytes = tlr_factor_bytes(N, nb, F->kmax);
    void *pf;
    if ((rc = dev_alloc(ctx, &pf, fbytes))) return bail(rc);
    f->tlr_bytes = fbytes;
    F->D = (double *)pf;
    // U / V segments: a quarter of the dense lower tiles at a time, at least the request
    const size_t seg_default = std::max((size_t)1 << 24, (size_t)F->T * (F->T - 1) / 8 * nb * nb / 2);
    F->grow = [ctx, F, seg_default](size_t need) -> double * {
        void *p = nullptr;
        const size_t n = std::max(need, seg_default);
        if (dev_alloc(ctx, &p, sizeof(double) * n) != GEO_OK) {
            // retry with exactly the request
            if (n == need || dev_alloc(ctx, &p, sizeof(double) * need) != GEO_OK) return nullptr;
            F->segs.push_back({(double *)p, need});
            return (double *)p;
        }
        F->segs.push_back({(double *)p, n});
        return (double *)p;
    };
    const size_t wbytes = std::max(tlr_workspace_bytes(N, nb, F->kmax), tlr_solve_workspace_bytes(N, nb, F->kmax));
    if ((rc = ensure_buffer(ctx, &ctx->tws, &ctx->tws_bytes, wbytes, s))) return bail(rc);
    const size_t abytes = TLR_ARENA_BYTES + sizeof(double) * (size_t)F->T * (F->kmax + 16) + 4096;
    if (ctx->tarena_bytes < abytes) {
        if (ctx->tarena) {
            cudaStreamSynchronize(s);
            cudaFreeHost(ctx->tarena);
            ctx->tarena = nullptr;
            ctx->tarena_bytes = 0;
        }
        if (cudaMallocHost(&ctx->tarena, abytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(ctx, GEO_ENOMEM, "pinned staging buffer"));
        }
        ctx->tarena_bytes = abytes;
    }
    void *py, *pp;
    if ((rc = dev_alloc(ctx, &py, sizeof(double) * N))) return bail(rc);
    f->ybuf = (double *)py;
    if ((rc = dev_alloc(ctx, &pp, sizeof(int) * n))) return bail(rc);
    int *d_perm = (int *)pp;
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_perm, f->perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
        (e = launch_gather_vec(z_dev, d_perm, n, p, f->ybuf, 1, s)) ||
        (e = tlr_factor(*F, f->cp, f->lx, f->ly, ctx->tws, ctx->tws_bytes, ctx->tarena, ctx->st, ctx->h_st, s))) {
        cudaStreamSynchronize(s);
        dev_free(ctx, d_perm, sizeof(int) * n);
        if (e == cudaErrorMemoryAllocation)
            return bail(fail(ctx, GEO_ENOMEM, "TLR: the tiles' ranks exceed the factor's pool (raise tlr_kmax or tlr_tol)"));
        return bail(cuda_fail(ctx, e, "TLR factorisation"));
    }
    CK(cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    dev_free(ctx, d_perm, sizeof(int) * n);
    if (ctx->h_st->info) {
        if (info) *info = ctx->h_st->info;
        if (loglik_host) *loglik_host = nan("");
        return bail(fail(ctx, GEO_ENOTSPD, "Sigma(theta) is not positive definite (TLR diagonal tile)"));
    }
    if ((e = tlr_solve(*F, f->ybuf, false, ctx->tws, ctx->tarena, s)) ||
        (e = tlr_reduce(*F, f->ybuf, ctx->st, ctx->res, s)) ||
        (e = cudaMemcpyAsync(ctx->h_res, ctx->res, sizeof(DevResults), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return bail(cuda_fail(ctx, e, "TLR solve"));
    f->loglik = ctx->h_res->loglik;
    f->logdet = ctx->h_res->logdet;
    f->quad = ctx->h_res->quad;
    if (loglik_host) *loglik_host = f->loglik;
    if (keep) {
        ctx->factors.push_back(f);
        *keep = f;
    } else {
        release_factor_buffers(ctx, f, false);
        delete f;
    }
    return GEO_OK;
}

int geo_loglik(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
               const geo_opts *opts, double *loglik_host, geo_factor **keep, int *info, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (keep) *keep = nullptr;
    if (info) *info = 0;
    geo_opts o;
    if (opts)
        o = *opts;
    else
        geo_opts_default(&o);
    if (n <= 0 || !locs_dev || !z_dev) return fail(ctx, GEO_EINVAL, "n must be > 0 and pointers non-NULL");
    if (o.nb == 0 && theta) resolve_tuned(ctx->device, theta->p * n, &o);
    if (o.nb < 64) return fail(ctx, GEO_EINVAL, "nb must be >= 64");
    if (int rc0 = check_dense_opts(ctx, o)) return rc0;
    if (o.prec != GEO_PREC_FP64 && o.prec != GEO_PREC_MIXED && o.prec != GEO_PREC_TLR)
        return fail(ctx, GEO_EUNSUPPORTED, "precision mode not built");
    if (o.prec == GEO_PREC_MIXED && (o.nb % 128 != 0 || o.band < 0))
        return fail(ctx, GEO_EINVAL, "mixed precision needs nb a multiple of 128 and band >= 0");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (o.prec == GEO_PREC_TLR) return loglik_tlr(ctx, locs_dev, n, z_dev, theta, o, loglik_host, keep, info, s);
    geo_factor *f = new geo_factor();
    f->ctx = ctx;
    int rc = prepare_matrix(ctx, locs_dev, n, theta, &o, 1, f, s);
    if (rc) {
        release_factor_buffers(ctx, f, false);
        delete f;
        return rc;
    }
    const int N = f->N;
    // z' into row N (internal order)
    void *pp;
    if ((rc = dev_alloc(ctx, &pp, sizeof(int) * n))) {
        release_factor_buffers(ctx, f, true);
        delete f;
        return rc;
    }
    int *d_perm = (int *)pp;
    cudaError_t e;
    const bool mixed = (o.prec == GEO_PREC_MIXED);
    const bool refine = mixed && o.refine_iters > 0;
    if (mixed) {
        const size_t abytes = sizeof(double) * (size_t)f->ld * (size_t)N;
        if ((rc = ensure_buffer(ctx, &ctx->mws, &ctx->mws_bytes, mixed_workspace_bytes(N, o.nb), s)) ||
            (refine && (rc = ensure_buffer(ctx, &ctx->sws, &ctx->sws_bytes, abytes, s))) ||
            (refine && (rc = ensure_buffer(ctx, &ctx->zws, &ctx->zws_bytes, sizeof(double) * N, s))) ||
            (refine && (rc = ensure_buffer(ctx, &ctx->rws, &ctx->rws_bytes, refine_workspace_bytes(N), s)))) {
            dev_free(ctx, d_perm, sizeof(int) * n);
            release_factor_buffers(ctx, f, true);
            delete f;
            return rc;
        }
        if (refine) {
            void *pw;
            if ((rc = dev_alloc(ctx, &pw, sizeof(double) * N))) {
                dev_free(ctx, d_perm, sizeof(int) * n);
                release_factor_buffers(ctx, f, true);
                delete f;
                return rc;
            }
            f->w = (double *)pw;
        }
    }
    if (!mixed && o.fp64_gemm == 1 &&
        (rc = ensure_buffer(ctx, &ctx->ows, &ctx->ows_bytes, oz_chol_workspace_bytes(N + 1, o.nb, oz_slices_of(o)),
                            s))) {
        dev_free(ctx, d_perm, sizeof(int) * n);
        release_factor_buffers(ctx, f, true);
        delete f;
        return rc;
    }
    double *Scopy = (double *)ctx->sws, *zsorted = (double *)ctx->zws;
    cudaError_t e_fac = cudaSuccess;
    if ((e = cudaMemcpyAsync(d_perm, f->perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
        (e = launch_gather_vec(z_dev, d_perm, n, f->p, f->A + N, f->ld, s)) ||
        (refine && (e = launch_gather_vec(z_dev, d_perm, n, f->p, zsorted, 1, s))) ||
        (refine && (e = cudaMemcpyAsync(Scopy, f->A, sizeof(double) * (size_t)f->ld * (size_t)N,
                                        cudaMemcpyDeviceToDevice, s))) ||
        (e = mixed ? chol_mixed_factor(f->A, f->ld, N, N + 1, o.nb, o.band, o.lowp, ctx->mws, ctx->mws_bytes,
                                       ctx->st, s)
                   : (dense_factor(ctx, f->A, f->ld, N, N + 1, o, s, &e_fac), e_fac)) ||
        (e = refine ? refine_solve(Scopy, f->A, f->ld, N, zsorted, f->A + N, f->ld, o.refine_iters, f->w, ctx->rws,
                                   ctx->st, ctx->res, s)
                    : launch_loglik_reduce(f->A, f->ld, N, f->A + N, f->ld, ctx->st, ctx->res, s)) ||
        (e = cudaMemcpyAsync(ctx->h_res, ctx->res, sizeof(DevResults), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        dev_free(ctx, d_perm, sizeof(int) * n);
        release_factor_buffers(ctx, f, false);
        delete f;
        return cuda_fail(ctx, e, "geo_loglik");
    }
    dev_free(ctx, d_perm, sizeof(int) * n);
    if (ctx->h_st->info) {
        if (info) *info = ctx->h_st->info;
        if (loglik_host) *loglik_host = nan("");
        release_factor_buffers(ctx, f, true);
        delete f;
        return fail(ctx, GEO_ENOTSPD, "Sigma(theta) is not positive definite (row " +
                                          std::to_string(ctx->h_st->info) + ")");
    }
    f->loglik = ctx->h_res->loglik;
    f->logdet = ctx->h_res->logdet;
    f->quad = ctx->h_res->quad;
    if (loglik_host) *loglik_host = f->loglik;
    if (keep) {
        ctx->factors.push_back(f);
        *keep = f;
    } else {
        release_factor_buffers(ctx, f, true);
        delete f;
    }
    return GEO_OK;
}

// Sec. 4.2: sigma^2_ii = n^-1 Z_i' R_ii^-1 Z_i.  Z_i is copied out of the
// Representation I vector with one strided copy and each R_ii is a p = 1
// likelihood (sigma^2 = 1, nu_ii, a) in the requested form; Z_i' R_ii^-1 Z_i is
// that likelihood's data term.
int geo_sigma2_hat(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                   const geo_opts *opts, double *sigma2_host, int *info, void *stream) {
    if (!ctx) return GEO_EINVAL;
    if (info) *info = 0;
    if (!theta || theta->p < 1 || theta->p > GEO_PMAX || !theta->nu || !sigma2_host || n <= 0 || !locs_dev ||
        !z_dev)
        return fail(ctx, GEO_EINVAL, "geo_sigma2_hat: bad arguments");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int p = theta->p;
    void *pz;
    int rc;
    if ((rc = dev_alloc(ctx, &pz, sizeof(double) * n))) return rc;
    double *zi = (double *)pz;
    const double one = 1.0;
    // tile-low-rank / DST: marginal tiles of nb / p rows cover the same location blocks as Sigma's tiles
    geo_opts om;
    const geo_opts *mo = opts;
    if (opts && opts->prec == GEO_PREC_TLR && opts->nb > 0) {
        om = *opts;
        om.nb = opts->nb / p;
        mo = &om;
    }
    for (int i = 0; i < p && rc == GEO_OK; ++i) {
        cudaError_t e = cudaMemcpy2DAsync(zi, sizeof(double), z_dev + i, sizeof(double) * p, sizeof(double), n,
                                          cudaMemcpyDeviceToDevice, s);
        if (e) {
            rc = cuda_fail(ctx, e, "geo_sigma2_hat");
            break;
        }
        geo_theta ti{1, &one, theta->nu + i, nullptr, theta->a};
        double ll;
        rc = geo_loglik(ctx, locs_dev, n, zi, &ti, mo, &ll, nullptr, info, stream);
        if (rc == GEO_OK) sigma2_host[i] = ctx->h_res->quad / n;
    }
    cudaStreamSynchronize(s);
    dev_free(ctx, zi, sizeof(double) * n);
    return rc;
}

int geo_loglik_profile(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                       const geo_opts *opts, double *loglik_host, double *sigma2_host, int *info, void *stream) {
    if (!ctx) return GEO_EINVAL;
    if (!theta || theta->p < 1 || theta->p > GEO_PMAX) return fail(ctx, GEO_EINVAL, "geo_loglik_profile: bad theta");
    double s2[GEO_PMAX];
    int rc = geo_sigma2_hat(ctx, locs_dev, n, z_dev, theta, opts, s2, info, stream);
    if (rc) return rc;
    if (sigma2_host)
        for (int i = 0; i < theta->p; ++i) sigma2_host[i] = s2[i];
    geo_theta t = *theta;
    t.sigma2 = s2;
    return geo_loglik(ctx, locs_dev, n, z_dev, &t, opts, loglik_host, nullptr, info, stream);
}

// The device workspace and pinned descriptor arena of tlr_solve (the
// workspace is released when a serving context is trimmed).
static int tlr_solve_buffers(geo_ctx *ctx, const TlrFactor &F, cudaStream_t s) {
    if (!ctx->tarena || ctx->tarena_bytes < TLR_ARENA_BYTES)
        return fail(ctx, GEO_EINVAL, "the tile-low-rank factor belongs to another context");
    return ensure_buffer(ctx, &ctx->tws, &ctx->tws_bytes, tlr_solve_workspace_bytes(F.N, F.nb, F.kmax), s);
}

// Sec. 4.3 variances on a tile-low-rank factor: c0 (N x p m, the factor's
// order) is formed transposed by the cross-covariance kernel, transposed to
// one contiguous column per right-hand side, solved column by column with the
// TLR forward solve, and var = C_ii(0) - |L^-1 c0|^2 per column.
static int predict_var_tlr(geo_ctx *ctx, const geo_factor *f, const double *new_locs_dev, int m, double *var_dev,
                           cudaStream_t s) {
    const int p = f->p, N = f->N, pm = p * m;
    const long long ldx = round_up(pm, 32);
    const size_t xbytes = sizeof(double) * (size_t)ldx * N, ybytes = sizeof(double) * (size_t)N * pm,
                 sbytes = sizeof(double) * pm;
    void *px = nullptr, *py = nullptr, *ps = nullptr;
    auto done = [&](int code) {
        cudaStreamSynchronize(s);
        if (px) dev_free(ctx, px, xbytes);
        if (py) dev_free(ctx, py, ybytes);
        if (ps) dev_free(ctx, ps, sbytes);
        return code;
    };
    int rc;
    cudaStreamSynchronize(s);   // no earlier descriptor copy may still read the pinned arena
    if ((rc = tlr_solve_buffers(ctx, *f->tlr, s)) || (rc = dev_alloc(ctx, &px, xbytes)) ||
        (rc = dev_alloc(ctx, &py, ybytes)) || (rc = dev_alloc(ctx, &ps, sbytes)))
        return done(rc);
    double c0d[GEO_PMAX];
    for (int i = 0; i < p; ++i) c0d[i] = f->cp.m[i * p + i].c0;
    double *X = (double *)px, *Y = (double *)py;
    cudaError_t e;
    if ((e = launch_covgen_cross(f->cp, new_locs_dev, m, f->lx, f->ly, f->n, X, ldx, s)) ||
        (e = launch_transpose(X, ldx, pm, N, Y, N, s)))
        return done(cuda_fail(ctx, e, "geo_predict_var"));
    for (int q = 0; q < pm; ++q) {
        // each solve stages its descriptors in the same pinned arena: wait before the next one refills it
        if ((e = tlr_solve(*f->tlr, Y + (size_t)q * N, false, ctx->tws, ctx->tarena, s)) ||
            (e = cudaStreamSynchronize(s)))
            return done(cuda_fail(ctx, e, "geo_predict_var (TLR solve)"));
    }
    if ((e = launch_col_sumsq(Y, N, N, pm, (double *)ps, s)) ||
        (e = launch_var_finish((const double *)ps, pm, p, c0d, var_dev, s)))
        return done(cuda_fail(ctx, e, "geo_predict_var"));
    return done(GEO_OK);
}

// w = Sigma^-1 Z of a kept factor (computed once, on first use).
static int ensure_weights(geo_ctx *ctx, geo_factor *f, cudaStream_t s) {
    if (f->w) return GEO_OK;
    int rc;
    if (f->tlr && (rc = tlr_solve_buffers(ctx, *f->tlr, s))) return rc;
    void *pw;
    if ((rc = dev_alloc(ctx, &pw, sizeof(double) * f->N))) return rc;
    f->w = (double *)pw;
    if (f->tlr) {
        CK(cudaMemcpyAsync(f->w, f->ybuf, sizeof(double) * f->N, cudaMemcpyDeviceToDevice, s));
        CK(tlr_solve(*f->tlr, f->w, true, ctx->tws, ctx->tarena, s));
        CK(cudaStreamSynchronize(s));   // the solve's descriptors sit in the shared pinned arena
    } else {
        CK(backward_solve(f->A, f->ld, f->N, f->A + f->N, f->ld, f->w, ctx->sync, &ctx->st->timeout, s));
    }
    return GEO_OK;
}

int geo_predict(geo_ctx *ctx, const geo_factor *factor, const double *new_locs_dev, int m, double *zhat_dev,
                void *stream) {
    if (!ctx || !factor) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (m < 0) return fail(ctx, GEO_EINVAL, "m < 0");
    if (m == 0) return GEO_OK;
    if (!new_locs_dev || !zhat_dev) return fail(ctx, GEO_EINVAL, "NULL pointer");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    geo_factor *f = const_cast<geo_factor *>(factor);
    if (int rc = ensure_weights(ctx, f, s)) return rc;
    CK(launch_predict(f->cp, new_locs_dev, m, f->lx, f->ly, f->n, f->w, zhat_dev, s));
    return GEO_OK;
}

int geo_predict_batch(geo_ctx *ctx, int count, const geo_factor *const *factors, const double *const *new_locs_dev,
                      const int *m, double *const *zhat_dev, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (count <= 0 || !factors || !new_locs_dev || !m || !zhat_dev)
        return fail(ctx, GEO_EINVAL, "count must be > 0 and arrays non-NULL");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<PredDesc> h(count);
    long long total = 0;
    double flops = 0.0;
    for (int k = 0; k < count; ++k) {
        geo_factor *f = const_cast<geo_factor *>(factors[k]);
        if (!f || m[k] < 0 || (m[k] > 0 && (!new_locs_dev[k] || !zhat_dev[k])))
            return fail(ctx, GEO_EINVAL, "batch entry " + std::to_string(k) + ": bad factor, size or pointer");
        if (int rc = ensure_weights(ctx, f, s)) return rc;
        h[k] = PredDesc{f->cp, f->lx, f->ly, f->w, new_locs_dev[k], zhat_dev[k], f->n, m[k], (int)total};
        total += m[k];
        flops += 2.0 * f->p * (double)m[k] * f->p * (double)f->n;
    }
    if (total == 0) return GEO_OK;
    if (total > (1LL << 31) - 1) return fail(ctx, GEO_EINVAL, "too many new locations");
    const size_t bytes = sizeof(PredDesc) * (size_t)count;
    if (ctx->pdesc_cap < bytes) {
        CK(cudaStreamSynchronize(s));
        if (ctx->pdesc_d) cudaFree(ctx->pdesc_d);
        if (ctx->pdesc_h) cudaFreeHost(ctx->pdesc_h);
        ctx->pdesc_d = ctx->pdesc_h = nullptr;
        ctx->pdesc_cap = 0;
        if (cudaMalloc(&ctx->pdesc_d, bytes) != cudaSuccess || cudaMallocHost(&ctx->pdesc_h, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, GEO_ENOMEM, "prediction descriptors");
        }
        ctx->pdesc_cap = bytes;
    }
    CK(cudaStreamSynchronize(s));   // the pinned staging buffer is reused by every call
    memcpy(ctx->pdesc_h, h.data(), bytes);
    CK(cudaMemcpyAsync(ctx->pdesc_d, ctx->pdesc_h, bytes, cudaMemcpyHostToDevice, s));
    CK(launch_predict_batch((const PredDesc *)ctx->pdesc_d, count, (int)total, flops, s));
    return GEO_OK;
}

int geo_simulate(geo_ctx *ctx, const double *locs_dev, int n, const double *e_dev, const geo_theta *theta,
                 const geo_opts *opts, double *z_dev, int *info, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (info) *info = 0;
    geo_opts o;
    if (opts)
        o = *opts;
    else
        geo_opts_default(&o);
    if (n <= 0 || !locs_dev || !e_dev || !z_dev) return fail(ctx, GEO_EINVAL, "bad arguments");
    if (o.nb == 0 && theta) o.nb = resolve_nb(ctx->device, form_of(o), theta->p * n);
    if (o.nb < 64) return fail(ctx, GEO_EINVAL, "nb must be >= 64");
    if (int rc0 = check_dense_opts(ctx, o)) return rc0;
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    geo_factor f;
    f.ctx = ctx;
    int rc = prepare_matrix(ctx, locs_dev, n, theta, &o, 0, &f, s);
    if (rc) {
        release_factor_buffers(ctx, &f, false);
        return rc;
    }
    const int N = f.N;
    void *pz, *pp;
    if ((rc = dev_alloc(ctx, &pz, sizeof(double) * N))) {
        release_factor_buffers(ctx, &f, true);
        return rc;
    }
    if ((rc = dev_alloc(ctx, &pp, sizeof(int) * n))) {
        dev_free(ctx, pz, sizeof(double) * N);
        release_factor_buffers(ctx, &f, true);
        return rc;
    }
    double *zs = (double *)pz;
    int *d_perm = (int *)pp;
    cudaError_t e;
    const bool mixed = (o.prec == GEO_PREC_MIXED);
    if (mixed && (o.nb % 128 != 0 ||
                  (rc = ensure_buffer(ctx, &ctx->mws, &ctx->mws_bytes, mixed_workspace_bytes(N, o.nb), s)))) {
        dev_free(ctx, zs, sizeof(double) * N);
        dev_free(ctx, d_perm, sizeof(int) * n);
        release_factor_buffers(ctx, &f, true);
        return rc ? rc : fail(ctx, GEO_EINVAL, "mixed precision needs nb a multiple of 128");
    }
    cudaError_t e_fac = cudaSuccess;
    if (!mixed && (rc = dense_factor(ctx, f.A, f.ld, N, N, o, s, &e_fac))) {
        dev_free(ctx, zs, sizeof(double) * N);
        dev_free(ctx, d_perm, sizeof(int) * n);
        release_factor_buffers(ctx, &f, true);
        return rc;
    }
    if ((e = mixed ? chol_mixed_factor(f.A, f.ld, N, N, o.nb, o.band, o.lowp, ctx->mws, ctx->mws_bytes, ctx->st, s)
                   : e_fac) ||
        (e = launch_trmv_lower(f.A, f.ld, N, e_dev, zs, s)) ||
        (e = cudaMemcpyAsync(d_perm, f.perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, s)) ||
        (e = launch_scatter_vec(zs, 1, d_perm, n, f.p, z_dev, s)) ||
        (e = cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        rc = cuda_fail(ctx, e, "geo_simulate");
    }
    dev_free(ctx, zs, sizeof(double) * N);
    dev_free(ctx, d_perm, sizeof(int) * n);
    release_factor_buffers(ctx, &f, true);
    if (rc) return rc;
    if (ctx->h_st->info) {
        if (info) *info = ctx->h_st->info;
        return fail(ctx, GEO_ENOTSPD, "Sigma(theta) is not positive definite");
    }
    return GEO_OK;
}

int geo_factor_stats_get(const geo_factor *f, geo_factor_stats *out) {
    if (!f || !out) return GEO_EINVAL;
    memset(out, 0, sizeof(*out));
    out->n = f->n;
    out->p = f->p;
    out->N = f->N;
    out->nb = f->nb;
    out->prec = f->prec;
    out->loglik = f->loglik;
    out->logdet = f->logdet;
    out->quad = f->quad;
    out->device_bytes = (long long)(f->A_bytes + sizeof(double) * (2 * (size_t)f->n + GEO_TAB_DOUBLES) +
                                    (f->w ? sizeof(double) * f->N : 0));
    out->tlr_bytes_ratio = 1.0;
    if (f->tlr) {
        const TlrFactor &F = *f->tlr;
        double used = (double)F.T * F.nb * F.nb;
        for (int r : F.rank) used += 2.0 * F.nb * r;
        const double dense = (double)F.T * (F.T + 1) / 2.0 * F.nb * F.nb;
        out->tlr_bytes_ratio = used / dense;
        out->tlr_max_rank = F.max_rank;
        out->tlr_dense_tiles = F.capped;
        out->device_bytes = (long long)(8.0 * used + sizeof(double) * (2.0 * f->n + GEO_TAB_DOUBLES + f->N));
    }
    return GEO_OK;
}

int geo_factor_read(const geo_factor *f, int what, long long r0, long long r1, long long c0, long long c1,
                    double *host_out) {
    if (!f || !host_out) return GEO_EINVAL;
    geo_ctx *ctx = f->ctx;
    SetDevice sd(ctx->device);
    if (what == 0) {
        if (r0 < 0 || c0 < 0 || r1 > f->N || c1 > f->N || r1 < r0 || c1 < c0)
            return fail(ctx, GEO_EINVAL, "block out of range");
        const long long nr = r1 - r0, nc = c1 - c0;
        std::vector<double> col((size_t)std::max(nr, 1LL));
        for (long long c = c0; c < c1; ++c) {
            if (nr > 0) CK(cudaMemcpy(col.data(), f->A + c * f->ld + r0, sizeof(double) * nr, cudaMemcpyDeviceToHost));
            for (long long r = r0; r < r1; ++r) host_out[(r - r0) * nc + (c - c0)] = (r >= c) ? col[r - r0] : 0.0;
        }
        return GEO_OK;
    }
    if (what == 1) {
        if (r0 < 0 || r1 > f->N || r1 < r0) return fail(ctx, GEO_EINVAL, "range out of bounds");
        for (long long k = r0; k < r1; ++k)
            CK(cudaMemcpy(host_out + (k - r0), f->A + k * f->ld + f->N, sizeof(double), cudaMemcpyDeviceToHost));
        return GEO_OK;
    }
    if (what == 2) {
        if (r0 < 0 || r1 > f->n || r1 < r0) return fail(ctx, GEO_EINVAL, "range out of bounds");
        for (long long k = r0; k < r1; ++k) host_out[k - r0] = (double)f->perm[k];
        return GEO_OK;
    }
    if (what >= 3 && what <= 6) {
        if (!f->tlr) return fail(ctx, GEO_EINVAL, "not a TLR factor");
        const TlrFactor &F = *f->tlr;
        auto mt = [&](long long t) { return (long long)std::min(F.nb, F.N - (int)t * F.nb); };
        if (what == 3) {   // ranks of tiles (r0, c0 = j) for rows r0 .. r1-1
            for (long long i = r0; i < r1; ++i)
                host_out[i - r0] = (i > c0 && i < F.T && c0 >= 0) ? (double)F.rank[(size_t)i * (i - 1) / 2 + c0] : -1.0;
            return GEO_OK;
        }
        if (what == 6) {   // diagonal tile r0 of L (mt x mt, column-major)
            if (r0 < 0 || r0 >= F.T) return fail(ctx, GEO_EINVAL, "tile out of range");
            const long long m = mt(r0);
            std::vector<double> buf((size_t)F.nb * m);
            CK(cudaMemcpy(buf.data(), F.D + (size_t)r0 * F.nb * F.nb, sizeof(double) * F.nb * m, cudaMemcpyDeviceToHost));
            for (long long c = 0; c < m; ++c)
                for (long long r = 0; r < m; ++r) host_out[c * m + r] = (r >= c) ? buf[(size_t)c * F.nb + r] : 0.0;
            return GEO_OK;
        }
        // U (what 4, mt(r0) x rank) or V (what 5, mt(c0) x rank) of tile (r0, c0), column-major
        if (!(r0 > c0 && c0 >= 0 && r0 < F.T)) return fail(ctx, GEO_EINVAL, "tile out of range");
        const size_t sl = (size_t)r0 * (r0 - 1) / 2 + c0;
        const long long k = F.rank[sl], m = (what == 4) ? mt(r0) : mt(c0);
        const double *src = (what == 4) ? F.Uof(sl) : F.Vof(sl);
        std::vector<double> buf((size_t)F.nb * std::max(k, 1LL));
        if (k) CK(cudaMemcpy(buf.data(), src, sizeof(double) * F.nb * k, cudaMemcpyDeviceToHost));
        for (long long c = 0; c < k; ++c)
            for (long long r = 0; r < m; ++r) host_out[c * m + r] = buf[(size_t)c * F.nb + r];
        return GEO_OK;
    }
    return fail(ctx, GEO_EINVAL, "unknown 'what'");
}

void geo_factor_free(geo_factor *f) {
    if (!f) return;
    geo_ctx *ctx = f->ctx;
    SetDevice sd(ctx->device);
    cudaDeviceSynchronize();
    release_factor_buffers(ctx, f, true);   // the matrix buffer becomes the context's workspace
    auto it = std::find(ctx->factors.begin(), ctx->factors.end(), f);
    if (it != ctx->factors.end()) ctx->factors.erase(it);
    delete f;
}

int geo_loglik_batch(geo_ctx *ctx, int count, const geo_batch_item *items, double *loglik_host, int *info_host,
                     void *stream) {
    if (!ctx) return GEO_EINVAL;
    if (count <= 0 || !items || !loglik_host) return fail(ctx, GEO_EINVAL, "count must be > 0 and arrays non-NULL");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<CovParams> cps(count);
    std::vector<size_t> offs(count);
    size_t total = 0;
    int nmax = 0, Nmax = 0;
    for (int k = 0; k < count; ++k) {
        const geo_batch_item &it = items[k];
        std::string err;
        if (it.n <= 0 || !it.locs_dev || !it.z_dev)
            return fail(ctx, GEO_EINVAL, "batch item " + std::to_string(k) + ": bad size or pointer");
        int rc = theta_to_params(&it.theta, &cps[k], &err);
        if (rc) return fail(ctx, rc, "batch item " + std::to_string(k) + ": " + err);
        const int N = it.theta.p * it.n;
        const long long ld = round_up((long long)N + 1, 32);
        offs[k] = total;
        total += (size_t)ld * N + GEO_TAB_DOUBLES;   // matrix, then the theta's K_nu tables
        nmax = std::max(nmax, it.n);
        Nmax = std::max(Nmax, N);
    }
    int rc;
    if ((rc = ensure_buffer(ctx, &ctx->bws, &ctx->bws_bytes, sizeof(double) * total, s))) return rc;
    // device buffer: descriptors, counters (4 + count ints), the unit count, the ticket table
    std::vector<int> orders(2 * count);   // orders, then location counts
    for (int k = 0; k < count; ++k) orders[k] = items[k].theta.p * items[k].n, orders[count + k] = items[k].n;
    const int nunits = -batch_units(orders.data(), orders.data() + count, count, 0, nullptr, 0);   // size query
    const size_t desc_bytes = batch_desc_bytes() * (size_t)count;
    const size_t cnt_off = (desc_bytes + 255) / 256 * 256;
    const size_t nun_off = cnt_off + (sizeof(int) * (4 + (size_t)count) + 255) / 256 * 256;
    const size_t unit_off = nun_off + 256;
    const size_t dbytes = unit_off + 16 * (size_t)nunits;
    if (ctx->bdesc_cap < dbytes) {
        CK(cudaStreamSynchronize(s));
        if (ctx->bdesc_d) cudaFree(ctx->bdesc_d);
        if (ctx->bdesc_h) cudaFreeHost(ctx->bdesc_h);
        ctx->bdesc_d = ctx->bdesc_h = nullptr;
        ctx->bdesc_cap = 0;
        if (cudaMalloc(&ctx->bdesc_d, dbytes) != cudaSuccess || cudaMallocHost(&ctx->bdesc_h, dbytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, GEO_ENOMEM, "batch descriptors");
        }
        ctx->bdesc_cap = dbytes;
        // graphs hold the old descriptor pointer
        for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second.first);
        ctx->graphs.clear();
    }
    double *base = (double *)ctx->bws;
    for (int k = 0; k < count; ++k) {
        const geo_batch_item &it = items[k];
        const int N = it.theta.p * it.n;
        const long long ld = round_up((long long)N + 1, 32);
        cps[k].tab = base + offs[k] + (size_t)ld * N;
        batch_fill_desc(ctx->bdesc_h, k, base + offs[k], ld, N, it.n, it.locs_dev, it.z_dev, cps[k]);
    }
    char *hb = (char *)ctx->bdesc_h, *db = (char *)ctx->bdesc_d;
    *(int *)(hb + nun_off) = nunits;
    // the ticket table depends only on the problem orders: rebuilt when they change
    if (ctx->border != orders) {
        ctx->bunits.resize(16 * (size_t)nunits);
        batch_units(orders.data(), orders.data() + count, count, batch_workers(), ctx->bunits.data(), (size_t)nunits);
        ctx->border = orders;
    }
    memcpy(hb + unit_off, ctx->bunits.data(), 16 * (size_t)nunits);
    CK(cudaMemcpyAsync(db, hb, desc_bytes, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(db + nun_off, hb + nun_off, dbytes - nun_off, cudaMemcpyHostToDevice, s));
    int *counters_d = (int *)(db + cnt_off);
    const int *nunits_d = (const int *)(db + nun_off);
    const void *units_d = db + unit_off;
    const auto key = std::make_tuple(count, nmax, Nmax);
    auto itg = ctx->graphs.find(key);
    if (itg == ctx->graphs.end()) {
        // capture the launch sequence of this batch shape; launches are counted, not event-timed
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        Profiler counter;
        ProfBind pb(&counter);
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_record(ctx->bdesc_d, units_d, nunits_d, counters_d, count, nmax, Nmax, ctx->cap_stream);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch capture");
        if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "batch capture end");
        cudaGraphExec_t exec;
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
        long long nodes = 0;
        for (int k = 0; k < GEO_K_COUNT; ++k) nodes += counter.launches[k];
        itg = ctx->graphs.emplace(key, std::make_pair(exec, nodes)).first;
    }
    CK(cudaGraphLaunch(itg->second.first, s));
    ctx->prof.launches[GEO_K_GEMM] += itg->second.second;   // kernel nodes of the replayed graph
    std::vector<int> info(count);
    CK(batch_results(ctx->bdesc_d, ctx->bdesc_h, count, loglik_host, info.data(), s));
    if (info_host)
        for (int k = 0; k < count; ++k) info_host[k] = info[k];
    int tmo = 0;   // a bounded wait of the persistent launch that expired
    CK(cudaMemcpy(&tmo, counters_d + 2, sizeof(int), cudaMemcpyDeviceToHost));
    if (tmo) return fail(ctx, GEO_ETIMEOUT, "a bounded wait of the batched factorisation expired");
    return GEO_OK;
}

int geo_predict_var(geo_ctx *ctx, const geo_factor *factor, const double *new_locs_dev, int m, double *var_dev,
                    void *stream) {
    if (!ctx || !factor) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (m < 0) return fail(ctx, GEO_EINVAL, "m < 0");
    if (m == 0) return GEO_OK;
    if (!new_locs_dev || !var_dev) return fail(ctx, GEO_EINVAL, "NULL pointer");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (factor->tlr) return predict_var_tlr(ctx, factor, new_locs_dev, m, var_dev, s);
    const geo_factor *f = factor;
    const int p = f->p, N = f->N, pm = p * m;
    const long long ldx = round_up(pm, 32);
    const size_t xbytes = sizeof(double) * (size_t)ldx * N, sbytes = sizeof(double) * pm,
                 dbytes = sizeof(GemmDesc) * 64;
    void *px = nullptr, *ps = nullptr, *pd = nullptr;
    auto done = [&](int code) {
        cudaStreamSynchronize(s);
        if (px) dev_free(ctx, px, xbytes);
        if (ps) dev_free(ctx, ps, sbytes);
        if (pd) dev_free(ctx, pd, dbytes);
        return code;
    };
    int rc;
    if ((rc = dev_alloc(ctx, &px, xbytes)) || (rc = dev_alloc(ctx, &ps, sbytes)) || (rc = dev_alloc(ctx, &pd, dbytes)))
        return done(rc);
    double c0d[GEO_PMAX];
    for (int i = 0; i < p; ++i) c0d[i] = f->cp.m[i * p + i].c0;
    cudaError_t e;
    // X = c0' (p m x N, the factor's location order), X <- X L^-T = (L^-1 c0)', var = C_ii(0) - |row|^2
    if ((e = launch_covgen_cross(f->cp, new_locs_dev, m, f->lx, f->ly, f->n, (double *)px, ldx, s)) ||
        (e = trsm_right_upper_t((double *)px, ldx, pm, f->A, f->ld, N, pd, s)) ||
        (e = launch_row_sums((double *)px, ldx, nullptr, 0, pm, N, (double *)ps, nullptr, s)) ||
        (e = launch_var_finish((const double *)ps, pm, p, c0d, var_dev, s)))
        return done(cuda_fail(ctx, e, "geo_predict_var"));
    return done(GEO_OK);
}

int geo_mloe_mmom(geo_ctx *ctx, const double *locs_dev, int n, const double *pred_dev, int m,
                  const geo_theta *theta_t, const geo_theta *theta_a, const geo_opts *opts, double *mloe,
                  double *mmom, double *loe_host, double *mom_host, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (!theta_t || !theta_a || theta_t->p != theta_a->p)
        return fail(ctx, GEO_EINVAL, "theta_t and theta_a must be given with the same p");
    if (n <= 0 || m <= 0 || !locs_dev || !pred_dev || !mloe || !mmom)
        return fail(ctx, GEO_EINVAL, "n, m must be > 0 and pointers non-NULL");
    geo_opts o;
    if (opts)
        o = *opts;
    else
        geo_opts_default(&o);
    o.prec = GEO_PREC_FP64;
    const int p = theta_t->p, N = p * n, pm = p * m;
    if (o.nb == 0) o.nb = resolve_nb(ctx->device, form_of(o), N);
    if (o.nb < 64) return fail(ctx, GEO_EINVAL, "nb must be >= 64");
    if (int rc0 = check_dense_opts(ctx, o)) return rc0;
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    geo_factor *ft = new geo_factor(), *fa = new geo_factor();
    ft->ctx = fa->ctx = ctx;
    const int nblk = (N + 63) / 64;
    const long long ldv = round_up(pm, 32);
    void *pv = nullptr, *psum = nullptr, *pdesc = nullptr, *hdesc = nullptr;
    const size_t vbytes = sizeof(double) * (size_t)ldv * N, dbytes = sizeof(GemmDesc) * (size_t)(nblk + 64);
    auto done = [&](int code) {
        cudaStreamSynchronize(s);
        release_factor_buffers(ctx, ft, true);
        release_factor_buffers(ctx, fa, true);
        delete ft;
        delete fa;
        if (pv) dev_free(ctx, pv, vbytes);
        if (psum) dev_free(ctx, psum, sizeof(double) * 4 * pm);
        if (pdesc) dev_free(ctx, pdesc, dbytes);
        if (hdesc) cudaFreeHost(hdesc);
        return code;
    };
    int rc;
    // Sigma_t with C_t' in rows [N, N + pm); Sigma_a with C_a' and C_t' below it
    if ((rc = prepare_matrix(ctx, locs_dev, n, theta_t, &o, pm, ft, s)) ||
        (rc = prepare_matrix(ctx, locs_dev, n, theta_a, &o, 2 * pm, fa, s)))
        return done(rc);
    if ((rc = dev_alloc(ctx, &pv, vbytes)) || (rc = dev_alloc(ctx, &psum, sizeof(double) * 4 * pm)) ||
        (rc = dev_alloc(ctx, &pdesc, dbytes)))
        return done(rc);
    if (cudaMallocHost(&hdesc, sizeof(GemmDesc) * (size_t)nblk) != cudaSuccess) {
        cudaGetLastError();
        hdesc = nullptr;
        return done(fail(ctx, GEO_ENOMEM, "pinned descriptor buffer"));
    }
    double *sum_t = (double *)psum, *sum_a = sum_t + pm, *cross = sum_a + pm, *sum_v = cross + pm;
    cudaError_t e, e_ft = cudaSuccess, e_fa = cudaSuccess;
    if (o.fp64_gemm == 1 &&
        (rc = ensure_buffer(ctx, &ctx->ows, &ctx->ows_bytes,
                            oz_chol_workspace_bytes(N + 2 * pm, o.nb, oz_slices_of(o)), s)))
        return done(rc);
    if ((e = launch_covgen_cross(ft->cp, pred_dev, m, ft->lx, ft->ly, n, ft->A + N, ft->ld, s)) ||
        (e = launch_covgen_cross(fa->cp, pred_dev, m, fa->lx, fa->ly, n, fa->A + N, fa->ld, s)) ||
        (e = launch_covgen_cross(ft->cp, pred_dev, m, fa->lx, fa->ly, n, fa->A + N + pm, fa->ld, s)) ||
        // factorisations: the rows below become (L^-1 c)'
        (dense_factor(ctx, ft->A, ft->ld, N, N + pm, o, s, &e_ft), e = e_ft) ||
        (dense_factor(ctx, fa->A, fa->ld, N, N + 2 * pm, o, s, &e_fa), e = e_fa) ||
        // |L_t^-1 c_t|^2, |L_a^-1 c_a|^2, (L_a^-1 c_t) . (L_a^-1 c_a)
        (e = launch_row_sums(ft->A + N, ft->ld, nullptr, 0, pm, N, sum_t, nullptr, s)) ||
        (e = launch_row_sums(fa->A + N, fa->ld, fa->A + N + pm, fa->ld, pm, N, sum_a, cross, s)) ||
        // w_a' = (L_a^-1 c_a)' L_a^-1 = (S_a^-1 c_a)', then (L_t' S_a^-1 c_a)' = w_a' L_t
        (e = trsm_right_lower(fa->A + N, fa->ld, pm, fa->A, fa->ld, N, pdesc, s)) ||
        (e = trmm_right_lower(fa->A + N, fa->ld, pm, ft->A, ft->ld, N, (double *)pv, ldv, (GemmDesc *)pdesc + 64,
                              hdesc, s)) ||
        (e = launch_row_sums((double *)pv, ldv, nullptr, 0, pm, N, sum_v, nullptr, s)) ||
        (e = cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)))
        return done(cuda_fail(ctx, e, "geo_mloe_mmom"));
    std::vector<double> h(4 * (size_t)pm);
    if ((e = cudaMemcpyAsync(h.data(), psum, sizeof(double) * 4 * pm, cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s)))
        return done(cuda_fail(ctx, e, "geo_mloe_mmom"));
    if (ctx->h_st->info) return done(fail(ctx, GEO_ENOTSPD, "Sigma(theta_t) or Sigma(theta_a) is not positive definite"));
    if (ctx->h_st->timeout) return done(fail(ctx, GEO_ETIMEOUT, "a bounded device wait expired"));
    // Eq. 5 - Eq. 8 per location; C_ii(0) = sigma^2_i (rho_ii = 1)
    double tr_t = 0.0, tr_a = 0.0;
    for (int i = 0; i < p; ++i) {
        tr_t += ft->cp.m[i * p + i].c0;
        tr_a += fa->cp.m[i * p + i].c0;
    }
    double sl = 0.0, sm = 0.0;
    for (int l = 0; l < m; ++l) {
        double et = tr_t, ea = tr_a, eta = tr_t;
        for (int i = 0; i < p; ++i) {
            const int q = p * l + i;
            et -= h[q];
            ea -= h[pm + q];
            eta += h[3 * (size_t)pm + q] - 2.0 * h[2 * (size_t)pm + q];
        }
        const double loe = eta / et - 1.0, mom = ea / eta - 1.0;
        if (loe_host) loe_host[l] = loe;
        if (mom_host) mom_host[l] = mom;
        sl += loe;
        sm += mom;
    }
    *mloe = sl / m;
    *mmom = sm / m;
    return done(GEO_OK);
}

// Median device time of `samples` evaluations after one warm-up; GEO_EINVAL /
// GEO_EUNSUPPORTED when the options are not valid for the form.
static int time_candidate(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                          const geo_opts &o, int samples, void *stream, cudaEvent_t e0, cudaEvent_t e1, double *ms_out) {
    cudaStream_t s = (cudaStream_t)stream;
    double ll;
    int rc = geo_loglik(ctx, locs_dev, n, z_dev, theta, &o, &ll, nullptr, nullptr, stream);   // warm-up
    if (rc != GEO_OK) return rc;
    std::vector<float> t;
    for (int k = 0; k < samples; ++k) {
        cudaEventRecord(e0, s);
        rc = geo_loglik(ctx, locs_dev, n, z_dev, theta, &o, &ll, nullptr, nullptr, stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        if (rc != GEO_OK) return rc;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        t.push_back(ms);
    }
    std::sort(t.begin(), t.end());
    *ms_out = t[t.size() / 2];
    return GEO_OK;
}

int geo_autotune(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                 const geo_opts *base, const int *nb_cand, int n_nb, const int *band_cand, int n_band, int samples,
                 int *best_nb, int *best_band, double *best_ms, void *stream) {
    if (!ctx || !theta || !nb_cand || n_nb <= 0 || (n_band > 0 && !band_cand) || n_band < 0) return GEO_EINVAL;
    if (samples < 1) samples = 3;
    SetDevice sd(ctx->device);
    geo_opts o;
    if (base)
        o = *base;
    else
        geo_opts_default(&o);
    const bool tune_band = o.prec == GEO_PREC_MIXED && n_band > 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int bnb = -1, bband = -1;
    double bms = 1e300;
    for (int c = 0; c < n_nb; ++c) {
        for (int b = 0; b < (tune_band ? n_band : 1); ++b) {
            o.nb = nb_cand[c];
            if (tune_band) o.band = band_cand[b];
            double ms = 0.0;
            const int rc = time_candidate(ctx, locs_dev, n, z_dev, theta, o, samples, stream, e0, e1, &ms);
            if (rc == GEO_EINVAL || rc == GEO_EUNSUPPORTED) continue;   // candidate not valid for this form
            if (rc != GEO_OK) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return rc;
            }
            if (ms < bms) {
                bms = ms;
                bnb = o.nb;
                bband = tune_band ? o.band : -1;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (bnb < 0) return fail(ctx, GEO_EINVAL, "no valid candidate");
    {
        std::lock_guard<std::mutex> lk(g_tuned_mu);
        g_tuned[std::make_tuple(ctx->device, form_of(o), order_bucket(theta->p * n))] = Tuned{bnb, bband};
    }
    if (best_nb) *best_nb = bnb;
    if (best_band) *best_band = bband;
    if (best_ms) *best_ms = bms;
    return GEO_OK;
}

int geo_autotune_nb(geo_ctx *ctx, const double *locs_dev, int n, const double *z_dev, const geo_theta *theta,
                    const geo_opts *base, const int *candidates, int ncand, int *best_nb, double *best_ms,
                    void *stream) {
    return geo_autotune(ctx, locs_dev, n, z_dev, theta, base, candidates, ncand, nullptr, 0, 3, best_nb, nullptr,
                        best_ms, stream);
}

int geo_gemm_f64e(geo_ctx *ctx, int m, int n, int k, const double *A_dev, long long lda, const double *B_dev,
                  long long ldb, double *C_dev, long long ldc, int slices, void *stream) {
    if (!ctx) return GEO_EINVAL;
    ProfBind pb(&ctx->prof);
    if (m < 0 || n < 0 || k < 0) return fail(ctx, GEO_EINVAL, "m, n, k must be >= 0");
    if (m == 0 || n == 0 || k == 0) return GEO_OK;
    if (!A_dev || !B_dev || !C_dev) return fail(ctx, GEO_EINVAL, "NULL operand");
    if (lda < m || ldb < n || ldc < m) return fail(ctx, GEO_EINVAL, "leading dimension below the row count");
    if (slices == 0) slices = 8;
    if (slices < 3 || slices > 8) return fail(ctx, GEO_EINVAL, "slices must be 0 (default 8) or 3..8");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_buffer(ctx, &ctx->ows, &ctx->ows_bytes, oz_gemm_workspace_bytes(m, n, k, slices), s);
    if (rc) return rc;
    CK(cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s));
    CK(oz_gemm(m, n, k, A_dev, lda, B_dev, ldb, C_dev, ldc, slices, ctx->ows, ctx->st, s));
    CK(cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->h_st->timeout) return fail(ctx, GEO_ETIMEOUT, "a bounded device wait expired");
    return GEO_OK;
}

namespace {
__global__ void k_identity(double *A, int N) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < (long long)N * N) A[t] = (t % N == t / N) ? 1.0 : 0.0;
}
}  // namespace

int geo_selftest_bounded_wait(geo_ctx *ctx, int n_blocks, long long wait_cycles, int *site, void *stream) {
    if (!ctx) return GEO_EINVAL;
    if (site) *site = 0;
    if (n_blocks < 2 || n_blocks > 64 || wait_cycles <= 0 || wait_cycles > 4000000000LL)
        return fail(ctx, GEO_EINVAL, "n_blocks must be in 2..64 and wait_cycles in 1..4e9");
    SetDevice sd(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int N = 64 * n_blocks;
    void *p = nullptr;
    int rc = dev_alloc(ctx, &p, sizeof(double) * ((size_t)N * N + N));
    if (rc) return rc;
    double *A = (double *)p, *x = A + (size_t)N * N;
    cudaError_t e;
    if ((e = cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s)) ||
        (e = cudaMemsetAsync(x, 0, sizeof(double) * N, s))) {
        dev_free(ctx, p, sizeof(double) * ((size_t)N * N + N));
        return cuda_fail(ctx, e, "geo_selftest_bounded_wait");
    }
    k_identity<<<(unsigned)(((long long)N * N + 255) / 256), 256, 0, s>>>(A, N);
    if ((e = cudaGetLastError()) ||
        (e = forward_solve_withheld(A, N, N, x, ctx->sync, &ctx->st->timeout, wait_cycles, s)) ||
        (e = cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s)) ||
        (e = cudaStreamSynchronize(s))) {
        cudaStreamSynchronize(s);
        dev_free(ctx, p, sizeof(double) * ((size_t)N * N + N));
        return cuda_fail(ctx, e, "geo_selftest_bounded_wait");
    }
    dev_free(ctx, p, sizeof(double) * ((size_t)N * N + N));
    const int code = ctx->h_st->timeout;
    if (site) *site = code;
    if (cudaMemsetAsync(ctx->st, 0, sizeof(DevStatus), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return cuda_fail(ctx, cudaGetLastError(), "geo_selftest_bounded_wait");
    if (code) return fail(ctx, GEO_ETIMEOUT, "the withheld dependency made the bounded wait give up (site " +
                                                 std::to_string(code) + ")");
    return GEO_OK;
}

int geo_profile_enable(geo_ctx *ctx, int enable) {
    if (!ctx) return GEO_EINVAL;
    SetDevice sd(ctx->device);
    if (enable) {
        cudaDeviceSynchronize();
        ctx->prof.clear();
        if (ctx->prof.d_tc_flops) cudaMemset(ctx->prof.d_tc_flops, 0, sizeof(unsigned long long));
    }
    ctx->prof.enabled = enable != 0;
    return GEO_OK;
}

int geo_profile_read(geo_ctx *ctx, geo_kstat *out) {
    if (!ctx || !out) return GEO_EINVAL;
    SetDevice sd(ctx->device);
    CK(cudaDeviceSynchronize());
    ctx->prof.resolve();
    for (int k = 0; k < GEO_K_COUNT; ++k) {
        out[k].launches = ctx->prof.launches[k];
        out[k].ms = ctx->prof.ms[k];
        out[k].flops = ctx->prof.flops[k];
        out[k].bytes = ctx->prof.bytes[k];
        out[k].timed = ctx->prof.timed[k];
        out[k].tensor_flops = 0.0;
    }
    unsigned long long tc = 0;
    if (ctx->prof.d_tc_flops)
        CK(cudaMemcpy(&tc, ctx->prof.d_tc_flops, sizeof(tc), cudaMemcpyDeviceToHost));
    out[GEO_K_TCGEMM].tensor_flops = (double)tc;
    return GEO_OK;
}

int geo_abi_layout(long long *out, int n) {
    const long long v[] = {(long long)sizeof(geo_theta),        (long long)sizeof(geo_opts),
                           (long long)sizeof(geo_factor_stats), (long long)sizeof(geo_mle_state),
                           (long long)sizeof(geo_batch_item),   (long long)sizeof(geo_request),
                           (long long)sizeof(geo_result),       (long long)sizeof(geo_kstat),
                           (long long)offsetof(geo_opts, oz_slices), (long long)offsetof(geo_opts, oz_cut),
                           (long long)offsetof(geo_kstat, tensor_flops)};
    const int count = (int)(sizeof(v) / sizeof(v[0]));
    if (n > 0 && !out) return GEO_EINVAL;
    for (int k = 0; k < n && k < count; ++k) out[k] = v[k];
    return count;
}

int geo_morton_order(const double *locs_host, int n, int *perm_host) {
    if (n < 0 || (n > 0 && (!locs_host || !perm_host))) return GEO_EINVAL;
    morton_perm_host(locs_host, n, perm_host);
    return GEO_OK;
}

}  // extern "C"

// ---- for the request server (serve.cu) --------------------------------------

size_t ctx_device_bytes(const geo_ctx *ctx) { return ctx ? ctx->used : 0; }

size_t ctx_trim(geo_ctx *ctx, cudaStream_t s) {
    if (!ctx) return 0;
    SetDevice sd(ctx->device);
    cudaStreamSynchronize(s);
    const size_t before = ctx->used;
    void **bufs[] = {(void **)&ctx->ws, &ctx->mws, &ctx->sws, &ctx->zws, &ctx->rws, &ctx->tws, &ctx->bws, &ctx->ows};
    size_t *sizes[] = {&ctx->ws_bytes, &ctx->mws_bytes, &ctx->sws_bytes, &ctx->zws_bytes,
                       &ctx->rws_bytes, &ctx->tws_bytes, &ctx->bws_bytes, &ctx->ows_bytes};
    for (int k = 0; k < 8; ++k) {
        dev_free(ctx, *bufs[k], *sizes[k]);
        *bufs[k] = nullptr;
        *sizes[k] = 0;
    }
    // batch graphs refer to the freed batch workspace
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.second.first);
    ctx->graphs.clear();
    return before - ctx->used;
}

size_t loglik_device_bytes(int device, int n, int p, const geo_opts *opts) {
    geo_opts o;
    if (opts)
        o = *opts;
    else
        geo_opts_default(&o);
    const size_t N = (size_t)p * n;
    if (o.nb == 0) o.nb = resolve_nb(device, form_of(o), (int)N);
    const size_t nb = (size_t)std::max(o.nb, 64);
    size_t b = sizeof(double) * (2 * (size_t)n + GEO_TAB_DOUBLES) + sizeof(int) * 2 * n + sizeof(double) * N;
    if (o.prec == GEO_PREC_TLR) {
        const int kmax = std::min(o.tlr_kmax, (int)nb);
        const size_t T = (N + nb - 1) / nb;
        b += tlr_factor_bytes((int)N, (int)nb, kmax) + sizeof(double) * N;
        b += std::max(tlr_workspace_bytes((int)N, (int)nb, kmax), tlr_solve_workspace_bytes((int)N, (int)nb, kmax));
        b += sizeof(double) * (T * (T - 1) / 2) * 2 * nb * nb;   // U / V pool if every tile fell back to dense
        return b + ((size_t)1 << 24);
    }
    const size_t ld = (size_t)round_up((long long)N + 1, 32);
    b += sizeof(double) * ld * N;
    if (o.prec == GEO_PREC_FP64 && o.fp64_gemm == 1) b += oz_chol_workspace_bytes((int)N + 1, (int)nb, oz_slices_of(o));
    if (o.prec == GEO_PREC_MIXED) {
        b += mixed_workspace_bytes((int)N, (int)nb);
        if (o.refine_iters > 0) b += sizeof(double) * ld * N + sizeof(double) * N + refine_workspace_bytes((int)N);
    }
    return b;
}
