// Maximum likelihood estimation of theta (Sec. 1 / Sec. 5.1: the MLE
// maximises Eq. 1, rebuilding Sigma(theta) at every evaluation; the paper
// uses NLopt without naming the algorithm).  Here: the Nelder-Mead simplex
// method with the textbook coefficients (reflection 1, expansion 2,
// contraction 1/2, shrink 1/2), minimising f(x) = -l(theta(x)) over
//   x = (log sigma^2_1..p, log a, log nu_1..p, beta_ij for i < j).
// Every evaluation is one geo_loglik on the device; this file only keeps the
// simplex.  The state is a plain caller-owned struct, so a run can be saved
// and resumed at any step.  Profile runs (Sec. 4.2) drop the sigma^2 from x,
// x = (log a, log nu_1..p, beta_ij for i < j), evaluate geo_loglik_profile and
// carry each vertex's sigma^2 estimate beside it.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "geo_internal.cuh"

namespace {

int q_of(int p, bool profile) { return (profile ? p : 2 * p) + 1 + p * (p - 1) / 2; }

struct ThetaBuf {
    double sigma2[GEO_PMAX], nu[GEO_PMAX], beta[GEO_PMAX * GEO_PMAX];
    geo_theta th;
};

// Full coordinates, or the profile ones (no sigma^2: x starts at log a, sigma^2 = 1).
void x_to_theta(const double *x, int p, bool profile, ThetaBuf *t) {
    const int o = profile ? 0 : p;
    for (int i = 0; i < p; ++i) t->sigma2[i] = profile ? 1.0 : exp(x[i]);
    const double a = exp(x[o]);
    for (int i = 0; i < p; ++i) t->nu[i] = exp(x[o + 1 + i]);
    int k = o + p + 1;
    for (int i = 0; i < p; ++i) {
        t->beta[i * p + i] = 1.0;
        for (int j = i + 1; j < p; ++j) {
            t->beta[i * p + j] = t->beta[j * p + i] = x[k++];
        }
    }
    t->th.p = p;
    t->th.sigma2 = t->sigma2;
    t->th.nu = t->nu;
    t->th.beta = t->beta;
    t->th.a = a;
}

// Unpivoted Cholesky of beta: every pivot must be > 0.
bool beta_pd(const double *beta, int p) {
    double L[GEO_PMAX][GEO_PMAX] = {};
    for (int j = 0; j < p; ++j) {
        double s = beta[j * p + j];
        for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
        if (!(s > 0.0)) return false;
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < p; ++i) {
            double t = beta[i * p + j];
            for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    return true;
}

struct Eval {
    geo_ctx *ctx;
    const double *locs;
    int n;
    const double *z;
    const geo_opts *opts;
    void *stream;
    geo_mle_state *st;
    int err = GEO_OK;

    // -l at x; a profile evaluation also leaves its sigma^2 estimate in s2 (NaN when infeasible)
    double operator()(const double *x, double *s2 = nullptr) {
        ThetaBuf t;
        const bool prof = st->profile != 0;
        x_to_theta(x, st->p, prof, &t);
        st->evals += 1;
        double tmp[GEO_PMAX];
        double *out = s2 ? s2 : tmp;
        for (int i = 0; i < st->p; ++i) out[i] = nan("");
        if (!beta_pd(t.beta, st->p)) {
            st->last_f = INFINITY;
            return INFINITY;
        }
        double l = 0.0;
        int rc = prof ? geo_loglik_profile(ctx, locs, n, z, &t.th, opts, &l, out, nullptr, stream)
                      : geo_loglik(ctx, locs, n, z, &t.th, opts, &l, nullptr, nullptr, stream);
        double f;
        if (rc == GEO_ENOTSPD || rc == GEO_EINVAL) {
            f = INFINITY;
        } else if (rc != GEO_OK) {
            err = rc;
            f = INFINITY;
        } else {
            f = -l;
        }
        st->last_f = f;
        return f;
    }
};

void order(geo_mle_state *s) {
    const int q = s->q;
    std::vector<int> idx(q + 1);
    for (int k = 0; k <= q; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s->f[a] < s->f[b]; });
    double X[GEO_MLE_QMAX + 1][GEO_MLE_QMAX], F[GEO_MLE_QMAX + 1], S2[GEO_MLE_QMAX + 1][GEO_PMAX];
    for (int k = 0; k <= q; ++k) {
        memcpy(X[k], s->x[idx[k]], sizeof(double) * q);
        memcpy(S2[k], s->s2[idx[k]], sizeof(double) * GEO_PMAX);
        F[k] = s->f[idx[k]];
    }
    for (int k = 0; k <= q; ++k) {
        memcpy(s->x[k], X[k], sizeof(double) * q);
        memcpy(s->s2[k], S2[k], sizeof(double) * GEO_PMAX);
        s->f[k] = F[k];
    }
}

// Replace the worst vertex by (x, f, sigma^2).
void take(geo_mle_state *s, const double *x, double f, const double *s2) {
    memcpy(s->x[s->q], x, sizeof(double) * s->q);
    memcpy(s->s2[s->q], s2, sizeof(double) * GEO_PMAX);
    s->f[s->q] = f;
}

int init_common(geo_mle_state *s, const geo_theta *th, double step, bool profile) {
    if (!s || !th || th->p < 1 || th->p > GEO_PMAX || !th->nu || (th->p > 1 && !th->beta)) return GEO_EINVAL;
    const int p = th->p;
    const int q = q_of(p, profile);
    if (q > GEO_MLE_QMAX) return GEO_EINVAL;
    if (!profile && !th->sigma2) return GEO_EINVAL;
    memset(s, 0, sizeof(*s));
    s->p = p;
    s->q = q;
    s->step = step;
    s->profile = profile ? 1 : 0;
    const int o = profile ? 0 : p;
    double x0[GEO_MLE_QMAX];
    for (int i = 0; i < p; ++i) {
        if (!(th->nu[i] > 0)) return GEO_EINVAL;
        if (!profile) {
            if (!(th->sigma2[i] > 0)) return GEO_EINVAL;
            x0[i] = log(th->sigma2[i]);
        }
        x0[o + 1 + i] = log(th->nu[i]);
    }
    if (!(th->a > 0)) return GEO_EINVAL;
    x0[o] = log(th->a);
    int k = o + p + 1;
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) x0[k++] = th->beta[i * p + j];
    for (int v = 0; v <= q; ++v) {
        memcpy(s->x[v], x0, sizeof(double) * q);
        if (v > 0) s->x[v][v - 1] = s->x[v][v - 1] + step;
    }
    return GEO_OK;
}

}  // namespace

extern "C" {

int geo_mle_init(geo_mle_state *s, const geo_theta *th, double step) { return init_common(s, th, step, false); }

int geo_mle_init_profile(geo_mle_state *s, const geo_theta *th, double step) {
    return init_common(s, th, step, true);
}

int geo_mle_step(geo_ctx *ctx, geo_mle_state *s, const double *locs_dev, int n, const double *z_dev,
                 const geo_opts *opts, void *stream) {
    if (!ctx || !s || s->q < 1 || s->q > GEO_MLE_QMAX) return GEO_EINVAL;
    Eval f{ctx, locs_dev, n, z_dev, opts, stream, s};
    const int q = s->q;
    if (!s->initialized) {
        for (int v = 0; v <= q; ++v) {
            s->f[v] = f(s->x[v], s->s2[v]);
            if (f.err) return f.err;
        }
        order(s);
        s->initialized = 1;
        return GEO_OK;
    }
    double xbar[GEO_MLE_QMAX], xr[GEO_MLE_QMAX], xe[GEO_MLE_QMAX], xc[GEO_MLE_QMAX];
    double sr[GEO_PMAX] = {}, se[GEO_PMAX] = {}, sc[GEO_PMAX] = {};
    for (int d = 0; d < q; ++d) xbar[d] = 0.0;
    for (int k = 0; k < q; ++k)
        for (int d = 0; d < q; ++d) xbar[d] = xbar[d] + s->x[k][d];
    for (int d = 0; d < q; ++d) xbar[d] = xbar[d] / q;
    const double *xw = s->x[q];
    const double fw = s->f[q];
    for (int d = 0; d < q; ++d) xr[d] = xbar[d] + 1.0 * (xbar[d] - xw[d]);
    const double fr = f(xr, sr);
    if (f.err) return f.err;
    if (s->f[0] <= fr && fr < s->f[q - 1]) {
        take(s, xr, fr, sr);
    } else if (fr < s->f[0]) {
        for (int d = 0; d < q; ++d) xe[d] = xbar[d] + 2.0 * (xr[d] - xbar[d]);
        const double fe = f(xe, se);
        if (f.err) return f.err;
        if (fe < fr)
            take(s, xe, fe, se);
        else
            take(s, xr, fr, sr);
    } else {
        bool shrink = false;
        if (fr < fw) {
            for (int d = 0; d < q; ++d) xc[d] = xbar[d] + 0.5 * (xr[d] - xbar[d]);
            const double fc = f(xc, sc);
            if (f.err) return f.err;
            if (fc <= fr)
                take(s, xc, fc, sc);
            else
                shrink = true;
        } else {
            for (int d = 0; d < q; ++d) xc[d] = xbar[d] - 0.5 * (xbar[d] - xw[d]);
            const double fc = f(xc, sc);
            if (f.err) return f.err;
            if (fc < fw)
                take(s, xc, fc, sc);
            else
                shrink = true;
        }
        if (shrink) {
            for (int k = 1; k <= q; ++k) {
                for (int d = 0; d < q; ++d) s->x[k][d] = s->x[0][d] + 0.5 * (s->x[k][d] - s->x[0][d]);
                s->f[k] = f(s->x[k], s->s2[k]);
                if (f.err) return f.err;
            }
        }
    }
    order(s);
    s->iter += 1;
    return GEO_OK;
}

int geo_mle_best(const geo_mle_state *s, double *sigma2, double *a, double *nu, double *beta, double *loglik) {
    if (!s || s->p < 1) return GEO_EINVAL;
    ThetaBuf t;
    x_to_theta(s->x[0], s->p, s->profile != 0, &t);
    for (int i = 0; i < s->p; ++i) {
        if (sigma2) sigma2[i] = s->profile ? (s->initialized ? s->s2[0][i] : nan("")) : t.sigma2[i];
        if (nu) nu[i] = t.nu[i];
    }
    if (a) *a = t.th.a;
    if (beta) memcpy(beta, t.beta, sizeof(double) * s->p * s->p);
    if (loglik) *loglik = s->initialized ? -s->f[0] : nan("");
    return GEO_OK;
}

}  // extern "C"
