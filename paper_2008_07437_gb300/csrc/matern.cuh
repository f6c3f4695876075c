// Device evaluation of the parsimonious multivariate Matern covariance, Eq. 2
// (Sec. 4.2), with an FP64 modified Bessel function K_nu of real order.
//
// K_nu has no CUDA library routine, so it is computed here from two published
// methods (no library source was used):
//
// * x <= 2: Temme's series (N. M. Temme, "On the numerical evaluation of the
//   modified Bessel function of the third kind", J. Comput. Phys. 19 (1975)
//   324-337).  With nu = mu + nl, |mu| <= 1/2, c_k = (x^2/4)^k / k!,
//     K_mu     = sum_k c_k f_k,
//     K_{mu+1} = (2/x) sum_k c_k (p_k - k f_k),
//     p_0 = (x/2)^-mu Gamma(1+mu) / 2, q_0 = (x/2)^mu Gamma(1-mu) / 2,
//     f_0 = (mu pi / sin mu pi) [cosh(s) G1(mu) + sinh(s)/s ln(2/x) G2(mu)], s = mu ln(2/x),
//     f_k = (k f_{k-1} + p_{k-1} + q_{k-1}) / (k^2 - mu^2),
//     p_k = p_{k-1} / (k - mu), q_k = q_{k-1} / (k + mu),
//   with G1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu) and
//   G2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2 computed on the host per theta.
//
// * x > 2: K_mu(x) = sqrt(pi) (2x)^mu e^-x U(mu + 1/2, 2 mu + 1, 2x) (Tricomi U).
//   u_k = U(mu + 1/2 + k, 2 mu + 1, 2x) is the minimal solution of
//     u_{k-1} - 2 (k + x) u_k + ((k + 1/2)^2 - mu^2) u_{k+1} = 0,
//   so its ratios r_k = u_{k+1}/u_k follow from a backward recurrence started
//   at r_K = 0 (Miller's principle; the continued fraction of Steed's method
//   evaluated backwards).  The binomial series of (1 + t)^(1/2 - mu) inside
//   the integral representation of U gives the normalisation
//     sum_k C_k u_k = (2x)^-(mu + 1/2),  C_k = prod_{j<k} ((j + 1/2)^2 - mu^2) / k!,
//   hence e^x K_mu(x) = sqrt(pi / (2x)) / S with S = sum_k C_k u_k / u_0,
//   accumulated backwards with the ratios.  The contiguous relations of U
//   give K_{mu+1}/K_mu = 1 + (mu + 1/2)/x + (mu^2 - 1/4) r_0 / x.
//
// Orders above 1/2 use the upward recurrence K_{v+1} = K_{v-1} + (2 v / x) K_v,
// which is stable for K.  Half-integer orders 1/2, 3/2, 5/2 use the exact
// closed forms of Eq. 2 (exponential times a polynomial).
//
// Those two methods are the reference evaluator.  The covariance kernels use
// a per-theta table built from it on the device (k_cheb_build): for each
// order nu_ij <= 3 that is not a half-integer,
//   F(x) = e^x x^nu K_nu(x)
// is interpolated on every dyadic interval [2^k, 2^(k+1)), k = -2 .. 9, by the
// Chebyshev polynomial of degree 23 through the 24 Chebyshev nodes of the
// interval.  F is analytic except at x = 0, which lies three half-widths from
// the centre of every such interval, so the interpolation error falls like
// (3 + sqrt 8)^-24: below 1e-19 relative up to nu = 3 (checked against
// arbitrary-precision K_nu).  Then x^nu K_nu(x) = e^-x F(x): one Clenshaw sum
// per order, and one exponential per location pair shared by all the orders
// (and the half-integer closed forms), instead of a recurrence of up to ~90
// terms with two divisions each.  Below x = 1/4
// Temme's series is used with the reciprocals 1/(k^2 - mu^2), 1/(k -+ mu), 1/k
// taken from the table (no divisions in the loop); at x >= 1024 the
// covariance underflows to 0.
#pragma once

#ifndef GEO_DEV
#define GEO_DEV __device__ __forceinline__
#endif

#define GEO_PMAX_DEV 4

// Chebyshev table of one order nu_ij: GEO_CHEB_NI intervals x GEO_CHEB_N
// coefficients, then the Temme reciprocals 1/(k^2 - mu^2), 1/(k - mu),
// 1/(k + mu) and 1/k for k = 1 .. GEO_TEMME_K.
#define GEO_CHEB_N 24
#define GEO_CHEB_K0 (-2)
#define GEO_CHEB_NI 12
#define GEO_TEMME_K 24
#define GEO_CHEB_NU_MAX 3.0
#define GEO_TAB_PER_PAIR (GEO_CHEB_NI * GEO_CHEB_N + 4 * GEO_TEMME_K)
#define GEO_TAB_DOUBLES (GEO_PMAX_DEV * (GEO_PMAX_DEV + 1) / 2 * GEO_TAB_PER_PAIR)

// Per (i, j) constants of Eq. 2 for one theta, computed on the host.
struct MaternConst {
    double nu;     // nu_ij
    double mu;     // reduced order: nu = mu + nl, -1/2 <= mu < 1/2
    double c0;     // rho_ij sigma_i sigma_j = C_ij(0)
    double pre;    // c0 / (2^(nu - 1) Gamma(nu))
    double g1;     // G1(mu)
    double g2;     // G2(mu)
    double gp;     // Gamma(1 + mu)
    double gm;     // Gamma(1 - mu)
    double fact;   // mu pi / sin(mu pi)  (1 at mu = 0)
    int nl;        // number of upward recurrence steps
    int kind;      // 0 general order, 1: nu = 1/2, 2: nu = 3/2, 3: nu = 5/2
    int toff;      // general order <= GEO_CHEB_NU_MAX: offset of its table in CovParams::tab; else -1
};

struct CovParams {
    int p;
    double inv_a;                                     // 1 / a
    const double *tab;                                // device tables (k_cheb_build), or null
    MaternConst m[GEO_PMAX_DEV * GEO_PMAX_DEV];       // m[i * p + j], symmetric
};

// e^x K_nu(x) (x > 2) or K_nu(x) (x <= 2) for x > 0, general order, by the
// reference methods; *scaled tells which.
GEO_DEV double besselk_ref(double x, const MaternConst &c, bool *scaled_out) {
    const double mu = c.mu;
    double kmu, kmu1;   // K_mu and K_{mu+1}, scaled by e^x when x > 2
    bool scaled;
    if (x <= 2.0) {
        scaled = false;
        const double lx = log(2.0 / x);
        const double s = mu * lx;
        double shs;
        if (fabs(s) < 1e-3) {
            const double s2 = s * s;
            shs = 1.0 + s2 * (1.0 / 6.0 + s2 * (1.0 / 120.0 + s2 * (1.0 / 5040.0)));
        } else {
            shs = sinh(s) / s;
        }
        const double es = exp(s);                 // (x/2)^-mu
        double f = c.fact * (cosh(s) * c.g1 + shs * lx * c.g2);
        double pk = 0.5 * es * c.gp;
        double qk = 0.5 / es * c.gm;
        const double d = 0.25 * x * x;
        double ck = 1.0;
        double sum = f, sum1 = pk;
        const double mu2 = mu * mu;
        for (int k = 1; k < 64; ++k) {
            const double kd = (double)k;
            f = (kd * f + pk + qk) / (kd * kd - mu2);
            ck *= d / kd;
            pk /= (kd - mu);
            qk /= (kd + mu);
            const double del = ck * f;
            sum += del;
            sum1 += ck * (pk - kd * f);
            if (fabs(del) < 1e-17 * fabs(sum)) break;
        }
        kmu = sum;
        kmu1 = sum1 * (2.0 / x);
    } else {
        scaled = true;
        const double mu2 = mu * mu;
        const int K = (int)(160.0 / x) + 10;
        double r = 0.0, A = 1.0;
        for (int k = K - 1; k >= 0; --k) {
            const double kd = (double)k;
            const double b = kd + 1.5;
            r = 1.0 / (2.0 * (kd + 1.0 + x) - (b * b - mu2) * r);
            const double a = kd + 0.5;
            A = 1.0 + (a * a - mu2) / (kd + 1.0) * r * A;
        }
        kmu = sqrt(1.5707963267948966 / x) / A;    // sqrt(pi / (2x)) / S
        kmu1 = kmu * (1.0 + (mu + 0.5) / x + (mu2 - 0.25) * r / x);
    }
    // upward recurrence from (K_mu, K_{mu+1}) to K_nu = K_{mu+nl}
    double kv;
    if (c.nl == 0) {
        kv = kmu;
    } else {
        double km = kmu, k0 = kmu1;
        for (int j = 1; j < c.nl; ++j) {
            const double kn = km + 2.0 * (mu + (double)j) / x * k0;
            km = k0;
            k0 = kn;
        }
        kv = k0;
    }
    *scaled_out = scaled;
    return kv;
}

// x^nu K_nu(x) by the reference methods.
GEO_DEV double xnu_besselk(double x, const MaternConst &c) {
    bool scaled;
    const double kv = besselk_ref(x, c, &scaled);
    if (scaled) return exp(c.nu * log(x) - x) * kv;
    return exp(c.nu * log(x)) * kv;
}

// F(x) = e^x x^nu K_nu(x), reference methods (table construction).
GEO_DEV double besselk_f_ref(double x, const MaternConst &c) {
    bool scaled;
    const double kv = besselk_ref(x, c, &scaled);
    const double xnu = exp(c.nu * log(x));
    return scaled ? xnu * kv : exp(x) * xnu * kv;
}

// One block of 32 threads of the table construction for order q = i p + j
// (i <= j) and interval k (k = GEO_CHEB_NI: the reciprocals), from the
// reference evaluator.  Node values F(x_t) at x_t = mid + half cos(pi (t + 1/2) / n),
// coefficients c_m = (2 - [m = 0]) / n sum_t F(x_t) cos(pi m (t + 1/2) / n),
// each summed in a fixed order.  hv: GEO_CHEB_N doubles of shared memory.
__device__ __forceinline__ void cheb_build_block(const CovParams &cp, double *tab, int q, int k, double *hv) {
    const int p = cp.p;
    if (q >= p * p || q % p < q / p) return;
    const MaternConst &c = cp.m[q];
    if (c.kind != 0 || c.toff < 0) return;
    double *T = tab + c.toff;
    const int t = threadIdx.x;
    if (k == GEO_CHEB_NI) {
        if (t < GEO_TEMME_K) {
            const double kd = (double)(t + 1), mu = c.mu;
            double *R = T + GEO_CHEB_NI * GEO_CHEB_N;
            R[t] = 1.0 / (kd * kd - mu * mu);
            R[GEO_TEMME_K + t] = 1.0 / (kd - mu);
            R[2 * GEO_TEMME_K + t] = 1.0 / (kd + mu);
            R[3 * GEO_TEMME_K + t] = 1.0 / kd;
        }
        return;
    }
    const double lo = ldexp(1.0, GEO_CHEB_K0 + k);
    if (t < GEO_CHEB_N) {
        const double xt = 1.5 * lo + 0.5 * lo * cospi((t + 0.5) / GEO_CHEB_N);
        hv[t] = besselk_f_ref(xt, c);
    }
    __syncthreads();
    if (t < GEO_CHEB_N) {
        double sum = 0.0;
        for (int m = 0; m < GEO_CHEB_N; ++m) sum += hv[m] * cospi(t * (m + 0.5) / GEO_CHEB_N);
        T[k * GEO_CHEB_N + t] = sum * ((t == 0) ? 1.0 : 2.0) / GEO_CHEB_N;
    }
}

// x^nu K_nu(x) for 0 < x < 1/4: Temme's series with tabulated reciprocals,
// then the upward recurrence.
GEO_DEV double xnu_besselk_small(double x, const MaternConst &c, const double *rt) {
    const double mu = c.mu;
    const double lx = log(2.0 / x);
    const double s = mu * lx;
    const double es = exp(s);                 // (x/2)^-mu
    const double ies = 1.0 / es;
    double shs;
    if (fabs(s) < 1e-3) {
        const double s2 = s * s;
        shs = 1.0 + s2 * (1.0 / 6.0 + s2 * (1.0 / 120.0 + s2 * (1.0 / 5040.0)));
    } else {
        shs = 0.5 * (es - ies) / s;
    }
    double f = c.fact * (0.5 * (es + ies) * c.g1 + shs * lx * c.g2);
    double pk = 0.5 * es * c.gp;
    double qk = 0.5 * ies * c.gm;
    const double d = 0.25 * x * x;
    double ck = 1.0;
    double sum = f, sum1 = pk;
    for (int k = 1; k <= GEO_TEMME_K; ++k) {
        const double kd = (double)k;
        f = (kd * f + pk + qk) * rt[k - 1];
        ck *= d * rt[3 * GEO_TEMME_K + k - 1];
        pk *= rt[GEO_TEMME_K + k - 1];
        qk *= rt[2 * GEO_TEMME_K + k - 1];
        const double del = ck * f;
        sum += del;
        sum1 += ck * (pk - kd * f);
        if (fabs(del) < 1e-17 * fabs(sum)) break;
    }
    const double ix = 1.0 / x;
    double kv;
    if (c.nl == 0) {
        kv = sum;
    } else {
        double km = sum, k0 = 2.0 * ix * sum1;
        for (int j = 1; j < c.nl; ++j) {
            const double kn = km + 2.0 * (mu + (double)j) * ix * k0;
            km = k0;
            k0 = kn;
        }
        kv = k0;
    }
    return exp(c.nu * (0.6931471805599453 - lx)) * kv;   // ln x = ln 2 - ln(2/x)
}

// F(x) = e^x x^nu K_nu(x) for 1/4 <= x < 1024 from the Chebyshev table of the order.
GEO_DEV double cheb_f(double x, const double *tab) {
    const int e = ilogb(x);                              // x in [2^e, 2^(e+1))
    const double *cf = tab + (e - GEO_CHEB_K0) * GEO_CHEB_N;
    const double t = ldexp(x, 1 - e) - 3.0;              // exact map to [-1, 1)
    const double t2 = t + t;
    double b1 = 0.0, b2 = 0.0;
#pragma unroll
    for (int m = GEO_CHEB_N - 1; m >= 1; --m) {
        const double b0 = fma(t2, b1, cf[m]) - b2;
        b2 = b1;
        b1 = b0;
    }
    return fma(t, b1, cf[0]) - b2;
}

// C_ij(h) of Eq. 2 given x = h / a (x >= 0), reference methods only.
GEO_DEV double matern_cov_ref(double x, const MaternConst &c) {
    if (x == 0.0) return c.c0;
    switch (c.kind) {
        case 1: return c.c0 * exp(-x);
        case 2: return c.c0 * (1.0 + x) * exp(-x);
        case 3: return c.c0 * (1.0 + x + x * x * (1.0 / 3.0)) * exp(-x);
        default: return c.pre * xnu_besselk(x, c);
    }
}

// C_ij(h) of Eq. 2 given x = h / a > 0 and emx = e^-x; tab: the theta's tables.
GEO_DEV double matern_cov_e(double x, double emx, const MaternConst &c, const double *tab) {
    switch (c.kind) {
        case 1: return c.c0 * emx;
        case 2: return c.c0 * (1.0 + x) * emx;
        case 3: return c.c0 * (1.0 + x + x * x * (1.0 / 3.0)) * emx;
        default:
            if (c.toff < 0 || !tab) return c.pre * xnu_besselk(x, c);
            if (x >= 1024.0) return 0.0;
            if (x < 0.25) return c.pre * xnu_besselk_small(x, c, tab + c.toff + GEO_CHEB_NI * GEO_CHEB_N);
            return c.pre * emx * cheb_f(x, tab + c.toff);
    }
}

// C_ij(h) of Eq. 2 given x = h / a (x >= 0); tab: the theta's tables.
GEO_DEV double matern_cov(double x, const MaternConst &c, const double *tab) {
    if (x == 0.0) return c.c0;
    return matern_cov_e(x, exp(-x), c, tab);
}

// The p x p block of C at x = h / a: v[i * GEO_PMAX_DEV + j], each distinct
// (i, j) evaluated once, one exponential shared by all of them.
GEO_DEV void matern_block(double x, const CovParams &cp, double *v) {
    const int p = cp.p;
    const double emx = exp(-x);
    for (int i = 0; i < p; ++i)
        for (int j = i; j < p; ++j) {
            const MaternConst &c = cp.m[i * p + j];
            const double val = (x == 0.0) ? c.c0 : matern_cov_e(x, emx, c, cp.tab);
            v[i * GEO_PMAX_DEV + j] = val;
            v[j * GEO_PMAX_DEV + i] = val;
        }
}
