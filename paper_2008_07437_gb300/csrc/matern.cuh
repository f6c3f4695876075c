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
#pragma once

#ifndef GEO_DEV
#define GEO_DEV __device__ __forceinline__
#endif

#define GEO_PMAX_DEV 4

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
};

struct CovParams {
    int p;
    double inv_a;                                     // 1 / a
    MaternConst m[GEO_PMAX_DEV * GEO_PMAX_DEV];       // m[i * p + j], symmetric
};

// x^nu K_nu(x) for x > 0, general order.
GEO_DEV double xnu_besselk(double x, const MaternConst &c) {
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
    if (scaled) return exp(c.nu * log(x) - x) * kv;
    return exp(c.nu * log(x)) * kv;
}

// C_ij(h) of Eq. 2 given x = h / a (x >= 0).
GEO_DEV double matern_cov(double x, const MaternConst &c) {
    if (x == 0.0) return c.c0;
    switch (c.kind) {
        case 1: return c.c0 * exp(-x);
        case 2: return c.c0 * (1.0 + x) * exp(-x);
        case 3: return c.c0 * (1.0 + x + x * x * (1.0 / 3.0)) * exp(-x);
        default: return c.pre * xnu_besselk(x, c);
    }
}
