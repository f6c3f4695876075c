/*
 * CPU FP64 oracle for the multivariate Matern log-likelihood and cokriging
 * (arxiv 2008.07437).  TEST INFRASTRUCTURE ONLY: a slow, plain, obviously
 * correct restatement of the paper's formulas.  Only the tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no code, header or constant with the CUDA path.
 *
 * Every function cites the passage it follows:
 *   Eq. 1  (Sec. 1)    log-likelihood l(theta) = -(np/2)log(2 pi) - 1/2 log|Sigma| - 1/2 Z' Sigma^-1 Z
 *   Eq. 2  (Sec. 4.2)  parsimonious multivariate Matern C_ij(h)
 *   Sec. 4.2           nu_ij = (nu_ii + nu_jj)/2 and the colocated correlation rho_ij
 *   Sec. 5.2           Representation I: row index p*l + i (location-major, variable-minor)
 *   Eq. 3, Eq. 4       cokriging predictor Zhat(s0) = c0' Sigma^-1 Z (Sec. 4.3)
 *
 * Readings where the paper is ambiguous:
 *   - rho_ij: the square roots apply to the marginal Gamma ratios only, so that
 *     rho_ii = 1 and C_ii(0) = sigma_ii^2.
 *   - sigma_ii in Eq. 2 is the square root of the variance parameter sigma_ii^2.
 *   - h = 0 takes the limit of Eq. 2, rho_ij sigma_ii sigma_jj; no nugget.
 *   - Distances are Euclidean in d = 2.
 *
 * Precision: double throughout.  The Bessel function K_nu uses a different
 * algorithm from the device (trapezoid quadrature of an integral
 * representation, not a series / continued fraction).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/*
 * e^x K_nu(x) for x > 0, from the integral representation
 *     K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 * (a standard identity for the modified Bessel function of the second kind,
 * the function in Eq. 2), written as
 *     e^x K_nu(x) = int_0^inf exp(-2 x sinh^2(t/2)) cosh(nu t) dt
 * so that nothing underflows for large x.  The integrand is even and entire,
 * so the trapezoid rule on [0, inf) converges geometrically in 1/h.  The step
 * keeps x h^2 <= 1/4, which keeps the aliasing error of the Gaussian-like peak
 * near t = 0 below e^-79 for large x; for small x the step 0.05 gives an error
 * of order e^-98.  Summation is compensated (Kahan) and stops once the
 * integrand is decreasing and below 1e-20 of the running sum.
 */
double oracle_besselk_scaled(double nu, double x) {
    double h = 0.05;
    double hx = 0.5 / sqrt(x);
    if (hx < h) h = hx;
    double tpeak = asinh(fabs(nu) / x);
    double sum = 0.5, comp = 0.0; /* t = 0 contributes f(0)/2 = 1/2 */
    for (long k = 1; k < 10000000L; k++) {
        double t = (double)k * h;
        double s = sinh(0.5 * t);
        double f = exp(-2.0 * x * s * s) * cosh(nu * t);
        double y = f - comp;
        double tmp = sum + y;
        comp = (tmp - sum) - y;
        sum = tmp;
        if (t > tpeak && f < 1e-20 * sum) break;
    }
    return h * sum;
}

double oracle_besselk(double nu, double x) {
    return exp(-x) * oracle_besselk_scaled(nu, x);
}

/*
 * Sec. 4.2: nu_ij = (nu_ii + nu_jj) / 2 and
 *   rho_ij = beta_ij * sqrt(G(nu_i + d/2)/G(nu_i)) * sqrt(G(nu_j + d/2)/G(nu_j))
 *            * G(nu_ij) / G(nu_ij + d/2)
 * (reading: square roots on the marginal ratios only, so rho_ii = 1).
 * Outputs are p x p row-major.
 */
void oracle_matern_params(int p, int d, const double *nu, const double *beta,
                          double *rho, double *nuij) {
    double hd = 0.5 * (double)d;
    for (int i = 0; i < p; i++) {
        for (int j = 0; j < p; j++) {
            double nij = 0.5 * (nu[i] + nu[j]);
            double gi = tgamma(nu[i] + hd) / tgamma(nu[i]);
            double gj = tgamma(nu[j] + hd) / tgamma(nu[j]);
            double bij = (i == j) ? 1.0 : beta[i * p + j];
            rho[i * p + j] = bij * sqrt(gi) * sqrt(gj) * tgamma(nij) / tgamma(nij + hd);
            nuij[i * p + j] = nij;
        }
    }
}

/*
 * Eq. 2:  C_ij(h) = rho_ij sigma_i sigma_j / (2^(nu_ij - 1) Gamma(nu_ij)) (h/a)^nu_ij K_nu_ij(h/a)
 * with the h = 0 limit rho_ij sigma_i sigma_j.
 */
double oracle_matern(double h, double a, double nuij, double rho_sig) {
    if (h == 0.0) return rho_sig;
    double x = h / a;
    /* (x)^nu K_nu(x) = exp(nu log x - x) * (e^x K_nu(x)) */
    double xk = exp(nuij * log(x) - x) * oracle_besselk_scaled(nuij, x);
    return rho_sig / (pow(2.0, nuij - 1.0) * tgamma(nuij)) * xk;
}

/*
 * Representation I cross-covariance (Sec. 5.2, Eq. 4): out is
 * (p*n1) x (p*n2), row-major, out[(p*l + i) * (p*n2) + (p*r + j)] =
 * C_ij(|s1_l - s2_r|).  Locations are n x 2 row-major (x, y).
 * sigma2, nu: p entries; beta: p x p row-major (diagonal ignored).
 */
void oracle_covgen(int p, const double *sigma2, const double *nu, const double *beta, double a,
                   const double *locs1, int n1, const double *locs2, int n2, double *out) {
    double *rho = (double *)malloc(sizeof(double) * p * p);
    double *nuij = (double *)malloc(sizeof(double) * p * p);
    oracle_matern_params(p, 2, nu, beta, rho, nuij);
    long ncol = (long)p * n2;
#pragma omp parallel for schedule(dynamic, 4)
    for (int l = 0; l < n1; l++) {
        for (int r = 0; r < n2; r++) {
            double dx = locs1[2 * l] - locs2[2 * r];
            double dy = locs1[2 * l + 1] - locs2[2 * r + 1];
            double h = sqrt(dx * dx + dy * dy);
            for (int i = 0; i < p; i++) {
                for (int j = 0; j < p; j++) {
                    double rs = rho[i * p + j] * sqrt(sigma2[i]) * sqrt(sigma2[j]);
                    out[((long)p * l + i) * ncol + (long)p * r + j] =
                        oracle_matern(h, a, nuij[i * p + j], rs);
                }
            }
        }
    }
    free(rho);
    free(nuij);
}

/*
 * Cholesky factorization Sigma = L L' (the factorization the paper uses to get
 * Sigma^-1 and log|Sigma|, Sec. 5.2), column-by-column Crout form: for each
 * column j, L_jj = sqrt(A_jj - sum_k<j L_jk^2), then every row i > j gets
 * L_ij = (A_ij - sum_k<j L_ik L_jk) / L_jj.  No blocking, no tiles.
 * A is N x N row-major; the lower triangle is overwritten by L and the strict
 * upper triangle is zeroed.  Returns 0, or the 1-based column of the first
 * non-positive pivot (LAPACK info convention).
 */
int oracle_cholesky(double *A, int N) {
    for (int j = 0; j < N; j++) {
        double *Lj = A + (long)j * N;
        double s = Lj[j];
        for (int k = 0; k < j; k++) s -= Lj[k] * Lj[k];
        if (!(s > 0.0)) return j + 1;
        double ljj = sqrt(s);
        Lj[j] = ljj;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < N; i++) {
            double *Li = A + (long)i * N;
            double t = Li[j];
            for (int k = 0; k < j; k++) t -= Li[k] * Lj[k];
            Li[j] = t / ljj;
        }
    }
    for (int i = 0; i < N; i++)
        for (int j = i + 1; j < N; j++) A[(long)i * N + j] = 0.0;
    return 0;
}

/* Forward substitution L y = z (in place on y); L row-major lower. */
void oracle_forward(const double *L, int N, double *y) {
    for (int i = 0; i < N; i++) {
        double t = y[i];
        const double *Li = L + (long)i * N;
        for (int k = 0; k < i; k++) t -= Li[k] * y[k];
        y[i] = t / Li[i];
    }
}

/* Back substitution L' w = y (in place on w); L row-major lower. */
void oracle_backward(const double *L, int N, double *w) {
    for (int i = N - 1; i >= 0; i--) {
        double t = w[i];
        for (int k = i + 1; k < N; k++) t -= L[(long)k * N + i] * w[k];
        w[i] = t / L[(long)i * N + i];
    }
}

/*
 * Eq. 1 from a factor: with L L' = Sigma and y = L^-1 Z,
 *   log|Sigma| = 2 sum_k log L_kk,   Z' Sigma^-1 Z = y' y,
 *   l = -(N/2) log(2 pi) - 1/2 log|Sigma| - 1/2 y'y,   N = p n.
 * out3 = {l, log|Sigma|, y'y}.
 */
void oracle_loglik_from_factor(const double *L, int N, const double *Z, double *y_out, double *out3) {
    double *y = y_out;
    memcpy(y, Z, sizeof(double) * N);
    oracle_forward(L, N, y);
    double logdet = 0.0, quad = 0.0;
    for (int k = 0; k < N; k++) logdet += 2.0 * log(L[(long)k * N + k]);
    for (int k = 0; k < N; k++) quad += y[k] * y[k];
    out3[0] = -0.5 * (double)N * log(2.0 * M_PI) - 0.5 * logdet - 0.5 * quad;
    out3[1] = logdet;
    out3[2] = quad;
}

/*
 * The whole Eq. 1 evaluation: build Sigma (Eq. 2, Rep. I), factor, solve.
 * work: N*N doubles (receives L), y: N doubles.  Returns the Cholesky info.
 */
int oracle_loglik(int p, const double *sigma2, const double *nu, const double *beta, double a,
                  const double *locs, int n, const double *Z, double *work, double *y, double *out3) {
    int N = p * n;
    oracle_covgen(p, sigma2, nu, beta, a, locs, n, locs, n, work);
    int info = oracle_cholesky(work, N);
    if (info) return info;
    oracle_loglik_from_factor(work, N, Z, y, out3);
    return 0;
}

/*
 * Eq. 3 / Eq. 4: Zhat(s0_l)_i = sum_{r,j} C_ij(|s0_l - s_r|) w_(p r + j),
 * w = Sigma^-1 Z = L'^-1 L^-1 Z.  L is the factor of the observed Sigma
 * (row-major N x N), zhat has p*m entries in Rep. I order.
 */
void oracle_predict(int p, const double *sigma2, const double *nu, const double *beta, double a,
                    const double *L, const double *locs, int n, const double *Z,
                    const double *new_locs, int m, double *zhat) {
    int N = p * n;
    double *w = (double *)malloc(sizeof(double) * N);
    memcpy(w, Z, sizeof(double) * N);
    oracle_forward(L, N, w);
    oracle_backward(L, N, w);
    double *c0 = (double *)malloc(sizeof(double) * (long)p * N);
    for (int l = 0; l < m; l++) {
        /* rows p*l .. p*l+p-1 of Sigma_21, i.e. c0' for this location */
        oracle_covgen(p, sigma2, nu, beta, a, new_locs + 2 * l, 1, locs, n, c0);
        for (int i = 0; i < p; i++) {
            double t = 0.0;
            for (int c = 0; c < N; c++) t += c0[(long)i * N + c] * w[c];
            zhat[p * l + i] = t;
        }
    }
    free(c0);
    free(w);
}

/*
 * y = L e for a lower-triangular L (row-major): the synthetic draw
 * Z ~ N(0, Sigma) from standard normals e (synthetic data of Sec. 6.4.1; the
 * paper does not state the method, read as Z = L e).
 */
void oracle_lower_matvec(const double *L, int N, const double *e, double *out) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; i++) {
        double t = 0.0;
        for (int k = 0; k <= i; k++) t += L[(long)i * N + k] * e[k];
        out[i] = t;
    }
}
