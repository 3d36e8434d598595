/*
 * plk_oracle.c -- plain, slow, FP64 CPU oracle for the profile log-likelihood
 * of the Box-Cox / anisotropic-Matern linear geostatistical model
 * (Xu & Brown, "Profile likelihoods for parameters in trans-Gaussian
 * geostatistical models", arXiv 2305.04318).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header or constant table with
 * the CUDA path.
 *
 * What it computes, in the paper's order (Section 3.3, "Step 3", items 1-8):
 *   1. V = R(omega) + nu^2 I                    (Section 2, eq. 1 and eq. matern)
 *   2. V = L L^T, log|V| = 2 sum log L_jj       (Step 3 item 2; LL^T in place of
 *                                                the paper's LDL^T: same log|V|)
 *   3. W = L^{-1} (y'(lambda_1..lambda_M), X)  (Step 3 item 3)
 *   4. ssqYX = W^T W                           (Step 3 item 4, Table 1)
 *   5. X^T V^-1 X = Q Q^T, log|X^T V^-1 X|     (Step 3 item 5, Table 1 detReml)
 *   6. c = Q^{-1} X^T V^{-1} y'                (Step 3 item 6)
 *   7. ssqBetahat = c^T c                      (Step 3 item 7)
 *   8. ssqResidual = y'^T V^-1 y' - ssqBetahat (Step 3 item 8)
 * and then beta-hat (eq. betahat), sigma-hat^2 (eq. 4) and the profile
 * log-likelihood l_p(omega, lambda) (eq. profile); the REML variant follows
 * eq. remlpro of the Appendix.
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - Matern normaliser 2^{1-kappa}/Gamma(kappa) (the printed 2^{kappa-1} makes
 *     rho(0+) != 1); argument u = sqrt(8 kappa) d as printed.
 *   - Rotation matrix taken literally as printed in eq. matern; phi_Y = phi_X / phi_R.
 *   - Box-Cox: lambda == 0 exactly -> log y, otherwise expm1(lambda log y)/lambda.
 *   - Likelihood CI: {theta : l_p(theta) >= max l_p - chi2_1(level)/2}, endpoints
 *     by linear interpolation between bracketing grid points; a side that never
 *     crosses the threshold is censored at the grid edge.
 *
 * Modified Bessel function K_nu(x) (needed by eq. matern):
 *   x <= 2 : Temme's series for K_mu, K_{mu+1}, |mu| <= 1/2 (N. M. Temme,
 *            J. Comput. Phys. 19 (1975) 324-337), then forward recurrence in the
 *            order, K_{v+1} = K_{v-1} + (2v/x) K_v (DLMF 10.29.1).
 *   x >  2 : the integral K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *            (DLMF 10.32.9) by the trapezoid rule on the scaled integrand
 *            exp(-2 x sinh^2(t/2)) cosh(nu t); the rule converges geometrically
 *            for this analytic integrand, with the step shrunk as 1/sqrt(x) so
 *            the peak of width ~1/sqrt(x) stays resolved.
 *
 * Parity pins (tests): scipy.special.kv over a (nu, x) lattice, closed forms
 * for K_{1/2}, K_{3/2}, the recurrence and the Wronskian; Matern closed forms at
 * kappa = 0.5, 1.5, 2.5 and the kappa -> infinity limit; brute-force dense
 * Gaussian density on n <= 10; GLS beta-hat; invariants (isotropy, rotation,
 * scaling, angle period pi, Box-Cox rescaling); the OLS limit; the CI of an
 * exactly quadratic profile.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_NOT_PD 1
#define OR_INVALID 2
#define OR_RSS_NONPOS 3

static const double OR_PI = 3.14159265358979323846;
static const double OR_LN2 = 0.69314718055994530942;
static const double OR_EULER = 0.57721566490153286061;

/* ------------------------------------------------------------------------ */
/* Bessel K                                                                  */
/* ------------------------------------------------------------------------ */

/* Gamma_1(mu) = (1/Gamma(1-mu) - 1/Gamma(1+mu)) / (2 mu) and
 * Gamma_2(mu) = (1/Gamma(1-mu) + 1/Gamma(1+mu)) / 2 of Temme's series.
 * The difference is formed as rp * expm1(lgamma(1+mu) - lgamma(1-mu)) so that it
 * keeps full relative accuracy as mu -> 0; Gamma_1(0) = -Euler's constant. */
static void temme_gamma12(double mu, double *g1, double *g2, double *rp, double *rm)
{
    double lp = lgamma(1.0 + mu), lm = lgamma(1.0 - mu);
    *rp = exp(-lp);            /* 1/Gamma(1+mu) */
    *rm = exp(-lm);            /* 1/Gamma(1-mu) */
    *g2 = 0.5 * (*rm + *rp);
    if (mu == 0.0)
        *g1 = -OR_EULER;
    else
        *g1 = (*rp) * expm1(lp - lm) / (2.0 * mu);
}

/* Temme's series, 0 < x <= 2, |mu| <= 1/2: returns K_mu(x), K_{mu+1}(x). */
static void bessel_k_temme(double mu, double x, double *kmu, double *kmu1)
{
    double g1, g2, rp, rm;
    temme_gamma12(mu, &g1, &g2, &rp, &rm);
    double l2x = log(2.0 / x);
    double sigma = mu * l2x;
    double a = (mu == 0.0) ? 1.0 : (OR_PI * mu) / sin(OR_PI * mu);
    double b = (sigma == 0.0) ? 1.0 : sinh(sigma) / sigma;
    double f = a * (cosh(sigma) * g1 + b * l2x * g2); /* f_0 */
    double es = exp(sigma);                            /* (x/2)^{-mu} */
    double p = 0.5 * es / rp;                          /* p_0 = (x/2)^{-mu} Gamma(1+mu) / 2 */
    double q = 0.5 / (es * rm);                        /* q_0 = (x/2)^{mu} Gamma(1-mu) / 2 */
    double c = 1.0;                                    /* c_k = (x^2/4)^k / k! */
    double x24 = 0.25 * x * x;
    double s0 = f;                                     /* sum c_k f_k */
    double s1 = p;                                     /* sum c_k h_k, h_0 = p_0 */
    for (int k = 1; k < 1000; ++k) {
        double dk = (double)k;
        f = (dk * f + p + q) / (dk * dk - mu * mu);
        p = p / (dk - mu);
        q = q / (dk + mu);
        c = c * x24 / dk;
        double h = p - dk * f;
        double t0 = c * f, t1 = c * h;
        s0 += t0;
        s1 += t1;
        if (fabs(t0) <= 1e-18 * fabs(s0) && fabs(t1) <= 1e-18 * fabs(s1))
            break;
    }
    *kmu = s0;
    *kmu1 = s1 * 2.0 / x;
}

/* e^x K_nu(x) for x > 2 by the trapezoid rule on
 * int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt. */
static double bessel_k_scaled_integral(double nu, double x)
{
    double h = 0.08;
    double hs = 0.4 / sqrt(x);
    if (hs < h) h = hs;
    double sum = 0.5; /* half weight at t = 0, integrand value 1 */
    double prev = 1.0;
    for (int k = 1; k < 100000; ++k) {
        double t = k * h;
        double sh = sinh(0.5 * t);             /* cosh t - 1 = 2 sinh^2(t/2), no cancellation */
        double g = exp(-2.0 * x * sh * sh) * cosh(nu * t);
        sum += g;
        /* stop once the integrand is decreasing and negligible */
        if (g < prev && g < 1e-19 * sum)
            break;
        prev = g;
    }
    return h * sum;
}

/* K_nu(x), nu >= 0, x > 0. */
double oracle_bessel_k(double nu, double x)
{
    if (!(x > 0.0) || nu < 0.0)
        return NAN;
    if (x > 2.0)
        return exp(-x) * bessel_k_scaled_integral(nu, x);
    int N = (int)floor(nu + 0.5);
    double mu = nu - N;
    double k0, k1;
    bessel_k_temme(mu, x, &k0, &k1); /* K_mu, K_{mu+1}; K_{-v} = K_v */
    if (N == 0)
        return k0;
    /* forward recurrence from orders mu, mu+1 up to mu+N = nu */
    for (int j = 1; j < N; ++j) {
        double k2 = k0 + 2.0 * (mu + j) / x * k1;
        k0 = k1;
        k1 = k2;
    }
    return k1;
}

/* e^x K_nu(x). */
double oracle_bessel_k_scaled(double nu, double x)
{
    if (x > 2.0)
        return bessel_k_scaled_integral(nu, x);
    return exp(x) * oracle_bessel_k(nu, x);
}

/* ------------------------------------------------------------------------ */
/* Matern correlation (eq. matern)                                           */
/* ------------------------------------------------------------------------ */

/* rho(d) = 2^{1-kappa} / Gamma(kappa) * u^kappa K_kappa(u), u = sqrt(8 kappa) d. */
double oracle_matern(double d, double kappa)
{
    if (d == 0.0)
        return 1.0;
    double u = sqrt(8.0 * kappa) * d;
    if (u > 740.0)
        return 0.0;
    /* the product u^kappa K_kappa(u) in log form: stays finite for small u */
    double lognorm = (1.0 - kappa) * OR_LN2 - lgamma(kappa) + kappa * log(u);
    if (u > 2.0)
        return exp(lognorm - u) * oracle_bessel_k_scaled(kappa, u);
    return exp(lognorm) * oracle_bessel_k(kappa, u);
}

/* Anisotropic distance of eq. matern, taken literally:
 *   (a, b) = Rot(phi_A) (h1, h2) with Rot = [[cos, -sin], [sin, cos]],
 *   d = || (a / phi_X, b / phi_Y) ||,  phi_Y = phi_X / phi_R. */
double oracle_aniso_distance(double h1, double h2, double phi_x, double phi_r, double phi_a)
{
    double c = cos(phi_a), s = sin(phi_a);
    double a = c * h1 - s * h2;
    double b = s * h1 + c * h2;
    double phi_y = phi_x / phi_r;
    double ax = a / phi_x, by = b / phi_y;
    return sqrt(ax * ax + by * by);
}

/* V = R + nu^2 I, full n x n row-major (both triangles). omega layout:
 * [phi_X, kappa, nu^2, phi_R, phi_A]. coords n x 2 row-major. */
void oracle_build_v(int64_t n, const double *coords, const double *omega, double *V)
{
    double phi_x = omega[0], kappa = omega[1], nug = omega[2], phi_r = omega[3], phi_a = omega[4];
    for (int64_t i = 0; i < n; ++i) {
        V[i * n + i] = 1.0 + nug;
        for (int64_t j = 0; j < i; ++j) {
            double h1 = coords[2 * i] - coords[2 * j];
            double h2 = coords[2 * i + 1] - coords[2 * j + 1];
            double d = oracle_aniso_distance(h1, h2, phi_x, phi_r, phi_a);
            double r = oracle_matern(d, kappa);
            V[i * n + j] = r;
            V[j * n + i] = r;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Dense linear algebra, unblocked                                           */
/* ------------------------------------------------------------------------ */

/* In-place Cholesky A = L L^T of a row-major n x n matrix (lower triangle is
 * read and overwritten).  Returns OR_NOT_PD on a pivot <= 0 or NaN. */
int oracle_cholesky(int64_t n, double *A)
{
    for (int64_t j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; ++k)
            s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0))
            return OR_NOT_PD;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; ++k)
                t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
    }
    return OR_OK;
}

/* Forward substitution L W = B for ncol right-hand sides; B, W n x ncol row-major. */
void oracle_forward(int64_t n, const double *L, int64_t ncol, const double *B, double *W)
{
    for (int64_t c = 0; c < ncol; ++c) {
        for (int64_t i = 0; i < n; ++i) {
            double t = B[i * ncol + c];
            for (int64_t k = 0; k < i; ++k)
                t -= L[i * n + k] * W[k * ncol + c];
            W[i * ncol + c] = t / L[i * n + i];
        }
    }
}

/* Box-Cox transform b(y; lambda) (Section 2). */
double oracle_boxcox(double y, double lambda)
{
    if (lambda == 0.0)
        return log(y);
    return expm1(lambda * log(y)) / lambda;
}

/* ------------------------------------------------------------------------ */
/* One omega point: Step 3 items 1-8 and the closed form (eq. profile)        */
/* ------------------------------------------------------------------------ */

/* Outputs (any may be NULL):
 *   logL[M]        l_p(omega, lambda_m) (eq. profile; eq. remlpro if reml)
 *   sigma2[M]      sigma-hat^2 (eq. 4; RSS/(n-p) if reml, eq. sigmahat_reml_y)
 *   beta[M*p]      beta-hat (eq. betahat)
 *   rss[M]         ssqResidual (Table 1)
 *   ssq[(M+p)^2]   (y', X)^T V^-1 (y', X) (Table 1 ssqYX), row-major
 *   logdet[2]      log|V| (detVar), log|X^T V^-1 X| (detReml)
 * Returns OR_OK, OR_NOT_PD (V or X^T V^-1 X not positive definite) or
 * OR_RSS_NONPOS; on failure the outputs are NaN. */
int oracle_profile_point(int64_t n, int32_t p, const double *coords, const double *y,
                         const double *X, const double *omega, int32_t M,
                         const double *lambdas, int reml, double *logL, double *sigma2,
                         double *beta, double *rss_out, double *ssq, double *logdet)
{
    int32_t q = M + p;
    int status = OR_OK;
    double *V = (double *)malloc(sizeof(double) * n * n);
    double *Bm = (double *)malloc(sizeof(double) * n * q);
    double *W = (double *)malloc(sizeof(double) * n * q);
    double *S = (double *)malloc(sizeof(double) * q * q);
    double *Q = (double *)malloc(sizeof(double) * p * p);
    double *cvec = (double *)malloc(sizeof(double) * p);
    double *bvec = (double *)malloc(sizeof(double) * p);
    if (!V || !Bm || !W || !S || !Q || !cvec || !bvec) {
        status = OR_INVALID;
        goto fail;
    }
    double sumlogy = 0.0;
    for (int64_t i = 0; i < n; ++i)
        sumlogy += log(y[i]);

    /* Step 3 item 1 */
    oracle_build_v(n, coords, omega, V);
    /* item 2 */
    if (oracle_cholesky(n, V) != OR_OK) {
        status = OR_NOT_PD;
        goto fail;
    }
    double ldv = 0.0;
    for (int64_t j = 0; j < n; ++j)
        ldv += 2.0 * log(V[j * n + j]);
    /* item 3: B = (y'(lambda_1), ..., y'(lambda_M), X) */
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t m = 0; m < M; ++m)
            Bm[i * q + m] = oracle_boxcox(y[i], lambdas[m]);
        for (int32_t k = 0; k < p; ++k)
            Bm[i * q + M + k] = X[i * p + k];
    }
    oracle_forward(n, V, q, Bm, W);
    /* item 4: S = W^T W */
    for (int32_t a = 0; a < q; ++a)
        for (int32_t b = 0; b < q; ++b) {
            double t = 0.0;
            for (int64_t i = 0; i < n; ++i)
                t += W[i * q + a] * W[i * q + b];
            S[a * q + b] = t;
        }
    /* item 5: Q Q^T = X^T V^-1 X */
    for (int32_t a = 0; a < p; ++a)
        for (int32_t b = 0; b < p; ++b)
            Q[a * p + b] = S[(M + a) * q + (M + b)];
    if (oracle_cholesky(p, Q) != OR_OK) {
        status = OR_NOT_PD;
        goto fail;
    }
    double ldx = 0.0;
    for (int32_t j = 0; j < p; ++j)
        ldx += 2.0 * log(Q[j * p + j]);
    if (logdet) {
        logdet[0] = ldv;
        logdet[1] = ldx;
    }
    if (ssq)
        memcpy(ssq, S, sizeof(double) * q * q);
    for (int32_t m = 0; m < M; ++m) {
        /* item 6: c = Q^{-1} X^T V^-1 y' */
        for (int32_t a = 0; a < p; ++a) {
            double t = S[(M + a) * q + m];
            for (int32_t k = 0; k < a; ++k)
                t -= Q[a * p + k] * cvec[k];
            cvec[a] = t / Q[a * p + a];
        }
        /* item 7: ssqBetahat = c^T c */
        double sbh = 0.0;
        for (int32_t a = 0; a < p; ++a)
            sbh += cvec[a] * cvec[a];
        /* item 8 */
        double rss = S[m * q + m] - sbh;
        /* beta-hat = Q^{-T} c (eq. betahat) */
        for (int32_t a = p - 1; a >= 0; --a) {
            double t = cvec[a];
            for (int32_t k = a + 1; k < p; ++k)
                t -= Q[k * p + a] * bvec[k];
            bvec[a] = t / Q[a * p + a];
        }
        double lam = lambdas[m];
        double jac = -2.0 * (lam - 1.0) * sumlogy;
        double m2l;
        double s2;
        if (!reml) {
            s2 = rss / (double)n;
            m2l = (double)n * log(s2) + ldv + jac + (double)n * log(2.0 * OR_PI) + (double)n;
        } else {
            double dof = (double)(n - p);
            s2 = rss / dof;
            m2l = dof * log(s2) + ldv + ldx + jac + (double)n * log(2.0 * OR_PI) + dof;
        }
        if (!(rss > 0.0)) {
            status = OR_RSS_NONPOS;
            m2l = NAN;
        }
        if (logL)
            logL[m] = -0.5 * m2l;
        if (sigma2)
            sigma2[m] = s2;
        if (rss_out)
            rss_out[m] = rss;
        if (beta)
            for (int32_t a = 0; a < p; ++a)
                beta[m * p + a] = bvec[a];
    }
    free(V); free(Bm); free(W); free(S); free(Q); free(cvec); free(bvec);
    return status;
fail:
    if (logL) for (int32_t m = 0; m < M; ++m) logL[m] = NAN;
    if (sigma2) for (int32_t m = 0; m < M; ++m) sigma2[m] = NAN;
    if (rss_out) for (int32_t m = 0; m < M; ++m) rss_out[m] = NAN;
    if (beta) for (int32_t m = 0; m < M * p; ++m) beta[m] = NAN;
    if (ssq) for (int32_t m = 0; m < q * q; ++m) ssq[m] = NAN;
    if (logdet) { logdet[0] = NAN; logdet[1] = NAN; }
    free(V); free(Bm); free(W); free(S); free(Q); free(cvec); free(bvec);
    return status;
}

/* Batch over K omega points (rows of params, K x 5), OpenMP-parallel over the
 * points.  Per-point outputs are laid out point-major: logL[K*M], sigma2[K*M],
 * beta[K*M*p], logdet[K*2], status[K].  Returns the number of threads used. */
int oracle_profile_batch(int64_t n, int32_t p, const double *coords, const double *y,
                         const double *X, int64_t K, const double *params, int32_t M,
                         const double *lambdas, int reml, int nthreads, double *logL,
                         double *sigma2, double *beta, double *logdet, int32_t *status)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads <= 0)
        nthreads = omp_get_max_threads();
    used = nthreads;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t k = 0; k < K; ++k) {
        int st = oracle_profile_point(n, p, coords, y, X, params + 5 * k, M, lambdas, reml,
                                      logL ? logL + k * M : NULL,
                                      sigma2 ? sigma2 + k * M : NULL,
                                      beta ? beta + k * M * p : NULL, NULL, NULL,
                                      logdet ? logdet + 2 * k : NULL);
        if (status)
            status[k] = st;
    }
    return used;
}

/* ------------------------------------------------------------------------ */
/* Profile reduction and likelihood-based CI (Section 3.6, eq. likelihood)    */
/* ------------------------------------------------------------------------ */

/* Upper quantile of chi^2_1: c with P(chi^2_1 <= c) = level, i.e. z^2 where
 * erfc(z / sqrt 2) = 1 - level, found by bisection on libm's erfc. */
double oracle_chi2_1_quantile(double level)
{
    double target = 1.0 - level;
    double lo = 0.0, hi = 40.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (erfc(mid / sqrt(2.0)) > target)
            lo = mid;
        else
            hi = mid;
    }
    double z = 0.5 * (lo + hi);
    return z * z;
}

/* prof[g] = max over the SM values vals[g*SM .. (g+1)*SM) that are not NaN
 * (NaN if none are). */
void oracle_profile_max(int64_t G, int64_t SM, const double *vals, double *prof)
{
    for (int64_t g = 0; g < G; ++g) {
        double best = NAN;
        for (int64_t j = 0; j < SM; ++j) {
            double v = vals[g * SM + j];
            if (isnan(v))
                continue;
            if (isnan(best) || v > best)
                best = v;
        }
        prof[g] = best;
    }
}

/* CI endpoints of a 1-D profile on an ascending grid.  argmax: lowest index
 * among ties (NaNs skipped).  threshold = max - chi2_1(level)/2.  On each side,
 * walk outward from the argmax to the first finite grid point strictly below
 * the threshold and interpolate linearly between it and the finite point just
 * inside it; if no such point exists the endpoint is the grid edge and
 * censored gets bit 1 (lower) or bit 2 (upper).  Returns OR_INVALID if no
 * finite value exists. */
int oracle_profile_ci(const double *grid, const double *prof, int64_t G, double level,
                      double *lo, double *hi, double *argmax, int32_t *censored)
{
    int64_t ib = -1;
    for (int64_t g = 0; g < G; ++g) {
        if (isnan(prof[g]))
            continue;
        if (ib < 0 || prof[g] > prof[ib])
            ib = g;
    }
    if (ib < 0)
        return OR_INVALID;
    double thr = prof[ib] - 0.5 * oracle_chi2_1_quantile(level);
    int32_t cens = 0;
    double l = grid[0], h = grid[G - 1];
    int found = 0;
    int64_t inner = ib; /* last finite point at or above the threshold */
    for (int64_t g = ib - 1; g >= 0; --g) {
        if (isnan(prof[g]))
            continue;
        if (prof[g] < thr) {
            double f = (thr - prof[g]) / (prof[inner] - prof[g]);
            l = grid[g] + f * (grid[inner] - grid[g]);
            found = 1;
            break;
        }
        inner = g;
    }
    if (!found)
        cens |= 1;
    found = 0;
    inner = ib;
    for (int64_t g = ib + 1; g < G; ++g) {
        if (isnan(prof[g]))
            continue;
        if (prof[g] < thr) {
            double f = (thr - prof[g]) / (prof[inner] - prof[g]);
            h = grid[g] + f * (grid[inner] - grid[g]);
            found = 1;
            break;
        }
        inner = g;
    }
    if (!found)
        cens |= 2;
    *lo = l;
    *hi = h;
    *argmax = grid[ib];
    *censored = cens;
    return OR_OK;
}
