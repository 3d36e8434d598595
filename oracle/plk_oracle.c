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
 * Post-processing of the Table-1 statistics (Sections 3.2, 3.4-3.6):
 *   profile of one beta_j (eq. profilebetai), of sigma (eq. profileSigma), of
 *   lambda (max over the omega points) and of any coordinate of the point
 *   cloud by its upper convex hull; internal parameters omega' (Section 3.2).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - Matern normaliser 2^{1-kappa}/Gamma(kappa) (the printed 2^{kappa-1} makes
 *     rho(0+) != 1); argument u = sqrt(8 kappa) d as printed.
 *   - Rotation matrix taken literally as printed in eq. matern; phi_Y = phi_X / phi_R.
 *   - Box-Cox: lambda == 0 exactly -> log y, otherwise expm1(lambda log y)/lambda.
 *   - Likelihood CI: {theta : l_p(theta) >= max l_p - chi2_1(level)/2}, endpoints
 *     by linear interpolation between bracketing grid points; a side that never
 *     crosses the threshold is censored at the grid edge.
 *   - beta_j profile: (X^T V^-1 X)^-1_[-j,-j] is the inverse of the submatrix
 *     (the GLS fit of the offset model y' - X_j b on X_-j), and the residual
 *     sum of squares is the difference of the two printed quadratic forms.
 *   - sigma profile: the grid is in sigma (not sigma^2); ML form only.
 *   - Hull profile: per distinct x only the largest value counts; points on a
 *     hull edge are not vertices; NaN outside the cloud's x range.
 *   - Internal parameters: a ratio phi_X/phi_Y below one is mapped to the same
 *     correlation with the axes exchanged before the square root is taken.
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
 * beta[K*M*p], logdet[K*2], ssq[K*(M+p)^2] (Table 1 ssqYX), status[K]; any
 * output may be NULL.  Returns the number of threads used. */
int oracle_profile_batch(int64_t n, int32_t p, const double *coords, const double *y,
                         const double *X, int64_t K, const double *params, int32_t M,
                         const double *lambdas, int reml, int nthreads, double *logL,
                         double *sigma2, double *beta, double *logdet, double *ssq,
                         int32_t *status)
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
                                      beta ? beta + k * M * p : NULL, NULL,
                                      ssq ? ssq + k * (M + p) * (M + p) : NULL,
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

/* ------------------------------------------------------------------------ */
/* Post-processing of the Table-1 statistics (Sections 3.4-3.6)               */
/* ------------------------------------------------------------------------ */

/* Inverse of the d x d matrix A (row-major) by Gauss-Jordan elimination with
 * partial pivoting; Ainv receives it.  Returns OR_NOT_PD when a pivot is zero
 * (A singular).  d == 0 is a valid empty matrix. */
static int oracle_invert(int32_t d, const double *A, double *Ainv)
{
    double *T = (double *)malloc(sizeof(double) * (d > 0 ? d * 2 * d : 1));
    if (!T)
        return OR_INVALID;
    for (int32_t r = 0; r < d; ++r)
        for (int32_t c = 0; c < 2 * d; ++c)
            T[r * 2 * d + c] = (c < d) ? A[r * d + c] : (c - d == r ? 1.0 : 0.0);
    for (int32_t c = 0; c < d; ++c) {
        int32_t piv = c;
        for (int32_t r = c + 1; r < d; ++r)
            if (fabs(T[r * 2 * d + c]) > fabs(T[piv * 2 * d + c]))
                piv = r;
        if (T[piv * 2 * d + c] == 0.0) {
            free(T);
            return OR_NOT_PD;
        }
        if (piv != c)
            for (int32_t k = 0; k < 2 * d; ++k) {
                double t = T[c * 2 * d + k];
                T[c * 2 * d + k] = T[piv * 2 * d + k];
                T[piv * 2 * d + k] = t;
            }
        double dv = T[c * 2 * d + c];
        for (int32_t k = 0; k < 2 * d; ++k)
            T[c * 2 * d + k] /= dv;
        for (int32_t r = 0; r < d; ++r) {
            if (r == c)
                continue;
            double f = T[r * 2 * d + c];
            for (int32_t k = 0; k < 2 * d; ++k)
                T[r * 2 * d + k] -= f * T[c * 2 * d + k];
        }
    }
    for (int32_t r = 0; r < d; ++r)
        for (int32_t c = 0; c < d; ++c)
            Ainv[r * d + c] = T[r * 2 * d + d + c];
    free(T);
    return OR_OK;
}

/* Profile log-likelihood of one regression coefficient beta_j (Section 3.4,
 * eq. profilebetai): for each grid value b = grid[g],
 *   prof[g] = max over points k (status 0) and lambdas m of
 *             l(beta_j = b, beta_-j-hat(b), sigma-hat(b), omega_k, lambda_m).
 * With beta_j fixed, X_j b is an offset and beta_-j-hat(b) is the GLS fit of
 * y' - X_j b on X_-j.  The two quadratic forms the section expands,
 *   t1 = (y' - X_j b)^T V^-1 (y' - X_j b)
 *      = y'^T V^-1 y' - 2 b (X^T V^-1 y')_j + b^2 (X^T V^-1 X)_jj,
 *   t2 = (X_-j beta_-j-hat)^T V^-1 (X_-j beta_-j-hat)
 *      = (q_y - b q_x)^T A^-1 (q_y - b q_x),   A = (X^T V^-1 X)_[-j,-j],
 *        q_y = (X^T V^-1 y')_[-j], q_x = (X^T V^-1 X)_[-j,j],
 * are read off ssqYX; their difference is the residual sum of squares
 * RSS(b) (as in Step 3 item 8), sigma-hat^2(b) = RSS(b)/n, and
 *   -2 l = n log sigma-hat^2(b) + log|V| - 2(lambda-1) sum log y + n log(2 pi) + n.
 * A^-1 is the inverse of the submatrix: the GLS normal equations of the
 * offset model involve only the columns X_-j.
 * ssq: K x (M+p) x (M+p) (Table 1 ssqYX, y' columns first); logdet: K x 2
 * ([0] = log|V|); status: K (NULL = all valid; a point counts when
 * (status & 15) == 0).  NaN where no point gives a finite value. */
int oracle_profile_beta_reml(int64_t n, int32_t p, int32_t M, int64_t K, const double *ssq,
                             const double *logdet, const int32_t *status, const double *lambdas,
                             double sumlogy, int32_t j, int64_t G, const double *grid, double *prof,
                             int32_t reml);

int oracle_profile_beta(int64_t n, int32_t p, int32_t M, int64_t K, const double *ssq,
                        const double *logdet, const int32_t *status, const double *lambdas,
                        double sumlogy, int32_t j, int64_t G, const double *grid, double *prof)
{
    return oracle_profile_beta_reml(n, p, M, K, ssq, logdet, status, lambdas, sumlogy, j, G, grid, prof, 0);
}

/* The same profile with the REML criterion when reml != 0 (Appendix,
 * subsection on beta_p with REML, eq. remlprofileytilde): with RSS(b) as above,
 *   -2 l* = (n-p) log(RSS(b)/(n-p)) + log|V| + log|X^T V^-1 X|
 *           - 2(lambda-1) sum log y + n log(2 pi) + n - p,
 * log|X^T V^-1 X| of the full X, as printed (logdet[2k+1]). */
int oracle_profile_beta_reml(int64_t n, int32_t p, int32_t M, int64_t K, const double *ssq,
                             const double *logdet, const int32_t *status, const double *lambdas,
                             double sumlogy, int32_t j, int64_t G, const double *grid, double *prof,
                             int32_t reml)
{
    if (j < 0 || j >= p)
        return OR_INVALID;
    int32_t q = M + p, d = p - 1;
    double *A = (double *)malloc(sizeof(double) * (d > 0 ? d * d : 1));
    double *Ai = (double *)malloc(sizeof(double) * (d > 0 ? d * d : 1));
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (d > 0 ? d : 1));
    if (!A || !Ai || !idx) {
        free(A); free(Ai); free(idx);
        return OR_INVALID;
    }
    for (int64_t g = 0; g < G; ++g)
        prof[g] = NAN;
    for (int32_t a = 0, t = 0; a < p; ++a)
        if (a != j)
            idx[t++] = a;
    for (int64_t k = 0; k < K; ++k) {
        if (status && (status[k] & 15) != 0)
            continue;
        const double *S = ssq + k * q * q;
        double ldv = logdet[2 * k];
        for (int32_t a = 0; a < d; ++a)
            for (int32_t b = 0; b < d; ++b)
                A[a * d + b] = S[(M + idx[a]) * q + (M + idx[b])];
        if (oracle_invert(d, A, Ai) != OR_OK)
            continue;
        for (int32_t m = 0; m < M; ++m) {
            double yy = S[m * q + m];
            double xyj = S[(M + j) * q + m];
            double xxjj = S[(M + j) * q + (M + j)];
            for (int64_t g = 0; g < G; ++g) {
                double b = grid[g];
                double t1 = yy - 2.0 * b * xyj + b * b * xxjj;
                double t2 = 0.0;
                for (int32_t a = 0; a < d; ++a) {
                    double ra = S[(M + idx[a]) * q + m] - b * S[(M + idx[a]) * q + (M + j)];
                    for (int32_t c = 0; c < d; ++c) {
                        double rc = S[(M + idx[c]) * q + m] - b * S[(M + idx[c]) * q + (M + j)];
                        t2 += ra * Ai[a * d + c] * rc;
                    }
                }
                double rss = t1 - t2;
                if (!(rss > 0.0))
                    continue;
                double m2l;
                if (reml) {
                    double ne = (double)(n - p);
                    m2l = ne * log(rss / ne) + ldv + logdet[2 * k + 1]
                        - 2.0 * (lambdas[m] - 1.0) * sumlogy
                        + (double)n * log(2.0 * OR_PI) + ne;
                } else {
                    m2l = (double)n * log(rss / (double)n) + ldv
                        - 2.0 * (lambdas[m] - 1.0) * sumlogy
                        + (double)n * log(2.0 * OR_PI) + (double)n;
                }
                double ll = -0.5 * m2l;
                if (ll == ll && (isnan(prof[g]) || ll > prof[g]))
                    prof[g] = ll;
            }
        }
    }
    free(A); free(Ai); free(idx);
    return OR_OK;
}

/* Profile log-likelihood of sigma (Section 3.5, eq. profileSigma): for each
 * grid value s = sgrid[g] > 0,
 *   prof[g] = max over valid points k and lambdas m of l_p(s, omega_k, lambda_m),
 *   -2 l_p - n log(2 pi) = RSS / s^2 + n log s^2 + log|V| - 2(lambda-1) sum log y,
 * with RSS = (y' - X beta-hat)^T V^-1 (y' - X beta-hat) expanded from ssqYX as
 * y'^T V^-1 y' - 2 beta-hat^T X^T V^-1 y' + beta-hat^T X^T V^-1 X beta-hat and
 * beta-hat = (X^T V^-1 X)^-1 X^T V^-1 y' (eq. betahat).  Arguments as for
 * oracle_profile_beta. */
int oracle_profile_sigma(int64_t n, int32_t p, int32_t M, int64_t K, const double *ssq,
                         const double *logdet, const int32_t *status, const double *lambdas,
                         double sumlogy, int64_t G, const double *sgrid, double *prof)
{
    int32_t q = M + p;
    double *A = (double *)malloc(sizeof(double) * p * p);
    double *Ai = (double *)malloc(sizeof(double) * p * p);
    double *bh = (double *)malloc(sizeof(double) * p);
    if (!A || !Ai || !bh) {
        free(A); free(Ai); free(bh);
        return OR_INVALID;
    }
    for (int64_t g = 0; g < G; ++g)
        prof[g] = NAN;
    for (int64_t k = 0; k < K; ++k) {
        if (status && (status[k] & 15) != 0)
            continue;
        const double *S = ssq + k * q * q;
        double ldv = logdet[2 * k];
        for (int32_t a = 0; a < p; ++a)
            for (int32_t b = 0; b < p; ++b)
                A[a * p + b] = S[(M + a) * q + (M + b)];
        if (oracle_invert(p, A, Ai) != OR_OK)
            continue;
        for (int32_t m = 0; m < M; ++m) {
            for (int32_t a = 0; a < p; ++a) {
                double t = 0.0;
                for (int32_t c = 0; c < p; ++c)
                    t += Ai[a * p + c] * S[(M + c) * q + m];
                bh[a] = t;
            }
            double rss = S[m * q + m];
            for (int32_t a = 0; a < p; ++a) {
                rss -= 2.0 * bh[a] * S[(M + a) * q + m];
                for (int32_t c = 0; c < p; ++c)
                    rss += bh[a] * A[a * p + c] * bh[c];
            }
            if (!(rss > 0.0))
                continue;
            for (int64_t g = 0; g < G; ++g) {
                double s2 = sgrid[g] * sgrid[g];
                double m2l = rss / s2 + (double)n * log(s2) + ldv
                           - 2.0 * (lambdas[m] - 1.0) * sumlogy + (double)n * log(2.0 * OR_PI);
                double ll = -0.5 * m2l;
                if (ll == ll && (isnan(prof[g]) || ll > prof[g]))
                    prof[g] = ll;
            }
        }
    }
    free(A); free(Ai); free(bh);
    return OR_OK;
}

typedef struct { double x, v; int64_t i; } oracle_xv;

static int oracle_xv_cmp(const void *pa, const void *pb)
{
    const oracle_xv *a = (const oracle_xv *)pa, *b = (const oracle_xv *)pb;
    if (a->x != b->x)
        return a->x < b->x ? -1 : 1;
    if (a->v != b->v)
        return a->v > b->v ? -1 : 1;   /* larger value first */
    return (a->i > b->i) - (a->i < b->i);
}

/* 1-D profile from a point cloud by its upper convex hull (Section 3.6): the
 * points (x[k], v[k]) with finite v, sorted by x; per distinct x only the
 * largest v (lowest k among equal values) is kept; the upper hull is built
 * left to right by the monotone chain, dropping a point whenever it does not
 * make a strict right turn (so points on a hull edge are not vertices); the
 * profile is the linear interpolation of the hull vertices.
 *   out[t] = that interpolant at xq[t] (NaN outside [min x, max x] or when no
 *            v is finite);
 *   on_hull[k] = 1 for hull vertices, else 0 (may be NULL).
 * Returns the number of hull vertices (0 if none), or -1 on allocation failure. */
int64_t oracle_profile_hull(int64_t K, const double *x, const double *v, int64_t Q,
                            const double *xq, double *out, int32_t *on_hull)
{
    oracle_xv *P = (oracle_xv *)malloc(sizeof(oracle_xv) * (K > 0 ? K : 1));
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * (K > 0 ? K : 1));
    if (!P || !H) {
        free(P); free(H);
        return -1;
    }
    int64_t np = 0;
    for (int64_t k = 0; k < K; ++k) {
        if (on_hull)
            on_hull[k] = 0;
        if (isfinite(v[k]) && isfinite(x[k])) {
            P[np].x = x[k]; P[np].v = v[k]; P[np].i = k;
            ++np;
        }
    }
    qsort(P, (size_t)np, sizeof(oracle_xv), oracle_xv_cmp);
    int64_t nh = 0;
    for (int64_t t = 0; t < np; ++t) {
        if (t > 0 && P[t].x == P[t - 1].x)
            continue;   /* a lower (or later) point at the same x */
        while (nh >= 2) {
            const oracle_xv *o = &P[H[nh - 2]], *a = &P[H[nh - 1]];
            double cross = (a->x - o->x) * (P[t].v - o->v) - (a->v - o->v) * (P[t].x - o->x);
            if (cross >= 0.0)
                --nh;   /* a lies on or below the segment o -> P[t] */
            else
                break;
        }
        H[nh++] = t;
    }
    if (on_hull)
        for (int64_t h = 0; h < nh; ++h)
            on_hull[P[H[h]].i] = 1;
    for (int64_t t = 0; t < Q; ++t) {
        double xv = xq[t], r = NAN;
        if (nh > 0 && xv >= P[H[0]].x && xv <= P[H[nh - 1]].x) {
            for (int64_t h = 0; h < nh; ++h) {
                const oracle_xv *a = &P[H[h]];
                if (a->x == xv) {
                    r = a->v;
                    break;
                }
                if (h + 1 < nh && xv < P[H[h + 1]].x) {
                    const oracle_xv *b = &P[H[h + 1]];
                    r = a->v + (b->v - a->v) * (xv - a->x) / (b->x - a->x);
                    break;
                }
            }
        }
        out[t] = r;
    }
    free(P); free(H);
    return nh;
}

/* Internal parameters omega' = (gamma_1, kappa~, nu, gamma_2, gamma_3) of a
 * natural parameter row omega = (phi_X, kappa, nu^2, phi_R, phi_A) (Section
 * 3.2, eq. shapeTransform and the range/anisotropy transform):
 *   gamma_1 = log phi_X + log phi_Y, phi_Y = phi_X / phi_R
 *   kappa~  = log kappa (kappa_hat_large == 0) or 1/sqrt(kappa) (otherwise)
 *   nu      = sqrt(nu^2)
 *   gamma_2 = sqrt(phi_X/phi_Y - 1) cos(2 phi_A),  gamma_3 = ... sin(2 phi_A).
 * A ratio below one is first mapped to the same correlation with the axes
 * exchanged, (phi_X, phi_Y, phi_A) -> (phi_Y, phi_X, phi_A + pi/2), so
 * gamma_2, gamma_3 = -sqrt(phi_Y/phi_X - 1) (cos 2 phi_A, sin 2 phi_A). */
void oracle_internal_params(const double *omega, int kappa_hat_large, double *out)
{
    double phx = omega[0], kap = omega[1], nug = omega[2], rat = omega[3], ang = omega[4];
    double phy = phx / rat;
    out[0] = log(phx) + log(phy);
    out[1] = kappa_hat_large ? 1.0 / sqrt(kap) : log(kap);
    out[2] = sqrt(nug);
    double r, sgn;
    if (phx / phy >= 1.0) {
        r = sqrt(phx / phy - 1.0);
        sgn = 1.0;
    } else {
        r = sqrt(phy / phx - 1.0);
        sgn = -1.0;
    }
    out[3] = sgn * r * cos(2.0 * ang);
    out[4] = sgn * r * sin(2.0 * ang);
}

/* Sum of log y_i: the Box-Cox Jacobian's data term (Section 2, eq. 2). */
double oracle_sum_log(int64_t n, const double *y)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i)
        s += log(y[i]);
    return s;
}
