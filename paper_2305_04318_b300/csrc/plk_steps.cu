// plk_steps.cu -- Steps 1 and 2 of the method around the evaluation (Xu & Brown,
// arXiv 2305.04318, Sections 3.1-3.2), host code:
//
//   Step 1  maximum-likelihood estimate of (omega, lambda) by a batched Newton
//           iteration in the internal parameters: every iteration evaluates one
//           batch (the Hessian stencil at three lambdas, then a batch of step
//           lengths), so the GPU sees a few hundred points at a time instead of
//           the one-at-a-time calls of a sequential optimiser;
//   Step 2  representative parameter points from the quadratic approximation:
//           the numerical Hessian of l_p(omega', lambda-hat(omega')) from the
//           (2 d^2 + 1) x 3 stencil, eigen-decomposition of -H with the fix-up
//           of negative and near-zero eigenvalues, maximin points on the unit
//           sphere, their images on the chi^2_d contour ellipsoids, the nugget
//           repair, and the lambda grid from the 1-D quadratic approximation.
//
// Both take the likelihood as a callback (plk_eval_fn), so the same code runs
// on the library's own GPU evaluation (plk_fit_mle, plk_quadratic_cloud: jobs
// of a context) and, in tests, on any other evaluator.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "plk.h"
#include "plk_kernels.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr int D5 = 5;

plk_status bad(const char *msg) {
    plk::set_last_error(msg);
    return PLK_E_INVALID;
}

// -------------------------------------------------------------------------
// internal <-> natural parameters (Section 3.2)
// -------------------------------------------------------------------------
// Natural row (phi_X, kappa, nu^2, phi_R, phi_A) -> internal (gamma_1, kappa~,
// nu, gamma_2, gamma_3): gamma_1 = log phi_X + log phi_Y, kappa~ = log kappa or
// 1/sqrt(kappa), nu = sqrt(nu^2), (gamma_2, gamma_3) = sqrt(phi_X/phi_Y - 1)
// (cos 2 phi_A, sin 2 phi_A); a ratio below one is the same correlation with
// the axes exchanged.
void to_internal(const double *w, bool kappa_large, double *o) {
    const double phx = w[0], kap = w[1], nug = w[2], rat = w[3], ang = w[4];
    const double phy = phx / rat;
    o[0] = std::log(phx) + std::log(phy);
    o[1] = kappa_large ? 1.0 / std::sqrt(kap) : std::log(kap);
    o[2] = std::sqrt(nug);
    const double r = rat >= 1.0 ? std::sqrt(rat - 1.0) : -std::sqrt(1.0 / rat - 1.0);
    o[3] = r * std::cos(2.0 * ang);
    o[4] = r * std::sin(2.0 * ang);
}

// Inverse: phi_X phi_Y = exp(gamma_1), phi_X / phi_Y = 1 + gamma_2^2 + gamma_3^2,
// phi_A = atan2(gamma_3, gamma_2) / 2 in [0, pi); kappa = exp(kappa~) or
// 1/kappa~^2; nu^2 = nu^2 (the sign of nu is handled by the caller).
void to_natural(const double *v, bool kappa_large, double *w) {
    const double r2 = v[3] * v[3] + v[4] * v[4];
    const double rat = 1.0 + r2;
    w[0] = std::exp(0.5 * v[0]) * std::sqrt(rat);
    w[1] = kappa_large ? 1.0 / (v[1] * v[1]) : std::exp(v[1]);
    w[2] = v[2] * v[2];
    w[3] = rat;
    double a = r2 > 0.0 ? 0.5 * std::atan2(v[4], v[3]) : 0.0;
    if (a < 0.0) a += PI;
    w[4] = a;
}

// -------------------------------------------------------------------------
// chi^2_d quantiles: the regularised lower incomplete gamma function P(a, x)
// by its power series (x < a + 1) or the continued fraction of Q = 1 - P
// (modified Lentz), then bisection in x.
// -------------------------------------------------------------------------
double gamma_p(double a, double x) {
    if (x <= 0.0) return 0.0;
    const double lg = std::lgamma(a);
    if (x < a + 1.0) {
        double term = 1.0 / a, sum = term, ap = a;
        for (int k = 0; k < 1000; ++k) {
            ap += 1.0;
            term *= x / ap;
            sum += term;
            if (std::fabs(term) < 1e-17 * std::fabs(sum)) break;
        }
        return sum * std::exp(-x + a * std::log(x) - lg);
    }
    const double tiny = 1e-300;
    double b = x + 1.0 - a, c = 1.0 / tiny, d = 1.0 / b, h = d;
    for (int i = 1; i < 1000; ++i) {
        const double an = -i * (i - a);
        b += 2.0;
        d = an * d + b;
        if (std::fabs(d) < tiny) d = tiny;
        c = b + an / c;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0 / d;
        const double del = d * c;
        h *= del;
        if (std::fabs(del - 1.0) < 1e-16) break;
    }
    return 1.0 - std::exp(-x + a * std::log(x) - lg) * h;
}

double chi2_quantile(int dof, double p) {
    double lo = 0.0, hi = 1.0;
    while (gamma_p(0.5 * dof, 0.5 * hi) < p && hi < 1e6) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (gamma_p(0.5 * dof, 0.5 * mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

// -------------------------------------------------------------------------
// symmetric eigen-decomposition (cyclic Jacobi), d <= 5:  A = E diag(D) E^T,
// E's columns the eigenvectors
// -------------------------------------------------------------------------
void jacobi_eigen(int d, const double *Ain, double *D, double *E) {
    double A[D5 * D5];
    std::memcpy(A, Ain, sizeof(double) * d * d);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) E[i * d + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                tot += A[i * d + j] * A[i * d + j];
                if (i != j) off += A[i * d + j] * A[i * d + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                const double apq = A[p * d + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * d + q] - A[p * d + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < d; ++k) {   // A <- J^T A J on columns p, q
                    const double akp = A[k * d + p], akq = A[k * d + q];
                    A[k * d + p] = c * akp - s * akq;
                    A[k * d + q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {   // rows p, q
                    const double apk = A[p * d + k], aqk = A[q * d + k];
                    A[p * d + k] = c * apk - s * aqk;
                    A[q * d + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) {
                    const double ekp = E[k * d + p], ekq = E[k * d + q];
                    E[k * d + p] = c * ekp - s * ekq;
                    E[k * d + q] = s * ekp + c * ekq;
                }
            }
    }
    for (int i = 0; i < d; ++i) D[i] = A[i * d + i];
}

// Eigen fix-up of -H (Section 3.2): negative eigenvalues by their absolute
// values; when the largest exceeds 100, eigenvalues below 0.1 ("close to 0")
// become 0.1; a numerically zero (below 1e-8 max(1, largest)) or non-finite
// eigenvalue becomes 0.1 in any case (its axis would otherwise be unbounded).
void fix_eigenvalues(int d, double *D) {
    double mx = 0.0;
    for (int i = 0; i < d; ++i) {
        D[i] = std::fabs(D[i]);
        if (std::isfinite(D[i])) mx = std::max(mx, D[i]);
    }
    for (int i = 0; i < d; ++i) {
        if (!std::isfinite(D[i]) || D[i] <= 1e-8 * std::max(1.0, mx)) D[i] = 0.1;
        else if (mx > 100.0 && D[i] < 0.1) D[i] = 0.1;
    }
}

// -------------------------------------------------------------------------
// Hessian stencil in the free internal coordinates (d = 5: all; d = 4: kappa~
// held fixed): the centre, +-delta e_i, and the four corners +-delta e_i
// +-delta e_j of every pair i < j: 2 d^2 + 1 points (51 for d = 5, 33 for 4).
// -------------------------------------------------------------------------
int free_coords(bool kappa_fixed, int *idx) {
    int d = 0;
    for (int k = 0; k < D5; ++k)
        if (!(kappa_fixed && k == 1)) idx[d++] = k;
    return d;
}

int stencil(const double *center, int d, const int *idx, double delta, std::vector<double> &pts) {
    const int S = 2 * d * d + 1;
    pts.assign((size_t)S * D5, 0.0);
    for (int s = 0; s < S; ++s) std::memcpy(&pts[(size_t)s * D5], center, sizeof(double) * D5);
    int s = 1;
    for (int i = 0; i < d; ++i) {
        pts[(size_t)s++ * D5 + idx[i]] += delta;
        pts[(size_t)s++ * D5 + idx[i]] -= delta;
    }
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            for (int c = 0; c < 4; ++c) {
                pts[(size_t)s * D5 + idx[i]] += (c < 2 ? delta : -delta);
                pts[(size_t)s * D5 + idx[j]] += (c % 2 == 0 ? delta : -delta);
                ++s;
            }
    return S;
}

// Maximum over lambda of the parabola through (lambda0 - dl, f_m), (lambda0, f_0),
// (lambda0 + dl, f_p), for the offset t = (lambda - lambda0)/dl in [-tmax, tmax]
// (the three values themselves when the parabola is not concave).  NaN if any
// value is NaN.
double lambda_profile(double fm, double f0, double fp, double tmax, double *t_out) {
    if (!(std::isfinite(fm) && std::isfinite(f0) && std::isfinite(fp))) {
        if (t_out) *t_out = 0.0;
        return NAN;
    }
    const double b = 0.5 * (fp - fm), c = 0.5 * (fp + fm - 2.0 * f0);
    double t = 0.0, v = f0;
    if (c < 0.0) {
        t = std::max(-tmax, std::min(tmax, -b / (2.0 * c)));
        v = f0 + b * t + c * t * t;
    }
    if (fm > v) { v = fm; t = -1.0; }   // (only when the parabola is not concave)
    if (fp > v) { v = fp; t = 1.0; }
    if (t_out) *t_out = t;
    return v;
}

// H, g of L(omega') = max_lambda l_p from the stencil's profiled values L[s].
void hessian_from_values(int d, double delta, const double *L, double *H, double *g) {
    int s = 1;
    std::vector<double> Lp(d), Lm(d);
    for (int i = 0; i < d; ++i) {
        Lp[i] = L[s++];
        Lm[i] = L[s++];
    }
    for (int i = 0; i < d; ++i) {
        H[i * d + i] = (Lp[i] - 2.0 * L[0] + Lm[i]) / (delta * delta);
        g[i] = (Lp[i] - Lm[i]) / (2.0 * delta);
    }
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j) {
            const double pp = L[s], pm = L[s + 1], mp = L[s + 2], mm = L[s + 3];
            s += 4;
            H[i * d + j] = H[j * d + i] = (pp - pm - mp + mm) / (4.0 * delta * delta);
        }
}

// -------------------------------------------------------------------------
// maximin points on the unit sphere S^{d-1}: a stochastic optimiser of
// min_{i != j} ||x_i - x_j||.  From seeded Gaussian directions, every round
// moves each point (in a random order) away from its nearest neighbour by a
// shrinking step plus a small random jitter and re-projects it onto the
// sphere; the configuration with the largest minimum distance is kept.
// -------------------------------------------------------------------------
struct Rng {   // splitmix64
    uint64_t s;
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }   // [0, 1)
    double normal() {
        double u = uniform(), v = uniform();
        if (u <= 0.0) u = 1e-300;
        return std::sqrt(-2.0 * std::log(u)) * std::cos(2.0 * PI * v);
    }
};

double min_pair_distance(int n, int d, const std::vector<double> &x) {
    double best = INFINITY;
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < d; ++k) {
                const double t = x[(size_t)i * d + k] - x[(size_t)j * d + k];
                s += t * t;
            }
            best = std::min(best, s);
        }
    return std::sqrt(best);
}

void normalise(double *v, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += v[k] * v[k];
    s = std::sqrt(s);
    for (int k = 0; k < d; ++k) v[k] /= s;
}

double sphere_points(int d, int n, uint64_t seed, int rounds, std::vector<double> &x) {
    Rng rng{seed};
    x.assign((size_t)n * d, 0.0);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < d; ++k) x[(size_t)i * d + k] = rng.normal();
        normalise(&x[(size_t)i * d], d);
    }
    if (n < 2) return INFINITY;
    std::vector<double> best = x;
    double best_min = min_pair_distance(n, d, x);
    // typical spacing of n points on S^{d-1}: area^(1/(d-1)) / n^(1/(d-1))
    const double spacing = 2.0 * std::pow((double)n, -1.0 / (d - 1));
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    for (int r = 0; r < rounds; ++r) {
        const double step = 0.5 * spacing * (1.0 - (double)r / rounds) + 1e-4 * spacing;
        for (int i = n - 1; i > 0; --i) std::swap(order[i], order[rng.next() % (uint64_t)(i + 1)]);
        for (int oi = 0; oi < n; ++oi) {
            const int i = order[oi];
            double *xi = &x[(size_t)i * d];
            int nn = -1;
            double nd = INFINITY;
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double t = xi[k] - x[(size_t)j * d + k];
                    s += t * t;
                }
                if (s < nd) { nd = s; nn = j; }
            }
            nd = std::sqrt(nd);
            const double *xj = &x[(size_t)nn * d];
            for (int k = 0; k < d; ++k)
                xi[k] += step * ((xi[k] - xj[k]) / std::max(nd, 1e-12) + 0.1 * rng.normal());
            normalise(xi, d);
        }
        const double m = min_pair_distance(n, d, x);
        if (m > best_min) {
            best_min = m;
            best = x;
        }
    }
    x = best;
    return best_min;
}

// -------------------------------------------------------------------------
// evaluation through a callback
// -------------------------------------------------------------------------
struct Evaluator {
    plk_eval_fn fn;
    void *user;
    int64_t calls = 0, points = 0;
    // internal rows -> natural rows -> l_p at the M lambdas (K x M)
    plk_status run(const std::vector<double> &nat, int64_t K, const double *lam, int M, std::vector<double> &out) {
        out.assign((size_t)K * M, NAN);
        ++calls;
        points += K;
        const int32_t r = fn(user, nat.data(), K, lam, M, out.data());
        if (r != 0) {
            plk::set_last_error("likelihood evaluation callback failed");
            return (plk_status)(r > 0 && r <= PLK_E_CANCELLED ? r : PLK_E_CUDA);
        }
        return PLK_OK;
    }
};

void natural_rows(const std::vector<double> &internal, int64_t K, bool kappa_large, std::vector<double> &nat) {
    nat.resize((size_t)K * D5);
    for (int64_t k = 0; k < K; ++k) to_natural(&internal[(size_t)k * D5], kappa_large, &nat[(size_t)k * D5]);
}

// Stencil around `center` (internal) at lambda0 +- dl: profiled values L[s],
// their lambda offsets T[s], and the raw centre values (fm, f0, fp).
plk_status eval_stencil(Evaluator &ev, const double *center, int d, const int *idx, double delta, bool kappa_large,
                        double lambda0, double dl, double tmax, std::vector<double> &L, std::vector<double> &T,
                        double *f3) {
    std::vector<double> pts, nat, out;
    const int S = stencil(center, d, idx, delta, pts);
    natural_rows(pts, S, kappa_large, nat);
    const double lam[3] = {lambda0 - dl, lambda0, lambda0 + dl};
    plk_status st = ev.run(nat, S, lam, 3, out);
    if (st != PLK_OK) return st;
    L.resize(S);
    T.resize(S);
    for (int s = 0; s < S; ++s) L[s] = lambda_profile(out[3 * s], out[3 * s + 1], out[3 * s + 2], tmax, &T[s]);
    if (f3) {
        f3[0] = out[0];
        f3[1] = out[1];
        f3[2] = out[2];
    }
    return PLK_OK;
}

bool kappa_is_large(double kappa) { return kappa >= 4.0; }

// The fit keeps kappa within [0.1, 20] (the widest range of shapes the method
// explores: its constrained fits hold kappa between 0.5 and 20): towards
// larger kappa the correlation approaches its Gaussian limit, the likelihood
// flattens into a ridge, and the integral behind the rho table loses accuracy
// (its trapezoid error grows like 2^kappa).
constexpr double KAPPA_MIN = 0.1, KAPPA_MAX = 20.0;
bool kappa_in_range(const double *internal, bool kappa_large) {
    const double k = kappa_large ? 1.0 / (internal[1] * internal[1]) : std::exp(internal[1]);
    return k >= KAPPA_MIN * (1.0 - 1e-12) && k <= KAPPA_MAX * (1.0 + 1e-12);
}
// Projection of kappa~ onto that range.
void clamp_kappa(double *internal, bool kappa_large) {
    if (kappa_large) {
        const double lo = 1.0 / std::sqrt(KAPPA_MAX), hi = 1.0 / std::sqrt(KAPPA_MIN);
        internal[1] = std::max(lo, std::min(hi, std::fabs(internal[1])));
    } else {
        internal[1] = std::max(std::log(KAPPA_MIN), std::min(std::log(KAPPA_MAX), internal[1]));
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// building blocks (host)
// ---------------------------------------------------------------------------
extern "C" plk_status plk_natural_params(const double *internal, int64_t K, int32_t kappa_hat_large, double *out) {
    if ((K > 0 && (!internal || !out)) || K < 0) return bad("plk_natural_params: bad arguments");
    for (int64_t k = 0; k < K; ++k) to_natural(internal + D5 * k, kappa_hat_large != 0, out + D5 * k);
    return PLK_OK;
}

extern "C" double plk_chi2_quantile(int32_t dof, double p) {
    if (dof < 1 || !(p > 0.0) || !(p < 1.0)) return NAN;
    return chi2_quantile(dof, p);
}

extern "C" plk_status plk_hessian_stencil(const double *center_internal, int32_t kappa_fixed, double delta,
                                          double *out, int32_t *S_out) {
    if (!center_internal || !out || !(delta > 0.0)) return bad("plk_hessian_stencil: bad arguments");
    int idx[D5];
    const int d = free_coords(kappa_fixed != 0, idx);
    std::vector<double> pts;
    const int S = stencil(center_internal, d, idx, delta, pts);
    std::memcpy(out, pts.data(), sizeof(double) * pts.size());
    if (S_out) *S_out = S;
    return PLK_OK;
}

extern "C" plk_status plk_hessian_from_stencil(int32_t kappa_fixed, double delta, const double *logL3,
                                               double tmax, double *H, double *grad, double *L_profiled,
                                               double *t_lambda) {
    if (!logL3 || !H || !grad || !(delta > 0.0) || !(tmax > 0.0)) return bad("plk_hessian_from_stencil: bad arguments");
    int idx[D5];
    const int d = free_coords(kappa_fixed != 0, idx);
    const int S = 2 * d * d + 1;
    std::vector<double> L(S), T(S);
    for (int s = 0; s < S; ++s) L[s] = lambda_profile(logL3[3 * s], logL3[3 * s + 1], logL3[3 * s + 2], tmax, &T[s]);
    hessian_from_values(d, delta, L.data(), H, grad);
    if (L_profiled) std::memcpy(L_profiled, L.data(), sizeof(double) * S);
    if (t_lambda) std::memcpy(t_lambda, T.data(), sizeof(double) * S);
    return PLK_OK;
}

extern "C" plk_status plk_fix_hessian(int32_t d, const double *H, double *E, double *D) {
    if (d < 1 || d > D5 || !H || !E || !D) return bad("plk_fix_hessian: bad arguments");
    double A[D5 * D5];
    for (int i = 0; i < d * d; ++i) A[i] = -H[i];
    jacobi_eigen(d, A, D, E);
    fix_eigenvalues(d, D);
    return PLK_OK;
}

extern "C" plk_status plk_sphere_points(int32_t d, int32_t n, uint64_t seed, int32_t rounds, double *x,
                                        double *min_distance) {
    if (d < 2 || d > 16 || n < 1 || rounds < 0 || !x) return bad("plk_sphere_points: bad arguments");
    std::vector<double> v;
    const double m = sphere_points(d, n, seed, rounds, v);
    std::memcpy(x, v.data(), sizeof(double) * v.size());
    if (min_distance) *min_distance = m;
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// Step 1: batched Newton iteration
// ---------------------------------------------------------------------------
extern "C" plk_status plk_fit_mle_cb(plk_eval_fn fn, void *user, const double *omega0, double lambda0,
                                     const plk_fit_options *opts, double *omega_hat, double *lambda_hat,
                                     double *logL_hat, int32_t *iterations) {
    if (!fn || !omega0 || !omega_hat || !lambda_hat) return bad("plk_fit_mle: NULL argument");
    plk_fit_options o{};
    o.delta = 0.05;
    o.delta_lambda = 0.05;
    o.max_iter = 60;
    o.tol = 1e-7;
    if (opts) {
        o = *opts;
        if (!(o.delta > 0.0)) o.delta = 0.05;
        if (!(o.delta_lambda > 0.0)) o.delta_lambda = 0.05;
        if (o.max_iter <= 0) o.max_iter = 60;
        if (!(o.tol > 0.0)) o.tol = 1e-7;
    }
    for (int k = 0; k < D5; ++k)
        if (!std::isfinite(omega0[k])) return bad("plk_fit_mle: non-finite start");
    if (!(omega0[0] > 0 && omega0[1] > 0 && omega0[2] >= 0 && omega0[3] > 0) || !std::isfinite(lambda0))
        return bad("plk_fit_mle: start outside the parameter domain");
    if (o.kappa_fixed && !(o.kappa > 0.0)) return bad("plk_fit_mle: kappa_fixed needs kappa > 0");
    Evaluator ev{fn, user};
    double w0[D5];
    std::memcpy(w0, omega0, sizeof w0);
    if (o.kappa_fixed) w0[1] = o.kappa;
    const bool klarge = o.kappa_fixed ? kappa_is_large(o.kappa) : kappa_is_large(w0[1]);
    double c[D5];
    to_internal(w0, klarge, c);
    if (!o.kappa_fixed) clamp_kappa(c, klarge);
    int idx[D5];
    const int d = free_coords(o.kappa_fixed != 0, idx);
    double lam = lambda0, cur = NAN;
    // finite-difference steps: shrunk by 4 (down to 1/16 of the initial ones)
    // whenever an iteration gains nothing, since the central differences' O(delta^2)
    // error then dominates the remaining gradient
    double delta = o.delta, dl = o.delta_lambda;
    const double delta_min = o.delta / 16.0 * (1.0 + 1e-9);
    const double trust = 1.0;
    const double alphas[] = {1.0, 0.5, 0.25, 0.125, 1.0 / 16, 0.0};
    const int NA = sizeof(alphas) / sizeof(alphas[0]);
    int it = 0;
    bool evaluated = false;   // cur is an evaluated l_p at (c, lam)
    for (; it < o.max_iter; ++it) {
        // the stencil at (c, lam): Hessian and gradient of the lambda-profiled
        // likelihood, and l_p at the current iterate itself (its centre value)
        std::vector<double> L, T;
        double f3[3];
        plk_status st = eval_stencil(ev, c, d, idx, delta, klarge, lam, dl, 1.0, L, T, f3);
        if (st != PLK_OK) return st;
        const int S = (int)L.size();
        cur = f3[1];
        evaluated = true;
        if (!std::isfinite(cur)) {
            plk::set_last_error("plk_fit_mle: the likelihood is not finite at the current point");
            return PLK_E_INVALID;
        }
        bool stencil_ok = true;
        for (int s = 0; s < S; ++s) stencil_ok = stencil_ok && std::isfinite(L[s]);
        // Newton direction from -H with its eigenvalues made positive (a
        // descent direction of -L whatever the curvature), capped to a trust radius
        double step[D5] = {0, 0, 0, 0, 0};
        if (stencil_ok) {
            double H[D5 * D5], g[D5];
            hessian_from_values(d, delta, L.data(), H, g);
            // active set: kappa~ at a bound of its range with the gradient
            // pointing outward is held (the step is solved in the others)
            int act[D5], na = 0;
            for (int i = 0; i < d; ++i) {
                if (idx[i] == 1 && !o.kappa_fixed) {
                    double probe[D5];
                    std::memcpy(probe, c, sizeof probe);
                    probe[1] += (g[i] > 0 ? 1e-9 : -1e-9) * std::max(1.0, std::fabs(c[1]));
                    if (!kappa_in_range(probe, klarge)) continue;
                }
                act[na++] = i;
            }
            double A[D5 * D5], E[D5 * D5], Dv[D5];
            for (int i = 0; i < na; ++i)
                for (int j = 0; j < na; ++j) A[i * na + j] = -H[act[i] * d + act[j]];
            jacobi_eigen(na, A, Dv, E);
            for (int i = 0; i < na; ++i) Dv[i] = std::max(std::fabs(Dv[i]), 1e-3);
            double nrm = 0.0;
            for (int i = 0; i < na; ++i) {
                double s2 = 0.0;
                for (int k = 0; k < na; ++k)
                    for (int m = 0; m < na; ++m) s2 += E[i * na + k] * E[m * na + k] / Dv[k] * g[act[m]];
                step[act[i]] = s2;
                nrm += s2 * s2;
            }
            nrm = std::sqrt(nrm);
            if (nrm > trust)
                for (int i = 0; i < d; ++i) step[i] *= trust / nrm;
        }
        // lambda step: vertex of the centre's parabola (up to 5 steps of dl away)
        double tc = 0.0;
        {
            const double bb = 0.5 * (f3[2] - f3[0]), cc = 0.5 * (f3[2] + f3[0] - 2.0 * f3[1]);
            tc = cc < 0.0 ? std::max(-5.0, std::min(5.0, -bb / (2.0 * cc))) : (f3[2] >= f3[0] ? 1.0 : -1.0);
        }
        const double lam_c = lam + tc * dl;
        // one batch: the Newton step at several lengths (and none) at lam_c +- dl
        std::vector<double> cand((size_t)NA * D5), nat, out;
        for (int a2 = 0; a2 < NA; ++a2) {
            std::memcpy(&cand[(size_t)a2 * D5], c, sizeof c);
            for (int i = 0; i < d; ++i) cand[(size_t)a2 * D5 + idx[i]] += alphas[a2] * step[i];
            if (!o.kappa_fixed) clamp_kappa(&cand[(size_t)a2 * D5], klarge);
        }
        natural_rows(cand, NA, klarge, nat);
        const double l3[3] = {lam_c - dl, lam_c, lam_c + dl};
        if ((st = ev.run(nat, NA, l3, 3, out)) != PLK_OK) return st;
        // the best of those and of the stencil points (each at its profiled lambda)
        double bestL = cur, best_lam = lam, bc[D5];
        std::memcpy(bc, c, sizeof bc);
        for (int a2 = 0; a2 < NA; ++a2) {
            double t;
            const double v = lambda_profile(out[3 * a2], out[3 * a2 + 1], out[3 * a2 + 2], 1.0, &t);
            if (std::isfinite(v) && v > bestL && kappa_in_range(&cand[(size_t)a2 * D5], klarge)) {
                bestL = v;
                best_lam = lam_c + t * dl;
                std::memcpy(bc, &cand[(size_t)a2 * D5], sizeof bc);
            }
        }
        std::vector<double> pts;
        stencil(c, d, idx, delta, pts);
        for (int s = 0; s < S; ++s)
            if (std::isfinite(L[s]) && L[s] > bestL && kappa_in_range(&pts[(size_t)s * D5], klarge)) {
                bestL = L[s];
                best_lam = lam + T[s] * dl;
                std::memcpy(bc, &pts[(size_t)s * D5], sizeof bc);
            }
        if (bestL - cur < o.tol) {
            if (delta > delta_min) {   // (c, lam) stays; retry with finer differences
                delta *= 0.25;
                dl *= 0.25;
                continue;
            }
            ++it;
            break;   // (c, lam) stays: cur is its evaluated value
        }
        std::memcpy(c, bc, sizeof c);
        lam = best_lam;
        evaluated = false;
    }
    if (!evaluated) {   // stopped by max_iter after a move: evaluate the final point
        std::vector<double> nat, out;
        std::vector<double> cv(c, c + D5);
        natural_rows(cv, 1, klarge, nat);
        plk_status st = ev.run(nat, 1, &lam, 1, out);
        if (st != PLK_OK) return st;
        cur = out[0];
    }
    const double Lc = cur;
    double w[D5];
    to_natural(c, klarge, w);
    if (o.kappa_fixed) w[1] = o.kappa;
    std::memcpy(omega_hat, w, sizeof w);
    *lambda_hat = lam;
    if (logL_hat) *logL_hat = Lc;
    if (iterations) *iterations = it;
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// Step 2: representative points
// ---------------------------------------------------------------------------
extern "C" plk_status plk_quadratic_cloud_cb(plk_eval_fn fn, void *user, const double *omega_hat, double lambda_hat,
                                             const plk_cloud_options *opts, double *params_out, int64_t capacity,
                                             int64_t *K_out, double *lambdas_out, double *hessian_out,
                                             double *eig_out) {
    if (!fn || !omega_hat || !K_out) return bad("plk_quadratic_cloud: NULL argument");
    plk_cloud_options o{};
    if (opts) o = *opts;
    if (!(o.delta > 0.0)) o.delta = 0.05;
    if (!(o.delta_lambda > 0.0)) o.delta_lambda = 0.05;
    if (o.n_sphere <= 0) o.n_sphere = o.kappa_fixed ? 120 : 726;
    if (o.n_lambda < 0) return bad("plk_quadratic_cloud: n_lambda < 0");
    if (o.sphere_rounds <= 0) o.sphere_rounds = 200;
    static const double kDefaultProbs[] = {0.05, 0.15, 0.25, 0.35, 0.45, 0.55, 0.65, 0.75, 0.85, 0.95, 0.99};
    const double *probs = o.level_probs ? o.level_probs : kDefaultProbs;
    const int nlev = o.level_probs ? o.n_levels : (int)(sizeof(kDefaultProbs) / sizeof(double));
    if (nlev < 1) return bad("plk_quadratic_cloud: no contour level");
    for (int l = 0; l < nlev; ++l)
        if (!(probs[l] > 0.0 && probs[l] < 1.0)) return bad("plk_quadratic_cloud: level probabilities in (0, 1)");
    int idx[D5];
    const int d = free_coords(o.kappa_fixed != 0, idx);
    const int64_t K = (int64_t)nlev * o.n_sphere;
    *K_out = K;
    if (!params_out || capacity < K) {   // size query
        if (!params_out) return PLK_OK;
        plk::set_last_error("plk_quadratic_cloud: params_out capacity below levels x points per level");
        return PLK_E_NOMEM;
    }
    const bool klarge = kappa_is_large(omega_hat[1]);
    double c[D5];
    to_internal(omega_hat, klarge, c);
    Evaluator ev{fn, user};
    std::vector<double> L, T;
    double f3[3];
    // a stencil point where V is not positive definite (typically nu^2 near 0
    // with a smooth, long-range correlation): retry with steps of 1/4, twice
    double delta = o.delta, dl = o.delta_lambda;
    bool finite = false;
    for (int attempt = 0; attempt < 3 && !finite; ++attempt) {
        if (attempt) {
            delta *= 0.25;
            dl *= 0.25;
        }
        plk_status st = eval_stencil(ev, c, d, idx, delta, klarge, lambda_hat, dl, 1.0, L, T, f3);
        if (st != PLK_OK) return st;
        finite = true;
        for (double v : L) finite = finite && std::isfinite(v);
    }
    if (!finite) {
        plk::set_last_error("plk_quadratic_cloud: the likelihood is not finite on the Hessian stencil");
        return PLK_E_INVALID;
    }
    double H[D5 * D5], g[D5], E[D5 * D5], Dv[D5];
    hessian_from_values(d, delta, L.data(), H, g);
    if (hessian_out) std::memcpy(hessian_out, H, sizeof(double) * d * d);
    double A[D5 * D5];
    for (int i = 0; i < d * d; ++i) A[i] = -H[i];
    jacobi_eigen(d, A, Dv, E);
    fix_eigenvalues(d, Dv);
    if (eig_out) std::memcpy(eig_out, Dv, sizeof(double) * d);
    // lambda grid: n_lambda values evenly between the 0.01 and 0.99 quantiles of
    // N(lambda-hat, 1 / (-d^2 l / d lambda^2)) at the centre
    if (lambdas_out && o.n_lambda > 0) {
        const double curv = (f3[0] + f3[2] - 2.0 * f3[1]) / (dl * dl);
        const double sd = curv < 0.0 ? 1.0 / std::sqrt(-curv) : 0.5;
        const double z = std::sqrt(chi2_quantile(1, 0.98));   // Phi^-1(0.99)
        for (int m = 0; m < o.n_lambda; ++m)
            lambdas_out[m] = o.n_lambda > 1 ? lambda_hat - z * sd + 2.0 * z * sd * m / (o.n_lambda - 1) : lambda_hat;
    }
    // points: x' = omega'-hat + sqrt(c_l) E D^{-1/2} E^T x on each contour level
    // (the symmetric inverse square root of -H~: independent of the order and
    // signs of the eigenvectors, and mapping the unit sphere onto the ellipsoid
    // (x' - omega'-hat)^T (-H~) (x' - omega'-hat) = c_l)
    std::vector<double> x;
    sphere_points(d, o.n_sphere, o.seed, o.sphere_rounds, x);
    Rng rng{o.seed ^ 0x5bd1e995ull};
    int64_t neg = 0;
    for (int l = 0; l < nlev; ++l) {
        const double rc = std::sqrt(chi2_quantile(d, probs[l]));
        for (int i = 0; i < o.n_sphere; ++i) {
            double v[D5];
            std::memcpy(v, c, sizeof v);
            for (int a = 0; a < d; ++a) {   // (E D^{-1/2} E^T x)_a
                double s = 0.0;
                for (int k = 0; k < d; ++k) {
                    double ex = 0.0;
                    for (int m = 0; m < d; ++m) ex += E[m * d + k] * x[(size_t)i * d + m];
                    s += E[a * d + k] / std::sqrt(Dv[k]) * ex;
                }
                v[idx[a]] += rc * s;
            }
            double *w = params_out + (size_t)(l * o.n_sphere + i) * D5;
            to_natural(v, klarge, w);
            if (o.kappa_fixed) w[1] = omega_hat[1];
            // nugget repair: a sampled nu below zero is a negative nugget; half
            // of these become 0, the other half uniform draws on (0, 2)
            if (v[2] < 0.0) w[2] = (neg++ % 2 == 0) ? 0.0 : 2.0 * rng.uniform();
        }
    }
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// the same on a context's GPU evaluation
// ---------------------------------------------------------------------------
namespace {
struct CtxEval {
    plk_ctx *ctx;
    plk_dataset ds;
    int32_t precision, reml;
};
int32_t ctx_eval(void *u, const double *params, int64_t K, const double *lam, int32_t M, double *logL) {
    CtxEval *e = static_cast<CtxEval *>(u);
    plk_options o{};
    o.precision = e->precision;
    o.reml = e->reml;
    plk_job job = 0;
    plk_status st = plk_submit_profile(e->ctx, e->ds, params, K, lam, M, &o, &job);
    if (st == PLK_OK) st = plk_poll(e->ctx, job, -1, logL, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
    return (int32_t)st;
}
}  // namespace

extern "C" plk_status plk_fit_mle(plk_ctx *ctx, plk_dataset ds, const double *omega0, double lambda0,
                                  const plk_fit_options *opts, double *omega_hat, double *lambda_hat, double *logL_hat,
                                  int32_t *iterations) {
    if (!ctx) return bad("plk_fit_mle: ctx is NULL");
    CtxEval e{ctx, ds, opts ? opts->precision : PLK_FP64, opts ? opts->reml : 0};
    return plk_fit_mle_cb(ctx_eval, &e, omega0, lambda0, opts, omega_hat, lambda_hat, logL_hat, iterations);
}

extern "C" plk_status plk_quadratic_cloud(plk_ctx *ctx, plk_dataset ds, const double *omega_hat, double lambda_hat,
                                          const plk_cloud_options *opts, double *params_out, int64_t capacity,
                                          int64_t *K_out, double *lambdas_out, double *hessian_out, double *eig_out) {
    if (!ctx) return bad("plk_quadratic_cloud: ctx is NULL");
    CtxEval e{ctx, ds, opts ? opts->precision : PLK_FP64, opts ? opts->reml : 0};
    return plk_quadratic_cloud_cb(ctx_eval, &e, omega_hat, lambda_hat, opts, params_out, capacity, K_out, lambdas_out,
                                  hessian_out, eig_out);
}
