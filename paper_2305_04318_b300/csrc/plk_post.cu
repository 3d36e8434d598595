// plk_post.cu -- post-processing of the Table-1 statistics on the device
// (Sections 3.2 and 3.4-3.6 of Xu & Brown, arXiv 2305.04318).
//
//   k_prof_closed   profile of one regression coefficient beta_j (eq.
//                   profilebetai) or of sigma (eq. profileSigma): each thread
//                   reduces one (omega_k, lambda_m) pair to a few coefficients
//                   of a closed form in the grid value, each block takes the
//                   max over its pairs for every grid value, blocks combine
//                   through an atomic max on order-preserving integer keys
//   k_keys_to_prof  keys -> doubles (NaN where no pair gave a finite value)
//   k_col_max       profile of lambda: max over the omega points per lambda
//   k_hull_flags    vertices of the upper convex hull of a 1-D point cloud
//   k_hull_query    linear interpolation of the hull vertices at query points
//   k_internal      internal parameters omega' (Section 3.2)
//
// All are small next to the evaluation itself (O(K M G) closed forms, O(K^2)
// pair tests for the hull); they exist so that the profiles come out of the
// statistics without a round trip through host memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "plk.h"
#include "plk_common.cuh"
#include "plk_kernels.cuh"

namespace plk {
namespace {

constexpr int NTP = 256;   // threads per block of every kernel here
constexpr int PMAX = 16;   // largest p the evaluation accepts

// Order-preserving map of non-NaN doubles to unsigned 64-bit keys (a larger
// double gives a larger key; -inf maps above 0), so that an integer atomic max
// reduces doubles.  Key 0 means "no value".
__device__ __forceinline__ unsigned long long dkey(double v) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__device__ __forceinline__ double dunkey(unsigned long long k) {
    return (k >> 63) ? __longlong_as_double((long long)(k & 0x7fffffffffffffffull))
                     : __longlong_as_double((long long)~k);
}

// sum_i log y_i by one block, in a fixed order (every block that calls it gets
// the same value).
__device__ double block_sum_log(int64_t n, const double *__restrict__ y, double *red) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += NTP) s += log(y[i]);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = NTP / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// In-place Cholesky of the d x d matrix in A (row-major, lower triangle used).
// Returns false if a pivot is not positive.
__device__ bool small_chol(int d, double *A) {
    for (int c = 0; c < d; ++c) {
        double v = A[c * PMAX + c];
        for (int k = 0; k < c; ++k) v -= A[c * PMAX + k] * A[c * PMAX + k];
        if (!(v > 0.0)) return false;
        const double l = sqrt(v);
        A[c * PMAX + c] = l;
        for (int r = c + 1; r < d; ++r) {
            double t = A[r * PMAX + c];
            for (int k = 0; k < c; ++k) t -= A[r * PMAX + k] * A[c * PMAX + k];
            A[r * PMAX + c] = t / l;
        }
    }
    return true;
}

// z = L^-1 b for the factor in A (row-major, PMAX stride).
__device__ void small_fwd(int d, const double *A, const double *b, double *z) {
    for (int r = 0; r < d; ++r) {
        double t = b[r];
        for (int k = 0; k < r; ++k) t -= A[r * PMAX + k] * z[k];
        z[r] = t / A[r * PMAX + r];
    }
}

// mode 0: profile of beta_j.  With beta_j = b fixed, the residual sum of
//   squares of the GLS fit of y' - X_j b on X_-j is the quadratic
//   RSS(b) = c0 - 2 c1 b + c2 b^2, where, with A_-j = (X^T V^-1 X)_[-j,-j]
//   = Q Q^T, z_y = Q^-1 (X^T V^-1 y')_[-j] and z_x = Q^-1 (X^T V^-1 X)_[-j,j]:
//   c0 = y'^T V^-1 y' - z_y.z_y, c1 = (X^T V^-1 y')_j - z_x.z_y,
//   c2 = (X^T V^-1 X)_jj - z_x.z_x (Section 3.4).  Then
//   l(b) = h - (n/2) log RSS(b),
//   h = -(1/2) [log|V| - 2 (lambda-1) sum log y + n log(2 pi) + n - n log n].
// mode 1: profile of sigma.  RSS = y'^T V^-1 y' - |Q^-1 X^T V^-1 y'|^2 with
//   X^T V^-1 X = Q Q^T, C = log|V| - 2 (lambda-1) sum log y + n log(2 pi), and
//   l(s) = -(1/2) [RSS / s^2 + n log s^2 + C] (eq. profileSigma).
// One thread per (k, m) pair; the block's pairs are then swept for every grid
// value.  keys: G order-preserving keys, zero on entry.
__global__ void __launch_bounds__(NTP) k_prof_closed(int mode, int reml, int64_t n, int p, int M, int64_t K,
                                                     const double *__restrict__ y,
                                                     const double *__restrict__ lambdas,
                                                     const double *__restrict__ ssq,
                                                     const double *__restrict__ logdet,
                                                     const int32_t *__restrict__ status, int j,
                                                     int64_t G, const double *__restrict__ grid,
                                                     unsigned long long *__restrict__ keys) {
    __shared__ double red[NTP];
    __shared__ double cf[4][NTP];
    __shared__ int valid[NTP];
    const double J = block_sum_log(n, y, red);
    const int q = M + p;
    const int64_t pairs = K * (int64_t)M;
    const int64_t pr = (int64_t)blockIdx.x * NTP + threadIdx.x;
    int ok = 0;
    double c0 = 0.0, c1 = 0.0, c2 = 0.0, h = 0.0;
    if (pr < pairs) {
        const int64_t k = pr / M;
        const int m = (int)(pr - k * M);
        const double *S = ssq + k * (int64_t)q * q;
        const double ldv = logdet[2 * k];
        const double ldx = logdet[2 * k + 1];   // log|X^T V^-1 X| (REML only)
        ok = (status == nullptr || (status[k] & 15) == 0) && isfinite(ldv) && (!reml || isfinite(ldx));
        double A[PMAX * PMAX], zy[PMAX], zx[PMAX], by[PMAX], bx[PMAX];
        const double two_pi_log = 1.8378770664093454836;   // log(2 pi)
        const double jac = -2.0 * (lambdas[m] - 1.0) * J;
        if (ok && mode == 0) {
            int d = 0;
            for (int a = 0; a < p; ++a) {
                if (a == j) continue;
                int e = 0;
                for (int c = 0; c <= a; ++c) {
                    if (c == j) continue;
                    A[d * PMAX + e] = S[(M + a) * q + (M + c)];
                    ++e;
                }
                by[d] = S[(M + a) * q + m];
                bx[d] = S[(M + a) * q + (M + j)];
                ++d;
            }
            ok = small_chol(d, A);
            if (ok) {
                small_fwd(d, A, by, zy);
                small_fwd(d, A, bx, zx);
                double yy = 0.0, xy = 0.0, xx = 0.0;
                for (int a = 0; a < d; ++a) {
                    yy += zy[a] * zy[a];
                    xy += zx[a] * zy[a];
                    xx += zx[a] * zx[a];
                }
                c0 = S[m * q + m] - yy;
                c1 = S[(M + j) * q + m] - xy;
                c2 = S[(M + j) * q + (M + j)] - xx;
                const double dn = (double)n;
                if (reml) {   // Appendix, eq. remlprofileytilde
                    const double de = (double)(n - p);
                    h = -0.5 * (ldv + ldx + jac + dn * two_pi_log + de - de * log(de));
                } else {
                    h = -0.5 * (ldv + jac + dn * two_pi_log + dn - dn * log(dn));
                }
            }
        } else if (ok) {
            for (int a = 0; a < p; ++a) {
                for (int c = 0; c <= a; ++c) A[a * PMAX + c] = S[(M + a) * q + (M + c)];
                by[a] = S[(M + a) * q + m];
            }
            ok = small_chol(p, A);
            if (ok) {
                small_fwd(p, A, by, zy);
                double yy = 0.0;
                for (int a = 0; a < p; ++a) yy += zy[a] * zy[a];
                c0 = S[m * q + m] - yy;
                ok = c0 > 0.0;
                h = ldv + jac + (double)n * two_pi_log;
            }
        }
        ok = ok && isfinite(c0) && isfinite(c1) && isfinite(c2) && isfinite(h);
    }
    cf[0][threadIdx.x] = c0;
    cf[1][threadIdx.x] = c1;
    cf[2][threadIdx.x] = c2;
    cf[3][threadIdx.x] = h;
    valid[threadIdx.x] = ok;
    __syncthreads();
    const int64_t first = (int64_t)blockIdx.x * NTP;
    const int np = (int)((pairs - first) < NTP ? (pairs - first) : NTP);
    const double dn = (double)n;
    const double de = reml ? (double)(n - p) : dn;   // the log term's weight
    for (int64_t g = threadIdx.x; g < G; g += NTP) {
        const double b = grid[g];
        double best = -INFINITY;
        int any = 0;
        for (int i = 0; i < np; ++i) {
            if (!valid[i]) continue;
            double v;
            if (mode == 0) {
                const double rss = cf[0][i] - 2.0 * cf[1][i] * b + cf[2][i] * b * b;
                v = rss > 0.0 ? cf[3][i] - 0.5 * de * log(rss) : NAN;
            } else {
                const double s2 = b * b;
                v = b > 0.0 ? -0.5 * (cf[0][i] / s2 + dn * log(s2) + cf[3][i]) : NAN;
            }
            if (v == v) {
                best = any ? fmax(best, v) : v;
                any = 1;
            }
        }
        if (any) atomicMax(keys + g, dkey(best));
    }
}

__global__ void k_keys_to_prof(int64_t G, double *prof) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const unsigned long long k = reinterpret_cast<unsigned long long *>(prof)[g];
    prof[g] = k ? dunkey(k) : NAN;
}

// prof[m] = NaN-skipping max over k of vals[k * M + m]; one block per m.
__global__ void __launch_bounds__(NTP) k_col_max(const double *__restrict__ vals, int64_t K, int M,
                                                 double *__restrict__ prof) {
    __shared__ double red[NTP];
    __shared__ int anyv[NTP];
    const int m = blockIdx.x;
    double best = -INFINITY;
    int any = 0;
    for (int64_t k = threadIdx.x; k < K; k += NTP) {
        const double v = vals[k * M + m];
        if (v == v) {
            best = any ? fmax(best, v) : v;
            any = 1;
        }
    }
    red[threadIdx.x] = best;
    anyv[threadIdx.x] = any;
    __syncthreads();
    for (int o = NTP / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            if (anyv[threadIdx.x + o]) {
                red[threadIdx.x] = anyv[threadIdx.x] ? fmax(red[threadIdx.x], red[threadIdx.x + o])
                                                     : red[threadIdx.x + o];
                anyv[threadIdx.x] = 1;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) prof[m] = anyv[0] ? red[0] : NAN;
}

// Upper convex hull of the points (x[k * xs], v[k]) with finite coordinates
// (Section 3.6).  Point i is a vertex when it is the only point with the
// largest value at its x (ties: lowest index) and some line through it has
// every other point strictly below: with s_L = the smallest slope from a point
// on its left to i and s_R = the largest slope from i to a point on its right,
// that is s_R < s_L (a missing side counts as +inf / -inf).  Slopes are
// compared by cross-multiplication (denominators are positive).  One thread per
// point; the other points stream through shared memory in tiles.
__global__ void __launch_bounds__(NTP) k_hull_flags(int64_t K, const double *__restrict__ x, int64_t xs,
                                                    const double *__restrict__ v, int32_t *__restrict__ on) {
    __shared__ double tx[NTP], tv[NTP];
    const int64_t i = (int64_t)blockIdx.x * NTP + threadIdx.x;
    double xi = NAN, vi = NAN;
    if (i < K) {
        xi = x[i * xs];
        vi = v[i];
    }
    const bool mine = i < K && isfinite(xi) && isfinite(vi);
    bool dominated = false, hasL = false, hasR = false;
    double lnum = 0.0, lden = 1.0, rnum = 0.0, rden = 1.0;   // s_L = lnum/lden, s_R = rnum/rden
    for (int64_t t0 = 0; t0 < K; t0 += NTP) {
        const int64_t jj = t0 + threadIdx.x;
        double a = NAN, b = NAN;
        if (jj < K) {
            a = x[jj * xs];
            b = v[jj];
        }
        if (!(isfinite(a) && isfinite(b))) a = NAN;
        tx[threadIdx.x] = a;
        tv[threadIdx.x] = b;
        __syncthreads();
        const int cnt = (K - t0) < NTP ? (int)(K - t0) : NTP;
        if (mine) {
            for (int u = 0; u < cnt; ++u) {
                const double xj = tx[u];
                if (xj != xj) continue;
                const double vj = tv[u];
                if (xj == xi) {
                    if (vj > vi || (vj == vi && t0 + u < i)) dominated = true;
                } else if (xj < xi) {
                    const double num = vi - vj, den = xi - xj;   // slope from j up to i
                    if (!hasL || num * lden < lnum * den) {
                        lnum = num;
                        lden = den;
                        hasL = true;
                    }
                } else {
                    const double num = vj - vi, den = xj - xi;   // slope from i to j
                    if (!hasR || num * rden > rnum * den) {
                        rnum = num;
                        rden = den;
                        hasR = true;
                    }
                }
            }
        }
        __syncthreads();
    }
    if (i < K) {
        int vert = 0;
        if (mine && !dominated) vert = (!hasL || !hasR) ? 1 : (rnum * lden < lnum * rden);
        on[i] = vert;
    }
}

// out[t] = the hull's linear interpolant at xq[t]; NaN outside the vertices'
// x range.  One warp per query scans the vertex flags.
__global__ void k_hull_query(int64_t K, const double *__restrict__ x, int64_t xs,
                             const double *__restrict__ v, const int32_t *__restrict__ on, int64_t Q,
                             const double *__restrict__ xq, double *__restrict__ out) {
    const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= Q) return;
    const double z = xq[t];
    // left: the vertex with the largest x <= z; right: the smallest x >= z
    double lx = -INFINITY, lv = NAN, rx = INFINITY, rv = NAN;
    for (int64_t k = lane; k < K; k += 32) {
        if (!on[k]) continue;
        const double a = x[k * xs];
        if (a <= z && a > lx) {
            lx = a;
            lv = v[k];
        }
        if (a >= z && a < rx) {
            rx = a;
            rv = v[k];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ox = __shfl_xor_sync(0xffffffffu, lx, o), ov = __shfl_xor_sync(0xffffffffu, lv, o);
        if (ox > lx) {
            lx = ox;
            lv = ov;
        }
        const double px = __shfl_xor_sync(0xffffffffu, rx, o), pv = __shfl_xor_sync(0xffffffffu, rv, o);
        if (px < rx) {
            rx = px;
            rv = pv;
        }
    }
    if (lane == 0) {
        double r = NAN;
        if (lx == z)
            r = lv;
        else if (lv == lv && rv == rv)
            r = lv + (rv - lv) * (z - lx) / (rx - lx);
        out[t] = r;
    }
}

// omega -> omega' = (gamma_1, kappa~, nu, gamma_2, gamma_3) (Section 3.2): a
// ratio phi_X/phi_Y below one is first expressed with the axes exchanged,
// (phi_X, phi_Y, phi_A) -> (phi_Y, phi_X, phi_A + pi/2), which leaves the
// correlation unchanged and flips the sign of (gamma_2, gamma_3).
__global__ void k_internal(const double *__restrict__ params, int64_t K, int large,
                           double *__restrict__ out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const double *w = params + 5 * k;
    const double phx = w[0], kap = w[1], nug = w[2], rat = w[3], ang = w[4];
    const double phy = phx / rat;
    double *o = out + 5 * k;
    o[0] = log(phx) + log(phy);
    o[1] = large ? rsqrt(kap) : log(kap);
    o[2] = sqrt(nug);
    const double ratio = phx / phy;
    const double r = ratio >= 1.0 ? sqrt(ratio - 1.0) : -sqrt(phy / phx - 1.0);
    double sn, cs;
    sincos(2.0 * ang, &sn, &cs);
    o[3] = r * cs;
    o[4] = r * sn;
}

plk_status post_fail(plk_status s, const std::string &msg) {
    set_last_error(msg.c_str());
    return s;
}

plk_status post_cuda(cudaError_t e, const char *where) {
    return post_fail(PLK_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

plk_status check_stats(const plk_stats_args *a, const char *who) {
    if (!a) return post_fail(PLK_E_INVALID, std::string(who) + ": stats is NULL");
    if (a->p < 1 || a->p > PMAX || a->n <= a->p || a->M < 1 || a->M + a->p > 64 || a->K < 0)
        return post_fail(PLK_E_INVALID, std::string(who) + ": bad sizes (need n > p >= 1, p <= 16, M >= 1, "
                                                           "M + p <= 64, K >= 0)");
    if (!a->y || !a->lambdas || (a->K > 0 && (!a->ssq_yx || !a->logdet)))
        return post_fail(PLK_E_INVALID, std::string(who) + ": NULL input");
    return PLK_OK;
}

plk_status run_closed(int mode, int reml, const plk_stats_args *a, int32_t j, const double *grid, int64_t G,
                      double *prof, void *stream, const char *who) {
    plk_status st = check_stats(a, who);
    if (st != PLK_OK) return st;
    if (mode == 0 && (j < 0 || j >= a->p)) return post_fail(PLK_E_INVALID, std::string(who) + ": j out of range");
    if (G < 0 || (G > 0 && (!grid || !prof))) return post_fail(PLK_E_INVALID, std::string(who) + ": bad grid");
    if (G == 0) return PLK_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(prof, 0, sizeof(double) * (size_t)G, s);
    if (e != cudaSuccess) return post_cuda(e, who);
    const int64_t pairs = a->K * (int64_t)a->M;
    if (pairs > 0) {
        const int64_t blocks = (pairs + NTP - 1) / NTP;
        if (blocks > INT32_MAX) return post_fail(PLK_E_INVALID, std::string(who) + ": K too large");
        k_prof_closed<<<(unsigned)blocks, NTP, 0, s>>>(mode, reml, a->n, a->p, a->M, a->K, a->y, a->lambdas, a->ssq_yx,
                                                       a->logdet, a->status, j, G, grid,
                                                       reinterpret_cast<unsigned long long *>(prof));
        if ((e = cudaGetLastError()) != cudaSuccess) return post_cuda(e, who);
    }
    k_keys_to_prof<<<(unsigned)((G + NTP - 1) / NTP), NTP, 0, s>>>(G, prof);
    if ((e = cudaGetLastError()) != cudaSuccess) return post_cuda(e, who);
    return PLK_OK;
}

}  // namespace
}  // namespace plk

using namespace plk;

extern "C" plk_status plk_profile_beta_device(const plk_stats_args *stats, int32_t j, const double *grid,
                                              int64_t G, double *prof, void *stream) {
    return run_closed(0, 0, stats, j, grid, G, prof, stream, "plk_profile_beta_device");
}

extern "C" plk_status plk_profile_beta_reml_device(const plk_stats_args *stats, int32_t j, const double *grid,
                                                   int64_t G, double *prof, void *stream) {
    return run_closed(0, 1, stats, j, grid, G, prof, stream, "plk_profile_beta_reml_device");
}

extern "C" plk_status plk_profile_sigma_device(const plk_stats_args *stats, const double *grid, int64_t G,
                                               double *prof, void *stream) {
    return run_closed(1, 0, stats, 0, grid, G, prof, stream, "plk_profile_sigma_device");
}

extern "C" plk_status plk_profile_lambda_device(const double *logL, int64_t K, int32_t M, double *prof,
                                                void *stream) {
    if (K < 0 || M < 1 || M > 65535 || !prof || (K > 0 && !logL))
        return post_fail(PLK_E_INVALID, "plk_profile_lambda_device: bad arguments");
    k_col_max<<<M, NTP, 0, static_cast<cudaStream_t>(stream)>>>(logL, K, M, prof);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PLK_OK : post_cuda(e, "plk_profile_lambda_device");
}

extern "C" plk_status plk_profile_hull_device(const double *x, int64_t x_stride, const double *v, int64_t K,
                                              const double *xq, int64_t Q, double *out, int32_t *on_hull,
                                              void *stream) {
    if (K < 0 || Q < 0 || x_stride < 1 || (K > 0 && (!x || !v || !on_hull)) || (Q > 0 && (!xq || !out)))
        return post_fail(PLK_E_INVALID, "plk_profile_hull_device: bad arguments");
    if ((K + NTP - 1) / NTP > INT32_MAX || (Q + 7) / 8 > INT32_MAX)
        return post_fail(PLK_E_INVALID, "plk_profile_hull_device: K or Q too large");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (K > 0) {
        k_hull_flags<<<(unsigned)((K + NTP - 1) / NTP), NTP, 0, s>>>(K, x, x_stride, v, on_hull);
        if ((e = cudaGetLastError()) != cudaSuccess) return post_cuda(e, "plk_profile_hull_device");
    }
    if (Q > 0) {
        k_hull_query<<<(unsigned)((Q + 7) / 8), NTP, 0, s>>>(K, x, x_stride, v, on_hull, Q, xq, out);
        if ((e = cudaGetLastError()) != cudaSuccess) return post_cuda(e, "plk_profile_hull_device");
    }
    return PLK_OK;
}

extern "C" plk_status plk_internal_params_device(const double *params, int64_t K, int32_t kappa_hat_large,
                                                 double *out, void *stream) {
    if (K < 0 || (K > 0 && (!params || !out)) || (K + NTP - 1) / NTP > INT32_MAX)
        return post_fail(PLK_E_INVALID, "plk_internal_params_device: bad arguments");
    if (K == 0) return PLK_OK;
    k_internal<<<(unsigned)((K + NTP - 1) / NTP), NTP, 0, static_cast<cudaStream_t>(stream)>>>(
        params, K, kappa_hat_large ? 1 : 0, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PLK_OK : post_cuda(e, "plk_internal_params_device");
}
