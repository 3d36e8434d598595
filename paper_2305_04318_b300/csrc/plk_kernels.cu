// plk_kernels.cu -- FP64 CUDA kernels of the profile-likelihood hot path
// (Xu & Brown, arXiv 2305.04318, Section 3.3 "Step 3" and Table 2), for sm_103a.
//
// Pipeline for a batch of parameter points omega (one CUDA block grid per step):
//   k_dataset_front B^T = [y'(lambda_1..lambda_M) | X]^T, sum log y  (Section 2 Box-Cox)
//                   and the smallest site distance, in one launch
//   k_omega_prep    per-omega constants, rotated/scaled coordinates  (eq. matern)
//   k_matern_table  per-omega piecewise polynomial of rho(w), w = 8 kappa d^2
//   k_build         bordered matrix tiles: V = R + nu^2 I and B^T     (Step 3 item 1)
//   k_build_f32     the same tiles as double-float planes, evaluated in FP32
//                   pair arithmetic (first pass of the mixed-precision path)
//   for each tile column J:
//     k_potrf       diagonal tile L_JJ, its inverse, log|V| partial   (item 2)
//     k_gemm_nt<0>  panel L_IJ = A_IJ L_JJ^-T (also W^T rows)         (items 2-3)
//     k_gemm_nt<1>  trailing A_IK -= L_IJ L_KJ^T (also -B^T V^-1 B)   (items 2-4)
//   k_finalize      p x p Cholesky, beta-hat, RSS, sigma-hat^2, l_p    (items 5-8, eqs. betahat,
//                                                                        4, profile, remlpro)
// On this part FP64 issues at ~1/67 of the FP32 rate, so every kernel here is
// bound by FP64 instruction count; the build evaluates rho with a handful of
// FP64 operations per matrix entry (no exp/sqrt per entry).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "plk.h"
#include "plk_common.cuh"
#include "plk_kernels.cuh"

namespace plk {

// ---------------------------------------------------------------------------
// Box-Cox rows and sum of log y
// ---------------------------------------------------------------------------

// Box-Cox rows, as block bid of nblk blocks
__device__ __forceinline__ void boxcox_rows_part(int bid, int nblk, int64_t n, int64_t n_pad, int p, int M,
                                                 const double *__restrict__ y, const double *__restrict__ X,
                                                 const double *__restrict__ lam, double *__restrict__ Bt) {
    const int q = M + p;
    const int64_t total = (int64_t)q * n_pad;
    for (int64_t e = bid * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)nblk * blockDim.x) {
        const int r = (int)(e / n_pad);
        const int64_t i = e - (int64_t)r * n_pad;
        double v = 0.0;
        if (i < n) {
            if (r < M) {
                const double l = lam[r];
                const double ly = log(y[i]);
                v = (l == 0.0) ? ly : expm1(l * ly) / l;   // b(y; lambda), Section 2
            } else {
                v = X[i * p + (r - M)];
            }
        }
        Bt[e] = v;
    }
}

// sum_i log y_i by one block (a fixed summation order)
__device__ __forceinline__ void sumlog_part(int64_t n, const double *__restrict__ y, double *__restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += log(y[i]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *out = s;
    }
}

// ---------------------------------------------------------------------------
// Per-omega constants and transformed coordinates
// ---------------------------------------------------------------------------
// a_i = sqrt(8k)/phi_X (cos x_i - sin y_i), b_i = sqrt(8k)/phi_Y (sin x_i + cos y_i), so that
// w_ij = (a_i - a_j)^2 + (b_i - b_j)^2 = u_ij^2 with u = sqrt(8 kappa) d (eq. matern,
// rotation matrix as printed, phi_Y = phi_X / phi_R).
__global__ void __launch_bounds__(256) k_omega_prep(const double *__restrict__ params, int64_t n, int64_t n_pad,
                                                    const double *__restrict__ coords,
                                                    const double *__restrict__ sumlogy, double *__restrict__ oconst,
                                                    double *__restrict__ coordT, double *__restrict__ logdet,
                                                    int *__restrict__ pstatus, int f32coords,
                                                    const int *__restrict__ gate, const int *__restrict__ dcount = nullptr) {
    const int w = blockIdx.x;
    if (gate && !gate[w]) return;   // gated pass: only the flagged slots
    if (beyond(dcount, w)) return;  // slots past the device-side count of a compacted batch
    const double *om = params + 5 * (int64_t)w;
    const double phix = om[0], kap = om[1], nug = om[2], ratio = om[3], ang = om[4];
    const bool ok = (phix > 0.0) && (kap > 0.0) && (nug >= 0.0) && (ratio > 0.0) &&
                    isfinite(phix) && isfinite(kap) && isfinite(nug) && isfinite(ratio) &&
                    isfinite(ang);
    // the point's transcendentals once per block, one per warp 0..3 (one per
    // SM sub-partition: an FP64 warp instruction holds its sub-partition's
    // FP64 pipe for 64 cycles, so four short chains run side by side)
    __shared__ double sc[6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        if (warp == 0) sc[0] = cos(ang);
        else if (warp == 1) sc[1] = sin(ang);
        else if (warp == 2) {
            sc[2] = sqrt(8.0 * kap);
            const double iphi = 1.0 / phix;
            sc[3] = sc[2] * iphi;
            sc[4] = sc[2] * ratio * iphi;
        } else if (warp == 3) {
            sc[5] = (1.0 - kap) * 0.69314718055994530942 - lgamma(kap);
        }
    }
    __syncthreads();
    const double c = sc[0], s = sc[1], s8k = sc[2], ia = sc[3], ib = sc[4];
    if (threadIdx.x == 0) {
        double *oc = oconst + OC_N * (int64_t)w;
        oc[OC_KAPPA] = kap;
        oc[OC_NUG] = nug;
        oc[OC_LOGC] = sc[5];
        oc[OC_S8K] = s8k;
        oc[OC_COS] = c;
        oc[OC_SIN] = s;
        oc[OC_IA] = ia;
        oc[OC_IB] = ib;
        logdet[w] = 0.0;
        pstatus[w] = ok ? PLK_POINT_OK : PLK_POINT_BAD_PARAM;
    }
    double *a = coordT + (int64_t)w * 2 * n_pad;
    double *b = a + n_pad;
    // f32coords: the same region as four float arrays [a_hi | a_lo | b_hi | b_lo]
    float *af = reinterpret_cast<float *>(a);
    // bounding box of the transformed sites: w = |a_i - a_j|^2 + |b_i - b_j|^2 is
    // at most its squared diagonal, and at least min(ia, ib)^2 times the
    // smallest squared site distance (the rotation keeps lengths).  The box is
    // reduced in FP32 with its edges rounded outwards (it only chooses table
    // octaves, with a margin).
    float alo = INFINITY, ahi = -INFINITY, blo = INFINITY, bhi = -INFINITY;
    for (int64_t i = threadIdx.x; i < n_pad; i += blockDim.x) {
        double ai = 0.0, bi = 0.0;
        if (i < n && ok) {
            const double x = coords[2 * i], yv = coords[2 * i + 1];
            ai = (c * x - s * yv) * ia;
            bi = (s * x + c * yv) * ib;
            alo = fminf(alo, __double2float_rd(ai));
            ahi = fmaxf(ahi, __double2float_ru(ai));
            blo = fminf(blo, __double2float_rd(bi));
            bhi = fmaxf(bhi, __double2float_ru(bi));
        }
        if (f32coords) {
            const float ah = __double2float_rn(ai), bh = __double2float_rn(bi);
            af[i] = ah;
            af[n_pad + i] = __double2float_rn(ai - (double)ah);
            af[2 * n_pad + i] = bh;
            af[3 * n_pad + i] = __double2float_rn(bi - (double)bh);
        } else {
            a[i] = ai;
            b[i] = bi;
        }
    }
    __shared__ float red[4][8];
    for (int o = 16; o > 0; o >>= 1) {
        alo = fminf(alo, __shfl_xor_sync(0xffffffffu, alo, o));
        ahi = fmaxf(ahi, __shfl_xor_sync(0xffffffffu, ahi, o));
        blo = fminf(blo, __shfl_xor_sync(0xffffffffu, blo, o));
        bhi = fmaxf(bhi, __shfl_xor_sync(0xffffffffu, bhi, o));
    }
    if (lane == 0) {
        red[0][warp] = alo;
        red[1][warp] = ahi;
        red[2][warp] = blo;
        red[3][warp] = bhi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            alo = fminf(alo, red[0][q]);
            ahi = fmaxf(ahi, red[1][q]);
            blo = fminf(blo, red[2][q]);
            bhi = fmaxf(bhi, red[3][q]);
        }
        int elo = TAB_ELO, ehi = TAB_EHI;
        if (ok && n > 1) {
            const double da = (double)ahi - (double)alo, db = (double)bhi - (double)blo;
            const double whi = da * da + db * db;
            const double sc = fmin(ia, ib);
            const double wlo = sc * sc * sumlogy[1];
            int e;
            if (whi > 0.0 && isfinite(whi)) {
                frexp(whi, &e);          // whi < 2^e
                ehi = min(TAB_EHI, max(TAB_ELO, e + 1));
            }
            if (wlo > 0.0 && isfinite(wlo)) {
                frexp(wlo, &e);          // wlo >= 2^(e - 1)
                elo = min(ehi, max(TAB_ELO, e - 2));
            }
        }
        double *oc = oconst + OC_N * (int64_t)w;
        oc[OC_ELO] = elo;
        oc[OC_EHI] = ehi;
    }
}

// Smallest squared distance between two sites (min over i < j), into *out
// (which holds a large positive value beforehand): gridDim.y (1, 2, 4 or 8)
// blocks per pair of 128-site tiles, non-negative doubles compared through
// their bit patterns.
__device__ __forceinline__ void min_dist2_part(int t, int split, int ys, int64_t n,
                                               const double *__restrict__ coords, double *__restrict__ out) {
    int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;   // tile pair J <= I
    __shared__ double xj[128], yj[128];
    const int64_t j0 = (int64_t)J * 128, i0 = (int64_t)I * 128;
    if (threadIdx.x < 128) {
        const int64_t j = j0 + threadIdx.x;
        xj[threadIdx.x] = j < n ? coords[2 * j] : 0.0;
        yj[threadIdx.x] = j < n ? coords[2 * j + 1] : 0.0;
    }
    __syncthreads();
    double best = INFINITY;
    // split blocks share the tile pair (few pairs: small n); this is block ys
    const int per = 128 * 128 / split, r0 = ys * per;
    for (int r = r0 + threadIdx.x; r < r0 + per; r += blockDim.x) {
        const int64_t i = i0 + (r >> 7), j = j0 + (r & 127);
        if (i < n && j < i) {
            const double dx = coords[2 * i] - xj[r & 127], dy = coords[2 * i + 1] - yj[r & 127];
            best = fmin(best, fma(dx, dx, dy * dy));
        }
    }
    for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best < INFINITY)
        atomicMin(reinterpret_cast<unsigned long long *>(out), (unsigned long long)__double_as_longlong(best));
}

__global__ void __launch_bounds__(256) k_min_dist2(int64_t n, const double *__restrict__ coords,
                                                   double *__restrict__ out) {
    min_dist2_part((int)blockIdx.x, (int)gridDim.y, (int)blockIdx.y, n, coords, out);
}

// The dataset's per-call preprocessing in one launch (the three parts are
// independent): blocks 0 .. nbox - 1 write the Box-Cox rows B^T, block nbox
// sums log y, the rest (split per tile pair) take the smallest squared site
// distance.
__global__ void __launch_bounds__(256) k_dataset_front(int nbox, int split, int64_t n, int64_t n_pad, int p, int M,
                                                       const double *__restrict__ y, const double *__restrict__ X,
                                                       const double *__restrict__ lam, double *__restrict__ Bt,
                                                       const double *__restrict__ coords,
                                                       double *__restrict__ sumlogy) {
    const int b = (int)blockIdx.x;
    if (b < nbox) {
        boxcox_rows_part(b, nbox, n, n_pad, p, M, y, X, lam, Bt);
    } else if (b == nbox) {
        sumlog_part(n, y, sumlogy);
    } else {
        const int r = b - nbox - 1;
        min_dist2_part(r / split, split, r % split, n, coords, sumlogy + 1);
    }
}

// ---------------------------------------------------------------------------
// rho(u) by the integral K_kappa(u) = int_0^inf exp(-u cosh t) cosh(kappa t) dt
// ---------------------------------------------------------------------------
// rho = exp(log c_kappa + kappa log u - u) * int_0^inf exp(-2u sinh^2(t/2)) cosh(kappa t) dt,
// trapezoid rule (geometric convergence for this analytic integrand).

// General evaluator: step min(0.1, 0.45/sqrt(u)), integrand formed in log space
// (no overflow of cosh(kappa t)); used for u > TAB_USPLIT and for tiny w.
__device__ double rho_integral(double u, double kap, double logc) {
    if (u < 1e-15 && kap >= 0.5) return 1.0;
    double h = 0.45 * rsqrt(u);
    if (h > 0.1) h = 0.1;
    // cosh(kappa t) = e^{kappa t} (1 + e^{-2 kappa t}) / 2, the second factor
    // advanced by one multiplication per node (its rounding stays below
    // k 2^-53 of a term at most 1 beside the 1)
    const double r = exp(-2.0 * kap * h);
    double rk = 1.0, sum = 0.5, prev = 1.0;
    for (int k = 1; k < 20000; ++k) {
        const double t = k * h;
        const double sh = sinh(0.5 * t);
        rk *= r;
        const double g = exp(kap * t - 0.69314718055994530942 - 2.0 * u * sh * sh) * (1.0 + rk);
        sum += g;
        if (g < prev && g < 1e-18 * sum) break;
        prev = g;
    }
    return exp(logc + kap * log(u) - u) * (h * sum);
}

// Table sharing: the rho table depends on the point only through kappa (and
// log c_kappa, a function of kappa), so slots of a batch with the same kappa
// read one table.  owner[w] = the smallest slot with the same kappa (bit
// pattern) and a valid parameter row; an invalid row keeps its own.
__global__ void __launch_bounds__(256) k_table_owner(int cnt, const double *__restrict__ oconst,
                                                     const int *__restrict__ pstatus, int *__restrict__ owner,
                                                     const int *__restrict__ dcount = nullptr) {
    const int w = blockIdx.x;
    if (beyond(dcount, w)) return;
    __shared__ int best[8];
    int b = w;
    if (pstatus[w] == PLK_POINT_OK) {
        const unsigned long long kw = (unsigned long long)__double_as_longlong(oconst[OC_N * (int64_t)w + OC_KAPPA]);
        for (int v = threadIdx.x; v < w; v += blockDim.x)
            if (pstatus[v] == PLK_POINT_OK &&
                (unsigned long long)__double_as_longlong(oconst[OC_N * (int64_t)v + OC_KAPPA]) == kw) {
                b = v;
                break;   // v grows with the loop: the first match is this thread's smallest
            }
    }
    for (int o = 16; o > 0; o >>= 1) b = min(b, __shfl_xor_sync(0xffffffffu, b, o));
    if ((threadIdx.x & 31) == 0) best[threadIdx.x >> 5] = b;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) b = min(b, best[i]);
        owner[w] = b;
    }
}

// The owner's table covers the union of its sharers' octave ranges.
// Both steps for a batch of at most 256 slots in one block (one launch
// instead of two where the batch is small): the keys in shared memory, then
// every slot's owner, then every owner's octave range over its members.
constexpr int TABLE_SHARE_SMALL = 256;
__global__ void __launch_bounds__(TABLE_SHARE_SMALL) k_table_share_small(int cnt, double *__restrict__ oconst,
                                                                         const int *__restrict__ pstatus,
                                                                         int *__restrict__ owner,
                                                                         const int *__restrict__ dcount = nullptr) {
    __shared__ unsigned long long key[TABLE_SHARE_SMALL];
    __shared__ int okw[TABLE_SHARE_SMALL], own[TABLE_SHARE_SMALL], elo[TABLE_SHARE_SMALL], ehi[TABLE_SHARE_SMALL];
    if (dcount) cnt = min(cnt, *dcount);
    const int w = threadIdx.x;
    if (w < cnt) {
        const double *oc = oconst + OC_N * (int64_t)w;
        key[w] = (unsigned long long)__double_as_longlong(oc[OC_KAPPA]);
        okw[w] = pstatus[w] == PLK_POINT_OK;
        elo[w] = (int)oc[OC_ELO];
        ehi[w] = (int)oc[OC_EHI];
    }
    __syncthreads();
    int b = w;
    if (w < cnt && okw[w])
        for (int v = 0; v < w; ++v)
            if (okw[v] && key[v] == key[w]) {
                b = v;
                break;
            }
    if (w < cnt) {
        own[w] = b;
        owner[w] = b;
    }
    __syncthreads();
    if (w < cnt && own[w] == w) {
        int lo = elo[w], hi = ehi[w];
        for (int v = w + 1; v < cnt; ++v)
            if (own[v] == w) {
                lo = min(lo, elo[v]);
                hi = max(hi, ehi[v]);
            }
        oconst[OC_N * (int64_t)w + OC_ELO] = lo;
        oconst[OC_N * (int64_t)w + OC_EHI] = hi;
    }
}

__global__ void __launch_bounds__(256) k_table_union(int cnt, double *__restrict__ oconst, const int *__restrict__ owner,
                                                     const int *__restrict__ dcount = nullptr) {
    const int w = blockIdx.x;
    if (dcount) cnt = min(cnt, *dcount);
    if (w >= cnt || owner[w] != w) return;
    __shared__ int sl[8], sh[8];
    int lo = (int)oconst[OC_N * (int64_t)w + OC_ELO], hi = (int)oconst[OC_N * (int64_t)w + OC_EHI];
    for (int v = w + 1 + threadIdx.x; v < cnt; v += blockDim.x)
        if (owner[v] == w) {
            lo = min(lo, (int)oconst[OC_N * (int64_t)v + OC_ELO]);
            hi = max(hi, (int)oconst[OC_N * (int64_t)v + OC_EHI]);
        }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        sl[threadIdx.x >> 5] = lo;
        sh[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
            lo = min(lo, sl[i]);
            hi = max(hi, sh[i]);
        }
        oconst[OC_N * (int64_t)w + OC_ELO] = lo;
        oconst[OC_N * (int64_t)w + OC_EHI] = hi;
    }
}

// ---------------------------------------------------------------------------
// Double-float (FP32 pair) arithmetic for the first pass's table
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum_f(float a, float b, float &s, float &e) {   // |a| >= |b| or a = 0
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ph, pl) <- (ph, pl) * (th, tl) + (ch, cl), dropping pl * tl
__device__ __forceinline__ void df_horner_step(float &ph, float &pl, float th, float tl, float ch, float cl) {
    const float x = __fmul_rn(ph, th);
    float ex = __fmaf_rn(ph, th, -x);
    ex = __fmaf_rn(ph, tl, ex);
    ex = __fmaf_rn(pl, th, ex);
    float s, es;
    two_sum_f(x, ch, s, es);
    ph = s;
    pl = __fadd_rn(__fadd_rn(es, ex), cl);
}

// ln 2 in three parts: 16 significant bits (k LN2_HI is exact for |k| < 2^8),
// then two FP32 parts of the remainder (from the double ln 2, ~2^-54 relative)
constexpr double LN2_D = 0.69314718055994530942;
constexpr float LN2_HI = 45426.0f / 65536.0f;
constexpr float LN2_MID = (float)(LN2_D - (double)LN2_HI);
constexpr float LN2_LO = (float)(LN2_D - (double)LN2_HI - (double)LN2_MID);
// 1 / n! as double-float, n = 2..4 (the higher terms need only FP32)
constexpr float IF2 = 0.5f;
constexpr float IF3H = (float)(1.0 / 6.0), IF3L = (float)(1.0 / 6.0 - (double)IF3H);
constexpr float IF4H = (float)(1.0 / 24.0), IF4L = (float)(1.0 / 24.0 - (double)IF4H);

// exp(x) for the double-float x = xh + xl, |x| <= 86 (0 below -86): relative
// error ~2^-45 for x >= -50 (below, the low part of the result leaves the
// FP32 normal range; such terms are far below the sums they enter).
// x = k ln2 + r with k = rint(x / ln2), |r| <= ln2 / 2 formed from the
// three-part ln 2 (k ln2_hi exact, k ln2_mid split exactly); exp(r) =
// p(r / 4)^4 with p the Taylor polynomial of degree 9 (remainder
// (ln2 / 8)^10 / 10! < 2^-56): terms 5..9 by Horner in FP32 (each below 2^-22,
// so their rounding stays below 2^-46), terms 0..4 in double-float; two
// double-float squarings; then 2^k.
__device__ __forceinline__ void df_exp(float xh, float xl, float &yh, float &yl) {
    if (xh != xh) {
        yh = xh;
        yl = 0.0f;
        return;
    }
    if (xh < -86.0f) {
        yh = yl = 0.0f;
        return;
    }
    if (xh > 86.0f) {
        yh = INFINITY;
        yl = 0.0f;
        return;
    }
    const float kf = rintf(__fmul_rn(xh, 1.44269504088896341f));
    const float t = __fmaf_rn(-kf, LN2_HI, xh);   // exact
    const float p = __fmul_rn(kf, LN2_MID);
    const float pe = __fmaf_rn(kf, LN2_MID, -p);  // k ln2_mid = p + pe
    float s, e, s2, e2;
    two_sum_f(t, -p, s, e);
    two_sum_f(s, xl, s2, e2);   // xl (up to 2^-24 |x|) joins exactly
    e = __fsub_rn(__fadd_rn(e, e2), __fmaf_rn(kf, LN2_LO, pe));
    float rh, rl;
    two_sum_f(s2, e, rh, rl);
    rh *= 0.25f;
    rl *= 0.25f;
    float q = 1.0f / 362880.0f;                 // 1/9!
    q = __fmaf_rn(q, rh, 1.0f / 40320.0f);
    q = __fmaf_rn(q, rh, 1.0f / 5040.0f);
    q = __fmaf_rn(q, rh, 1.0f / 720.0f);
    q = __fmaf_rn(q, rh, 1.0f / 120.0f);
    float ph = q, pl = 0.0f;
    df_horner_step(ph, pl, rh, rl, IF4H, IF4L);
    df_horner_step(ph, pl, rh, rl, IF3H, IF3L);
    df_horner_step(ph, pl, rh, rl, IF2, 0.0f);
    df_horner_step(ph, pl, rh, rl, 1.0f, 0.0f);
    df_horner_step(ph, pl, rh, rl, 1.0f, 0.0f);
    fast_two_sum_f(ph, pl, ph, pl);
#pragma unroll
    for (int i = 0; i < 2; ++i) {   // square
        const float x = __fmul_rn(ph, ph);
        float ex = __fmaf_rn(ph, ph, -x);
        ex = __fmaf_rn(2.0f * ph, pl, ex);
        fast_two_sum_f(x, ex, ph, pl);
    }
    const float sc = __int_as_float(((int)kf + 127) << 23);   // 2^k, k in [-125, 125]
    yh = ph * sc;
    yl = pl * sc;
}

// 1 / a for a double-float a > 0: FP32 reciprocal y, then y + y (1 - a y) with
// the residual formed to ~2^-47 (a_hi y split exactly)
__device__ __forceinline__ void df_recip(float ah, float al, float &yh, float &yl) {
    const float y = __frcp_rn(ah);
    const float p = __fmul_rn(ah, y);
    const float pe = __fmaf_rn(ah, y, -p);
    const float r = __fsub_rn(__fsub_rn(1.0f, p), __fmaf_rn(al, y, pe));   // 1 - p is exact
    fast_two_sum_f(y, __fmul_rn(y, r), yh, yl);
}
// (ah, al) * (bh, bl), dropping al bl, normalised
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &ph, float &pl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum_f(p, e, ph, pl);
}
constexpr float IF5H = (float)(1.0 / 120.0), IF5L = (float)(1.0 / 120.0 - (double)IF5H);
constexpr float IF7H = (float)(1.0 / 5040.0), IF7L = (float)(1.0 / 5040.0 - (double)IF7H);

// 2 sinh^2(x) = cosh(2x) - 1 for an FP32 x >= 0 (x <= 43) as double-float,
// relative error ~2^-44.  x < 1/2: sinh x = x sum_n y^n / (2n+1)!, y = x^2
// (terms n >= 4 in FP32, each below 2^-26 relative; remainder y^8 / 17! <
// 2^-64); else (e^x - e^-x) / 2 with the double-float exp and reciprocal
// (no cancellation: e^-x <= 0.61 e^x).
__device__ __forceinline__ void df_e1(float x, float &eh, float &el) {
    float sh, sl;
    if (x < 0.5f) {
        const float yh = __fmul_rn(x, x), yl = __fmaf_rn(x, x, -yh);
        float q = 1.0f / 1307674368000.0f;        // 1/15!
        q = __fmaf_rn(q, yh, 1.0f / 6227020800.0f);   // 1/13!
        q = __fmaf_rn(q, yh, 1.0f / 39916800.0f);     // 1/11!
        q = __fmaf_rn(q, yh, 1.0f / 362880.0f);       // 1/9!
        float ph = q, pl = 0.0f;
        df_horner_step(ph, pl, yh, yl, IF7H, IF7L);
        df_horner_step(ph, pl, yh, yl, IF5H, IF5L);
        df_horner_step(ph, pl, yh, yl, IF3H, IF3L);
        df_horner_step(ph, pl, yh, yl, 1.0f, 0.0f);
        fast_two_sum_f(ph, pl, ph, pl);
        const float p = __fmul_rn(x, ph);
        fast_two_sum_f(p, __fmaf_rn(x, pl, __fmaf_rn(x, ph, -p)), sh, sl);
    } else {
        float Eh, El, Ih, Il;
        df_exp(x, 0.0f, Eh, El);
        df_recip(Eh, El, Ih, Il);
        float s, e;
        two_sum_f(Eh, -Ih, s, e);
        fast_two_sum_f(s, __fadd_rn(e, __fsub_rn(El, Il)), sh, sl);
        sh *= 0.5f;
        sl *= 0.5f;
    }
    df_mul(sh, sl, sh, sl, eh, el);
    eh *= 2.0f;
    el *= 2.0f;
}

// Trapezoid sum of the first pass's table in double-float arithmetic (its
// entries need ~2^-40; FP64 issues at 1/68 of FP32 on this part).  With the
// integrand written as cosh(kappa t) e^{-u (cosh t - 1)} =
// e^{a(t)} (1 + e^{-2 kappa t}) / 2, a(t) = kappa t - u (cosh t - 1):
//   fixed grid (u <= TAB_USPLIT): nodes t_k = k QH, cosh t_k - 1 staged in
//     E1f; the terms are scaled by e^{-A}, A the largest a(t_k) (an FP32 scan),
//     so that they stay in the FP32 range (a reaches 350 at kappa = 20);
//   adaptive (u > TAB_USPLIT): step h = the power of two at or below
//     min(0.1, 0.45 / sqrt(u)) (so that t_k = k h is exact), cosh t_k - 1 from
//     df_e1, A = 0 (a stays below kappa^2 / (2u) < 13).
// e^{-2 kappa t_k} = r^k by repeated double-float products.  Each a(t_k) carries
// ~2^-48 of the larger of its two parts (<= kappa t_k): ~1e-13 of rho at
// kappa <= 8.  The stopping rule is that of the FP64 evaluation.
// The trapezoid step: QH on the fixed grid (u <= TAB_USPLIT), else the power of
// two at or below min(0.1, 0.45 / sqrt(u)).
__device__ __forceinline__ float rho_df_step(float uh) {
    if (uh <= (float)TAB_USPLIT) return (float)QH;
    int ex;
    frexpf(fminf(0.1f, 0.45f * rsqrtf(uh)), &ex);   // value in [2^(ex-1), 2^ex)
    return __int_as_float((ex - 1 + 127) << 23);
}

// The scaled double-float trapezoid sum sum_k w_k e^{a(t_k) - A} (1 + r^k) of
// one node (u = uh + ul, kappa = kh + kl, step h), and its offset A.
// S > 1: the S consecutive lanes sub = 0 .. S - 1 of a group share one node;
// lane sub sums the terms k = 1 + sub, 1 + sub + S, ... (r^k from r^(1+sub)
// by products with r^S; the node t = 0 in lane 0), and the partial sums are
// added in a fixed order by shuffles (every lane of the warp takes part, so
// the caller calls this in all lanes, with any u in (0, TAB_USPLIT] in unused
// ones); A is the maximum over all nodes, reduced the same way (exact).  All S
// lanes return the same sum and A.
template <int S = 1>
__device__ __forceinline__ float2 rho_df_sum(float uh, float ul, float kh, float kl, float h,
                                             const float2 *__restrict__ E1f, int sub, float &A) {
    const bool fixed = uh <= (float)TAB_USPLIT;
    A = 0.0f;   // a(0) = 0
    if (fixed)
        for (int k = 1 + sub; k < QNODES; k += S) A = fmaxf(A, __fmaf_rn(-uh, E1f[k].x, kh * (float)k * h));
    if constexpr (S > 1) {
#pragma unroll
        for (int o = 1; o < S; o <<= 1) A = fmaxf(A, __shfl_xor_sync(0xffffffffu, A, o));
    }
    float rh, rl;   // r = e^{-2 kappa h}
    {
        const float t2 = __fmul_rn(-2.0f * kh, h), t2e = __fmaf_rn(-2.0f * kh, h, -t2);   // exact split
        df_exp(t2, __fmaf_rn(-2.0f * kl, h, t2e), rh, rl);
    }
    float sh = 0.0f, sl = 0.0f;   // sum: the node t = 0 (weight 1/2, term 2 e^{-A}) in lane 0
    if (sub == 0) df_exp(-A, 0.0f, sh, sl);
    float prev = sub == 0 ? 2.0f * sh : INFINITY;
    float qh = rh, ql = rl;   // r^k for this lane's next term k = 1 + sub (then + S per term)
    for (int i = 0; i < sub; ++i) df_mul(qh, ql, rh, rl, qh, ql);
    float sth = rh, stl = rl;   // r^S
    for (int i = 1; i < S; ++i) df_mul(sth, stl, rh, rl, sth, stl);
    const int kmax = fixed ? QNODES : 8192;
    bool stop = false;
    for (int k = 1 + sub; k < kmax && !stop; k += 4 * S) {
        float gh[4], gl[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            gh[i] = gl[i] = 0.0f;
            const int kk = k + i * S;
            if (kk >= kmax) continue;
            const float t = (float)kk * h;   // exact
            float e1h, e1l;
            if (fixed) {
                e1h = E1f[kk].x;
                e1l = E1f[kk].y;
            } else {
                df_e1(0.5f * t, e1h, e1l);
            }
            // a - A = kappa t - u e1 - A, each product split exactly
            const float kt = __fmul_rn(kh, t), kte = __fmaf_rn(kh, t, -kt);
            const float pr = __fmul_rn(uh, e1h);
            float pe = __fmaf_rn(uh, e1h, -pr);
            pe = __fmaf_rn(uh, e1l, pe);
            pe = __fmaf_rn(ul, e1h, pe);
            float s1, c1, s2, c2;
            two_sum_f(kt, -pr, s1, c1);
            two_sum_f(s1, -A, s2, c2);
            const float lo = __fadd_rn(__fadd_rn(c1, c2), __fsub_rn(__fmaf_rn(kl, t, kte), pe));
            float xh, xl;
            df_exp(s2, lo, xh, xl);
            float oh, ol;                      // 1 + r^kk
            two_sum_f(1.0f, qh, oh, ol);
            ol = __fadd_rn(ol, ql);
            df_mul(xh, xl, oh, ol, gh[i], gl[i]);
            df_mul(qh, ql, sth, stl, qh, ql);  // r^(kk + S)
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (stop || k + i * S >= kmax) {
                stop = true;
                continue;
            }
            float s, e;
            two_sum_f(sh, gh[i], s, e);
            fast_two_sum_f(s, __fadd_rn(e, __fadd_rn(sl, gl[i])), sh, sl);
            if (gh[i] < prev && gh[i] < 1e-18f * sh) stop = true;
            prev = gh[i];
        }
    }
    if constexpr (S > 1) {
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {   // lanes (sub, sub ^ o): lower sub first
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
            const bool low = (sub & o) == 0;
            const float ah = low ? sh : oh, al = low ? sl : ol, bh = low ? oh : sh, bl = low ? ol : sl;
            float s, e;
            two_sum_f(ah, bh, s, e);
            fast_two_sum_f(s, __fadd_rn(e, __fadd_rn(al, bl)), sh, sl);
        }
    }
    return make_float2(sh, sl);
}

// rho(u) = c_kappa u^kappa e^{-u} e^A (h / 2) sum (FP64 from here)
__device__ __forceinline__ double rho_df_finish(double u, double kap, double logc, float A, float h, float2 sum) {
    return exp(logc + kap * log(u) - u + (double)A) * (0.5 * (double)h * ((double)sum.x + (double)sum.y));
}

__device__ __forceinline__ double rho_df(double u, double kap, double logc, const float2 *__restrict__ E1f) {
    const float uh = __double2float_rn(u), ul = __double2float_rn(u - (double)uh);
    const float kh = __double2float_rn(kap), kl = __double2float_rn(kap - (double)kh);
    const float h = rho_df_step(uh);
    float A;
    const float2 sum = rho_df_sum<1>(uh, ul, kh, kl, h, E1f, 0, A);
    return rho_df_finish(u, kap, logc, A, h, sum);
}

#include "plk_quad_consts.inc"   // QUAD_E1, QUAD_E1F_HI/LO, QUAD_CT, QUAD_TM

// FP64 trapezoid sum of rho(u) / (c u^kappa e^{-u} h) at one table node,
// shared by the S consecutive lanes sub = 0 .. S - 1 of a group (the terms
// k = 1 + sub, 1 + sub + S, ...; the node t = 0, weight 1/2, in lane 0; each
// lane stops by the FP64 evaluation's rule on its own terms; the partial sums
// added in a fixed order by shuffles, so every lane of the group returns the
// same sum and every lane of the warp must call this).  Fixed grid t_k = k QH
// (u <= TAB_USPLIT: terms exp(log cosh(kappa t_k) - u (cosh t_k - 1)) from E1,
// L2), else the step h = min(0.1, 0.45 / sqrt(u)) with cosh(kappa t) e^{-u cosh t}
// written as e^{kappa t - u (cosh t - 1)} (1 + e^{-2 kappa t}) / 2 and
// e^{-2 kappa t_k} = r^k by products.  *h_out receives the step.
template <int S>
__device__ __forceinline__ double rho_fp64_sum(double u, double kap, const double *__restrict__ E1,
                                               const double *__restrict__ L2, int sub, double *h_out) {
    double sum = sub == 0 ? 0.5 : 0.0, prev = sub == 0 ? 1.0 : INFINITY;
    if (u <= TAB_USPLIT) {
        *h_out = QH;
        bool stop = false;
        for (int k = 1 + sub; k < QNODES && !stop; k += 4 * S) {
            double g[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int kk = k + i * S;
                g[i] = (kk < QNODES) ? exp(L2[kk] - u * E1[kk]) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (stop || k + i * S >= QNODES) {
                    stop = true;
                    continue;
                }
                sum += g[i];
                if (g[i] < prev && g[i] < 1e-18 * sum) stop = true;
                prev = g[i];
            }
        }
    } else {
        double h = 0.45 * rsqrt(u);
        if (h > 0.1) h = 0.1;
        *h_out = h;
        const double r = exp(-2.0 * kap * h);
        double rS = r, rk = r;   // r^S, r^(1 + sub)
        for (int i = 1; i < S; ++i) rS *= r;
        for (int i = 0; i < sub; ++i) rk *= r;
        for (int k = 1 + sub; k < 20000; k += S) {
            const double t = k * h;
            const double sh = sinh(0.5 * t);
            const double g = exp(kap * t - 0.69314718055994530942 - 2.0 * u * sh * sh) * (1.0 + rk);
            rk *= rS;
            sum += g;
            if (g < prev && g < 1e-18 * sum) break;
            prev = g;
        }
    }
    if constexpr (S > 1) {
#pragma unroll
        for (int o = 1; o < S; o <<= 1) {   // lanes (sub, sub ^ o): lower sub first
            const double other = __shfl_xor_sync(0xffffffffu, sum, o);
            sum = ((sub & o) == 0) ? sum + other : other + sum;
        }
    }
    return sum;
}



// Table builder: one block per BPB sub-intervals (buckets) of a slot's table,
// TAB_NC Chebyshev nodes each (BPB = 32 for the tiled paths; fewer for the
// fused small-n path, whose batches often share one table: more blocks per
// table).  F32TAB writes each sub-interval's coefficients as TAB_F32 floats
// instead of TAB_NC doubles: c_0..c_3 as double-float pairs, c_4..c_9 rounded
// to FP32 (the layout k_build_f32 reads; it fits in the same per-point
// region), and sums the trapezoid rules in double-float arithmetic.
// For u <= TAB_USPLIT the trapezoid nodes are the fixed grid t_k = k QH, whose
// cosh(t_k) - 1 (QUAD_E1, kappa-independent, correctly rounded constants) and
// log cosh(kappa t_k) are staged in shared memory, so one exp per node remains.
// SPLIT > 1 (double-float tables): SPLIT consecutive lanes per node share its
// trapezoid sum (rho_df_sum<SPLIT>); the FP64 steps around it (the node u,
// the final scaling, the Chebyshev fit) run in BPB x TAB_NC threads only, in
// separate phases, since an FP64 warp instruction costs the same issue time
// with one lane active as with 32.
template <bool F32TAB, int BPB = 32, int SPLIT = 1>
__global__ void __launch_bounds__(BPB * TAB_NC * SPLIT) k_matern_table(const double *__restrict__ oconst,
                                                               double *__restrict__ tab,
                                                               const int *__restrict__ owner,
                                                               const int *__restrict__ gate = nullptr,
                                                               const int *__restrict__ dcount = nullptr) {
    constexpr int NN = BPB * TAB_NC;   // nodes per block
    __shared__ double E1[F32TAB ? 1 : QNODES];   // FP64: cosh(t_k) - 1
    __shared__ double L2[F32TAB ? 1 : QNODES];   // FP64: log cosh(kappa t_k)
    __shared__ float2 E1f[F32TAB ? QNODES : 1];  // double-float: cosh(t_k) - 1
    __shared__ double F[NN];
    __shared__ double Ach[NN];                   // Chebyshev coefficients per bucket
    __shared__ double CT[TAB_NC * TAB_NC];       // cos(pi k (m + 1/2) / NC)
    __shared__ double TM[TAB_NC * TAB_NC];       // T_k(t) = sum_m TM[k][m] t^m
    __shared__ double Us[SPLIT > 1 ? NN : 1];    // SPLIT > 1: node u, then its sum, offset, step
    __shared__ float2 Ss[SPLIT > 1 && F32TAB ? NN : 1];
    __shared__ float As[SPLIT > 1 && F32TAB ? NN : 1];
    __shared__ double Sd[SPLIT > 1 && !F32TAB ? NN : 1], Hd[SPLIT > 1 && !F32TAB ? NN : 1];
    const int w = blockIdx.y;
    if (beyond(dcount, w)) return;        // past the device-side count of a compacted batch
    if (owner && owner[w] != w) return;   // this slot reads another slot's table (same kappa)
    if (gate && !gate[w]) return;         // gated pass: only the flagged slots
    const double *oc = oconst + OC_N * (int64_t)w;
    const double kap = oc[OC_KAPPA], logc = oc[OC_LOGC];
    const int elo = (int)oc[OC_ELO], ehi = (int)oc[OC_EHI];
    {   // this block's buckets: octaves TAB_ELO + BPB blockIdx.x / TAB_S .. + BPB / TAB_S - 1
        const int bx = (int)blockIdx.x;
        const int e0 = TAB_ELO + (bx * BPB) / TAB_S, e1 = TAB_ELO + (bx * BPB + BPB - 1) / TAB_S;
        if (e1 < elo || e0 >= ehi) return;   // none of them is read
    }
    const bool kap_ok = !(kap != kap) && kap > 0.0;
    for (int k = threadIdx.x; k < QNODES; k += blockDim.x) {
        if constexpr (F32TAB) {
            E1f[k] = make_float2(QUAD_E1F_HI[k], QUAD_E1F_LO[k]);
        } else {
            E1[k] = QUAD_E1[k];
            const double kt = kap * (k * QH);
            L2[k] = kt + log1p(exp(-2.0 * kt)) - 0.69314718055994530942;
        }
    }
    for (int t = threadIdx.x; t < TAB_NC * TAB_NC; t += blockDim.x) {
        CT[t] = QUAD_CT[t];
        TM[t] = (double)QUAD_TM[t];
    }
    // node nd = (bucket lb, Chebyshev node l): u = sqrt(w) at the node
    const int nd = threadIdx.x, lb = nd / TAB_NC, l = nd % TAB_NC;
    const int bucket = blockIdx.x * BPB + lb;
    const int eb = TAB_ELO + bucket / TAB_S;
    const bool used = nd < NN && bucket < TAB_NBUCKET && eb >= elo && eb < ehi;
    auto node_u = [&]() {
        const int e = TAB_ELO + bucket / TAB_S, j = bucket % TAB_S;
        const double tl = QUAD_CT[TAB_NC + l];   // cos(pi (l + 1/2) / NC): the Chebyshev node
        return sqrt(ldexp(1.0 + (j + 0.5 * (tl + 1.0)) / TAB_S, e));
    };
    if constexpr (SPLIT > 1) {
        if (nd < NN) Us[nd] = used ? node_u() : 1.0;   // unused: any u on the fixed grid
        __syncthreads();
        if (kap_ok) {   // block-uniform: every lane reaches the shuffles
            const int node = threadIdx.x / SPLIT, sub = threadIdx.x % SPLIT;
            const double u = Us[node];
            if constexpr (F32TAB) {
                const float uh = __double2float_rn(u), ul = __double2float_rn(u - (double)uh);
                const float kh = __double2float_rn(kap), kl = __double2float_rn(kap - (double)kh);
                float Av;
                const float2 sum = rho_df_sum<SPLIT>(uh, ul, kh, kl, rho_df_step(uh), E1f, sub, Av);
                if (sub == 0) {
                    Ss[node] = sum;
                    As[node] = Av;
                }
            } else {
                double h;
                const double sum = rho_fp64_sum<SPLIT>(u, kap, E1, L2, sub, &h);
                if (sub == 0) {
                    Sd[node] = sum;
                    Hd[node] = h;
                }
            }
        }
        __syncthreads();
        if (used) {
            const double u = Us[nd];
            if constexpr (F32TAB)
                F[nd] = kap_ok ? rho_df_finish(u, kap, logc, As[nd], rho_df_step(__double2float_rn(u)), Ss[nd]) : nan("");
            else
                F[nd] = kap_ok ? exp(logc + kap * log(u) - u) * (Hd[nd] * Sd[nd]) : nan("");
        }
    } else {
        __syncthreads();
        if (used) {
            const double u = node_u();
            double r;
            if (!kap_ok) {
                r = nan("");
            } else if (F32TAB) {
                r = rho_df(u, kap, logc, E1f);
            } else if (u <= TAB_USPLIT) {
                // the terms of four nodes are computed ahead (independent exps),
                // then added in order with the same stopping rule
                double sum = 0.5, prev = 1.0;
                bool stop = false;
                for (int k = 1; k < QNODES && !stop; k += 4) {
                    double g[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) g[i] = (k + i < QNODES) ? exp(L2[k + i] - u * E1[k + i]) : 0.0;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (stop || k + i >= QNODES) {
                            stop = true;
                            continue;
                        }
                        sum += g[i];
                        if (g[i] < prev && g[i] < 1e-18 * sum) stop = true;
                        prev = g[i];
                    }
                }
                r = exp(logc + kap * log(u) - u) * (QH * sum);
            } else {
                r = rho_integral(u, kap, logc);
            }
            F[nd] = r;
        }
    }
    __syncthreads();
    // Chebyshev coefficient a_l of the bucket's interpolant (thread l), then the
    // monomial coefficient c_l of t^l (thread l)
    if (used) {
        double s2 = 0.0;
        for (int m = 0; m < TAB_NC; ++m) s2 += F[lb * TAB_NC + m] * CT[l * TAB_NC + m];
        Ach[nd] = (l == 0 ? 1.0 : 2.0) * s2 / TAB_NC;
    }
    __syncthreads();
    if (used) {
        double c = 0.0;
        for (int k = 0; k < TAB_NC; ++k) c += Ach[lb * TAB_NC + k] * TM[k * TAB_NC + l];
        if (F32TAB) {
            float *dst = reinterpret_cast<float *>(tab + (int64_t)w * TAB_SIZE) + (int64_t)bucket * TAB_F32;
            if (l < TAB_DF) {
                const float h = __double2float_rn(c);
                dst[2 * l] = h;
                dst[2 * l + 1] = __double2float_rn(c - (double)h);
            } else {
                dst[TAB_DF + l] = __double2float_rn(c);
            }
            if (l == 0)
                for (int m = TAB_DF + TAB_NC; m < TAB_F32; ++m) dst[m] = 0.0f;
        } else {
            tab[(int64_t)w * TAB_SIZE + (int64_t)bucket * TAB_NC + l] = c;
        }
    }
}

// rho at w = u^2 from the table: exponent/mantissa bits give the sub-interval
// and an exact local variable t; Horner in t.
__device__ __forceinline__ double rho_table(const double *__restrict__ tab, double w, double kap,
                                            double logc, int elo, int ehi) {
    const int hi = __double2hiint(w);
    const int lo = __double2loint(w);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    if (e >= TAB_EHI) return 0.0;
    // below the table, or outside the octaves built for this point (the range
    // bounds every site pair, so this is a safety net): the integral itself
    if (e < elo || e >= ehi) return (w == 0.0) ? 1.0 : rho_integral(sqrt(w), kap, logc);
    const int j = (hi >> (20 - TAB_SB)) & (TAB_S - 1);
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // in [1, 2)
    const double t = fma(m, 2.0 * TAB_S, -(2.0 * TAB_S + 2.0 * j + 1.0));    // exact, in [-1, 1)
    const double *c = tab + ((e - TAB_ELO) * TAB_S + j) * TAB_NC;
    double r = __ldg(c + TAB_NC - 1);
#pragma unroll
    for (int k = TAB_NC - 2; k >= 0; --k) r = fma(r, t, __ldg(c + k));
    return r;
}

// ---------------------------------------------------------------------------
// Build of the bordered matrix tiles (Step 3 item 1)
// ---------------------------------------------------------------------------
// Double-float split of a double without FP64-pipe instructions: hi keeps the
// sign, exponent and top 23 mantissa bits (truncated), lo the remaining 29 bits
// rounded to 24 (hi + lo carries ~48 bits).  Values below 2^-100 become 0.
__device__ __forceinline__ void split_df_bits(double v, float &hi, float &lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((u >> 52) & 0x7ff) - 1023;
    const unsigned int sgn = (unsigned int)(u >> 63) << 31;
    if (e < -100 || e > 127) {   // (our values are in [-1e4, 1e4] or exactly 0)
        hi = (e > 127) ? __int_as_float(sgn | 0x7f800000u) : 0.0f;
        lo = 0.0f;
        return;
    }
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    hi = __int_as_float(sgn | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29));
    const float r = __uint2float_rn((unsigned int)(m & 0x1FFFFFFFull));   // remainder, units of 2^(e-52)
    const int es = e - 52;
    const float sc = (es < -126) ? 0.0f : __int_as_float((es + 127) << 23);
    lo = __int_as_float(__float_as_int(r * sc) | sgn);
}

template <bool DF>
__global__ void __launch_bounds__(256) k_build(int nb, int64_t n, int64_t n_pad, int q, int64_t tpo,
                                               double *__restrict__ tiles,
                                               const double *__restrict__ oconst,
                                               const double *__restrict__ coordT,
                                               const double *__restrict__ tab,
                                               const double *__restrict__ Bt, const int *__restrict__ owner,
                                               const int *__restrict__ dcount = nullptr) {
    const int w = blockIdx.y;
    if (beyond(dcount, w)) return;
    const int t = blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;
    double *T = tiles + ((int64_t)w * tpo + t) * NT;
    float *TH = reinterpret_cast<float *>(T);   // double-float planes (DF)
    float *TL = TH + NT;
    const int c = threadIdx.x & (TB - 1);
    const int r0 = threadIdx.x >> 7;
    const int64_t j = (int64_t)J * TB + c;
    auto put = [&](int r, double v) {
        if (DF) {
            float h, l;
            split_df_bits(v, h, l);
            TH[r * TB + c] = h;
            TL[r * TB + c] = l;
        } else {
            T[r * TB + c] = v;
        }
    };
    if (I == nb) {   // right-hand-side rows: B^T, zero beyond q rows / n columns
        for (int r = r0; r < TB; r += 2) {
            double v = 0.0;
            if (J < nb && r < q && j < n) v = Bt[(int64_t)r * n_pad + j];
            put(r, v);
        }
        return;
    }
    const double *oc = oconst + OC_N * (int64_t)w;
    const double nug = oc[OC_NUG], kap = oc[OC_KAPPA], logc = oc[OC_LOGC];
    const int ow = owner ? owner[w] : w;   // the table (and its octave range) of the slot that built it
    const int elo = (int)oconst[OC_N * (int64_t)ow + OC_ELO], ehi = (int)oconst[OC_N * (int64_t)ow + OC_EHI];
    const double *ca = coordT + (int64_t)w * 2 * n_pad;
    const double *cb = ca + n_pad;
    const double *tw = tab + (int64_t)ow * TAB_SIZE;
    const double aj = ca[j], bj = cb[j];
    for (int r = r0; r < TB; r += 2) {
        const int64_t i = (int64_t)I * TB + r;
        double v;
        if (i >= n || j >= n) {
            v = (i == j) ? 1.0 : 0.0;              // identity padding
        } else if (i == j) {
            v = 1.0 + nug;
        } else if (i < j) {
            v = 0.0;                               // upper part of a diagonal tile, unused
        } else {
            const double da = ca[i] - aj, db = cb[i] - bj;
            const double wv = fma(da, da, db * db);
            v = rho_table(tw, wv, kap, logc, elo, ehi);
        }
        put(r, v);
    }
}

// Double-float build for the first (5-slice) pass of the mixed path: the same
// tiles as k_build<true>, evaluated in FP32 pair arithmetic (FP32 issues at
// ~68x the FP64 rate here).  Per entry:
//   w = (a_i - a_j)^2 + (b_i - b_j)^2 from double-float coordinates (error-free
//       differences and squares, a positive sum: relative error ~2^-44);
//   sub-interval from the FP32 bits of w_hi, local variable t = t_hi + t_lo with
//       t_hi exact (fma of the mantissa) and t_lo = w_lo scaled by a power of 2;
//   Horner: c_9..c_4 in FP32 on t_hi (these terms are below ~1e-6 of rho),
//       c_3..c_0 in double-float on (t_hi, t_lo).
// Against the FP64 evaluation of the same polynomial the entries differ by
// ~1e-13 absolute, four orders below the 5-slice products' 2^-30 relative
// error.  Pairs outside the table's octaves take the FP64 integral (rare).
// (volatile: the load must not be moved ahead of the range checks that guard
// its address)
__device__ __forceinline__ void ldg_v8(const float *p, float (&v)[8]) {   // 32-byte aligned
    asm volatile("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
                 : "l"(p));
}

// One entry rho(w_ij) of the first pass's double-float build, sites i (row)
// and j (column) given by their double-float transformed coordinates:
//   w = (a_i - a_j)^2 + (b_i - b_j)^2 from double-float coordinates (error-free
//       differences and squares, a positive sum: relative error ~2^-44);
//   sub-interval from the FP32 bits of w_hi, local variable t = t_hi + t_lo with
//       t_hi exact (fma of the mantissa) and t_lo = w_lo scaled by a power of 2;
//   Horner: c_9..c_4 in FP32 on t_hi (these terms are below ~1e-6 of rho),
//       c_3..c_0 in double-float on (t_hi, t_lo).
// Pairs outside the table's octaves take the FP64 integral (rare).
__device__ __forceinline__ void rho_entry_df(float aih, float ail, float bih, float bil, float ajh, float ajl,
                                             float bjh, float bjl, const float *__restrict__ tf, int elo, int ehi,
                                             double kap, double logc, float &vh, float &vl) {
    vl = 0.0f;
    float s, e, dah, dal, dbh, dbl;
    two_sum_f(aih, -ajh, s, e);
    e = __fadd_rn(e, __fsub_rn(ail, ajl));
    two_sum_f(s, e, dah, dal);
    two_sum_f(bih, -bjh, s, e);
    e = __fadd_rn(e, __fsub_rn(bil, bjl));
    two_sum_f(s, e, dbh, dbl);
    const float p1 = __fmul_rn(dah, dah), p2 = __fmul_rn(dbh, dbh);
    float e1 = __fmaf_rn(dah, dah, -p1), e2 = __fmaf_rn(dbh, dbh, -p2);
    e1 = __fmaf_rn(dah + dah, dal, e1);
    e2 = __fmaf_rn(dbh + dbh, dbl, e2);
    two_sum_f(p1, p2, s, e);
    float wh, wl;
    fast_two_sum_f(s, __fadd_rn(e, __fadd_rn(e1, e2)), wh, wl);
    const unsigned bits = __float_as_uint(wh);
    const int ew = (int)(bits >> 23) - 127;   // w >= 0
    if (wh == 0.0f) {
        vh = 1.0f;                         // coincident sites
    } else if (ew >= TAB_EHI) {
        vh = 0.0f;
    } else if (ew < elo || ew >= ehi) {    // outside the octaves built for this point
        split_df_bits(rho_integral(sqrt((double)wh + (double)wl), kap, logc), vh, vl);
    } else {
        const int jb = (int)(bits >> (23 - TAB_SB)) & (TAB_S - 1);
        const float m = __uint_as_float((bits & 0x007fffffu) | 0x3f800000u);   // [1, 2)
        const float th = __fmaf_rn(m, 2.0f * TAB_S, -(float)(2 * TAB_S + 2 * jb + 1));   // exact
        const float tl = __fmul_rn(wl, __uint_as_float((unsigned)(127 + TAB_SB + 1 - ew) << 23));
        const float *cb = tf + ((ew - TAB_ELO) * TAB_S + jb) * TAB_F32;
        float q0[8], q1[8];
        ldg_v8(cb, q0);
        ldg_v8(cb + 8, q1);
        // c_9 .. c_4 in FP32
        float ph = __fmaf_rn(q1[5], th, q1[4]);
        ph = __fmaf_rn(ph, th, q1[3]);
        ph = __fmaf_rn(ph, th, q1[2]);
        ph = __fmaf_rn(ph, th, q1[1]);
        ph = __fmaf_rn(ph, th, q1[0]);
        float pl = 0.0f;
        // c_3 .. c_0 in double-float
        df_horner_step(ph, pl, th, tl, q0[6], q0[7]);
        df_horner_step(ph, pl, th, tl, q0[4], q0[5]);
        df_horner_step(ph, pl, th, tl, q0[2], q0[3]);
        df_horner_step(ph, pl, th, tl, q0[0], q0[1]);
        fast_two_sum_f(ph, pl, vh, vl);
    }
}

__global__ void __launch_bounds__(256) k_build_f32(int nb, int64_t n, int64_t n_pad, int q, int64_t tpo,
                                                   double *__restrict__ tiles,
                                                   const double *__restrict__ oconst,
                                                   const double *__restrict__ coordT,
                                                   const double *__restrict__ tab,
                                                   const double *__restrict__ Bt, const int *__restrict__ owner) {
    const int w = blockIdx.y;
    const int t = blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;
    double *T = tiles + ((int64_t)w * tpo + t) * NT;
    float *TH = reinterpret_cast<float *>(T);
    float *TL = TH + NT;
    const int c = threadIdx.x & (TB - 1);
    const int r0 = threadIdx.x >> 7;
    const int64_t j = (int64_t)J * TB + c;
    if (I == nb) {   // right-hand-side rows: B^T, zero beyond q rows / n columns
        for (int r = r0; r < TB; r += 2) {
            double v = 0.0;
            if (J < nb && r < q && j < n) v = Bt[(int64_t)r * n_pad + j];
            float h, l;
            split_df_bits(v, h, l);
            TH[r * TB + c] = h;
            TL[r * TB + c] = l;
        }
        return;
    }
    const double *oc = oconst + OC_N * (int64_t)w;
    const double nug = oc[OC_NUG], kap = oc[OC_KAPPA], logc = oc[OC_LOGC];
    const int ow = owner ? owner[w] : w;   // the table (and its octave range) of the slot that built it
    const int elo = (int)oconst[OC_N * (int64_t)ow + OC_ELO], ehi = (int)oconst[OC_N * (int64_t)ow + OC_EHI];
    float dgh, dgl;   // 1 + nu^2
    split_df_bits(1.0 + nug, dgh, dgl);
    const float *cf = reinterpret_cast<const float *>(coordT + (int64_t)w * 2 * n_pad);
    const float *tf = reinterpret_cast<const float *>(tab + (int64_t)ow * TAB_SIZE);
    const float ajh = cf[j], ajl = cf[n_pad + j], bjh = cf[2 * n_pad + j], bjl = cf[3 * n_pad + j];
    for (int r = r0; r < TB; r += 2) {
        const int64_t i = (int64_t)I * TB + r;
        float vh, vl = 0.0f;
        if (i >= n || j >= n) {
            vh = (i == j) ? 1.0f : 0.0f;           // identity padding
        } else if (i == j) {
            vh = dgh;
            vl = dgl;
        } else if (i < j) {
            vh = 0.0f;                             // upper part of a diagonal tile, unused
        } else {
            rho_entry_df(cf[i], cf[n_pad + i], cf[2 * n_pad + i], cf[3 * n_pad + i], ajh, ajl, bjh, bjl, tf, elo, ehi,
                         kap, logc, vh, vl);
        }
        TH[r * TB + c] = vh;
        TL[r * TB + c] = vl;
    }
}

// ---------------------------------------------------------------------------
// Diagonal tile: Cholesky, inverse of the factor, log-det (Step 3 item 2)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_potrf(int J, int64_t tpo, double *__restrict__ tiles,
                                               double *__restrict__ inv,
                                               double *__restrict__ logdet,
                                               int *__restrict__ pstatus, const int *__restrict__ dcount = nullptr) {
    extern __shared__ double sm[];
    double *P = sm;         // packed lower L
    double *Wp = sm + PK;   // packed lower L^-1
    __shared__ double s_ld;
    __shared__ int s_bad;
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (beyond(dcount, w)) return;
    double *T = tiles + ((int64_t)w * tpo + tile_index(J, J)) * NT;
    for (int e = tid; e < NT; e += 256) {
        const int r = e >> 7, c = e & (TB - 1);
        if (c <= r) P[pk(r, c)] = T[e];
    }
    if (tid == 0) {
        s_ld = 0.0;
        s_bad = 0;
    }
    __syncthreads();
    for (int j = 0; j < TB; ++j) {
        if (tid == 0) {
            const double d = P[pk(j, j)];
            if (!(d > 0.0)) {
                s_bad = 1;
                P[pk(j, j)] = nan("");
            } else {
                P[pk(j, j)] = sqrt(d);
                s_ld += log(d);
            }
        }
        __syncthreads();
        const double rl = 1.0 / P[pk(j, j)];
        for (int i = j + 1 + tid; i < TB; i += 256) P[pk(i, j)] *= rl;
        __syncthreads();
        for (int i = j + 1 + warp; i < TB; i += 8) {
            const double lij = P[pk(i, j)];
            const int bi = pk(i, 0);
            for (int k = j + 1 + lane; k <= i; k += 32) P[bi + k] -= lij * P[pk(k, j)];
        }
        __syncthreads();
    }
    // W = L^-1, row by row: W_ii = 1/L_ii, W_ij = -(sum_{k=j}^{i-1} L_ik W_kj) / L_ii
    for (int i = 0; i < TB; ++i) {
        const int bi = pk(i, 0);
        const double lii = P[bi + i];
        for (int jj = tid; jj <= i; jj += 256) {
            if (jj == i) {
                Wp[bi + i] = 1.0 / lii;
            } else {
                double s = 0.0;
                for (int k = jj; k < i; ++k) s = fma(P[bi + k], Wp[pk(k, jj)], s);
                Wp[bi + jj] = -s / lii;
            }
        }
        __syncthreads();
    }
    double *Wg = inv + (int64_t)w * NT;
    for (int e = tid; e < NT; e += 256) {
        const int r = e >> 7, c = e & (TB - 1);
        T[e] = (c <= r) ? P[pk(r, c)] : 0.0;
        Wg[e] = (c <= r) ? Wp[pk(r, c)] : 0.0;
    }
    if (tid == 0) {
        logdet[w] += s_ld;
        if (s_bad && pstatus[w] == PLK_POINT_OK) pstatus[w] = PLK_POINT_NOT_PD;
    }
}

// ---------------------------------------------------------------------------
// Panel solve (MODE 0: C = A B^T, B = L_JJ^-1, in place) and trailing update
// (MODE 1: C -= A B^T), FP64, 128 x 128 tiles, 8 x 8 outputs per thread
// (rows ty + 16 i, columns tx + 16 j).  RB < 8: only the first 16 RB rows of
// A and C (a tile of the right-hand-side row, whose rows from q on are zero
// in A: the skipped rows of C would stay as they are, zero or unchanged).
// ---------------------------------------------------------------------------
template <int MODE, int RB>
__device__ __forceinline__ void gemm_tile(const double *__restrict__ A, const double *__restrict__ B, double *C,
                                          double (*As)[TB + 2], double (*Bs)[TB + 2], int tid) {
    const int tx = tid & 15, ty = tid >> 4;
    double acc[RB][8];
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.0;
    for (int k0 = 0; k0 < TB; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            const int e = tid + 256 * l;
            const int r = e >> 4, kk = e & 15;
            if (l < RB) As[kk][r] = A[r * TB + k0 + kk];
            Bs[kk][r] = B[r * TB + k0 + kk];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[RB], b[8];
#pragma unroll
            for (int i = 0; i < RB; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) b[jj] = Bs[kk][tx + 16 * jj];
#pragma unroll
            for (int i = 0; i < RB; ++i)
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < RB; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int idx = (ty + 16 * i) * TB + tx + 16 * jj;
            if (MODE == 0)
                C[idx] = acc[i][jj];
            else
                C[idx] -= acc[i][jj];
        }
}

template <int MODE>
__global__ void __launch_bounds__(256, 1) k_gemm_nt(int J, int64_t tpo, double *tiles,
                                                    const double *__restrict__ inv, int nb, int q,
                                                    const int *__restrict__ dcount = nullptr) {
    __shared__ double As[16][TB + 2];
    __shared__ double Bs[16][TB + 2];
    const int w = blockIdx.y, t = blockIdx.x, tid = threadIdx.x;
    if (beyond(dcount, w)) return;
    double *base = tiles + (int64_t)w * tpo * NT;
    const double *A;
    const double *B;
    double *C;
    int I;
    if (MODE == 0) {
        I = J + 1 + t;
        C = base + tile_index(I, J) * NT;
        A = C;
        B = inv + (int64_t)w * NT;
    } else {
        int K;
        decode_trailing(t, J, I, K);
        A = base + tile_index(I, J) * NT;
        B = base + tile_index(K, J) * NT;
        C = base + tile_index(I, K) * NT;
    }
    if (I == nb && q <= 16)   // the right-hand-side row: q = M + p <= 64 non-zero rows
        gemm_tile<MODE, 1>(A, B, C, As, Bs, tid);
    else if (I == nb && q <= 32)
        gemm_tile<MODE, 2>(A, B, C, As, Bs, tid);
    else if (I == nb && q <= 64)
        gemm_tile<MODE, 4>(A, B, C, As, Bs, tid);
    else
        gemm_tile<MODE, 8>(A, B, C, As, Bs, tid);
}

// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(256, 1) k_gemm_nt(int J, int64_t tpo, double *tiles,
                                                    const double *__restrict__ inv, const int *__restrict__ dcount = nullptr) {
    __shared__ double As[16][TB + 2];
    __shared__ double Bs[16][TB + 2];
    const int w = blockIdx.y, t = blockIdx.x, tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (beyond(dcount, w)) return;
    double *base = tiles + (int64_t)w * tpo * NT;
    const double *A;
    const double *B;
    double *C;
    if (MODE == 0) {
        const int I = J + 1 + t;
        C = base + tile_index(I, J) * NT;
        A = C;
        B = inv + (int64_t)w * NT;
    } else {
        int I, K;
        decode_trailing(t, J, I, K);
        A = base + tile_index(I, J) * NT;
        B = base + tile_index(K, J) * NT;
        C = base + tile_index(I, K) * NT;
    }
    double acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.0;
    for (int k0 = 0; k0 < TB; k0 += 16) {
#pragma unroll
        for (int l = 0; l < 8; ++l) {
            const int e = tid + 256 * l;
            const int r = e >> 4, kk = e & 15;
            As[kk][r] = A[r * TB + k0 + kk];
            Bs[kk][r] = B[r * TB + k0 + kk];
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double a[8], b[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) b[jj] = Bs[kk][tx + 16 * jj];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fma(a[i], b[jj], acc[i][jj]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int idx = (ty + 16 * i) * TB + tx + 16 * jj;
            if (MODE == 0)
                C[idx] = acc[i][jj];
            else
                C[idx] -= acc[i][jj];
        }
}

// ---------------------------------------------------------------------------
// Closed form per omega (Step 3 items 5-8; eqs. betahat, 4, profile, remlpro)
// ---------------------------------------------------------------------------
__global__ void k_finalize(int count, int64_t k0, int M, int p, int64_t n, int nb, int reml,
                           int64_t tpo, const double *__restrict__ tiles,
                           const double *__restrict__ ldv, const int *__restrict__ pstatus,
                           const double *__restrict__ sumlogy, const double *__restrict__ lambdas,
                           double *logL, double *sigma2, double *beta, double *logdet,
                           double *ssq, int32_t *status, const int *__restrict__ out_index,
                           int32_t status_or, const int *__restrict__ gate, const int *__restrict__ dcount = nullptr,
                           double *__restrict__ err_zero = nullptr) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= count || beyond(dcount, w)) return;
    if (gate && !gate[w]) return;   // gated pass: only the flagged slots
    const int64_t k = out_index ? (int64_t)out_index[w] : k0 + w;
    const double *S = tiles + ((int64_t)w * tpo + tile_index(nb, nb)) * NT;   // -B^T V^-1 B
    int st = pstatus[w];
    const double NaN = nan("");
    // One thread per point: every FP64 instruction here holds its warp's
    // sub-partition pipe for 64 cycles whatever the active lanes, so the chain
    // is kept short: 1 / l_jj = rsqrt(d_jj) once per pivot, multiplications
    // instead of divisions, and log|X^T V^-1 X| = log of the pivots' product
    // (renormalised by frexp) instead of p logs.
    double Q[16 * 16];
    double il[16];   // 1 / l_jj
    double cv[16], bv[16];
    double ldx = NaN;
    if (st == PLK_POINT_OK) {
        for (int a = 0; a < p; ++a)
            for (int b = 0; b <= a; ++b) Q[a * p + b] = -S[(M + a) * TB + (M + b)];
        double prod = 1.0;
        int pex = 0;
        for (int jj = 0; jj < p && st == PLK_POINT_OK; ++jj) {
            double d = Q[jj * p + jj];
            for (int kk = 0; kk < jj; ++kk) d -= Q[jj * p + kk] * Q[jj * p + kk];
            if (!(d > 0.0)) {
                st = PLK_POINT_NOT_PD;
                break;
            }
            int e;
            prod = frexp(prod * d, &e);
            pex += e;
            const double r = rsqrt(d);
            il[jj] = r;
            Q[jj * p + jj] = d * r;
            for (int i = jj + 1; i < p; ++i) {
                double s = Q[i * p + jj];
                for (int kk = 0; kk < jj; ++kk) s -= Q[i * p + kk] * Q[jj * p + kk];
                Q[i * p + jj] = s * r;
            }
        }
        if (st == PLK_POINT_OK) ldx = log(prod) + (double)pex * 0.69314718055994530942;
    }
    const bool good = (st == PLK_POINT_OK);
    const double ld = good ? ldv[w] : NaN;
    const double two_pi_log = 1.8378770664093454836;   // log(2 pi)
    const double slog = *sumlogy;
    for (int m = 0; m < M; ++m) {
        double ll = NaN, s2 = NaN;
        if (good) {
            for (int a = 0; a < p; ++a) {
                double tt = -S[(M + a) * TB + m];
                for (int kk = 0; kk < a; ++kk) tt -= Q[a * p + kk] * cv[kk];
                cv[a] = tt * il[a];
            }
            double sbh = 0.0;
            for (int a = 0; a < p; ++a) sbh += cv[a] * cv[a];
            const double rss = -S[m * TB + m] - sbh;
            for (int a = p - 1; a >= 0; --a) {
                double tt = cv[a];
                for (int kk = a + 1; kk < p; ++kk) tt -= Q[kk * p + a] * bv[kk];
                bv[a] = tt * il[a];
            }
            const double jac = -2.0 * (lambdas[m] - 1.0) * slog;
            double m2;
            if (!reml) {
                s2 = rss / (double)n;
                m2 = (double)n * log(s2) + ld + jac + (double)n * two_pi_log + (double)n;
            } else {
                const double dof = (double)(n - p);
                s2 = rss / dof;
                m2 = dof * log(s2) + ld + ldx + jac + (double)n * two_pi_log + dof;
            }
            if (!(rss > 0.0)) {
                st = PLK_POINT_RSS_NONPOS;
                m2 = NaN;
            }
            ll = -0.5 * m2;
        }
        if (logL) logL[k * M + m] = ll;
        if (sigma2) sigma2[k * M + m] = s2;
        if (beta)
            for (int a = 0; a < p; ++a) beta[(k * M + m) * p + a] = good ? bv[a] : NaN;
    }
    if (logdet) {
        logdet[2 * k] = ld;
        logdet[2 * k + 1] = good ? ldx : NaN;
    }
    if (ssq) {
        // Table 1 ssqYX = B^T V^-1 B, from the lower triangle of the tile
        const int q = M + p;
        double *o = ssq + k * q * q;
        for (int a = 0; a < q; ++a)
            for (int c = 0; c < q; ++c)
                o[a * q + c] = good ? -S[(a >= c ? a : c) * TB + (a >= c ? c : a)] : NaN;
    }
    if (status) status[k] = st | status_or;
    if (err_zero) err_zero[k] = 0.0;   // an FP64 re-evaluation: no bound to carry
}

// ---------------------------------------------------------------------------
// Profile reduction and likelihood CI (Section 3.6, eq. likelihood)
// ---------------------------------------------------------------------------
__global__ void k_profile_max(const double *__restrict__ vals, int64_t G, int64_t SM,
                              double *__restrict__ prof) {
    const int64_t g = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= G) return;
    double best = -INFINITY;
    int any = 0;
    for (int64_t j = lane; j < SM; j += 32) {
        const double v = vals[g * SM + j];
        if (v == v) {
            any = 1;
            best = fmax(best, v);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        any |= __shfl_xor_sync(0xffffffffu, any, o);
    }
    if (lane == 0) prof[g] = any ? best : nan("");
}

__global__ void k_profile_ci(const double *__restrict__ grid, const double *__restrict__ prof,
                             int64_t G, double half_q, double *__restrict__ out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t ib = -1;
    for (int64_t g = 0; g < G; ++g) {
        const double v = prof[g];
        if (v != v) continue;
        if (ib < 0 || v > prof[ib]) ib = g;
    }
    if (ib < 0) {
        out[0] = out[1] = out[2] = out[3] = nan("");
        return;
    }
    const double thr = prof[ib] - half_q;
    double lo = grid[0], hi = grid[G - 1];
    int cens = 0;
    int64_t in = ib;
    int64_t g = ib - 1;
    for (; g >= 0; --g) {
        const double v = prof[g];
        if (v != v) continue;
        if (v < thr) break;
        in = g;
    }
    if (g >= 0) {
        const double f = (thr - prof[g]) / (prof[in] - prof[g]);
        lo = grid[g] + f * (grid[in] - grid[g]);
    } else {
        cens |= 1;
    }
    in = ib;
    for (g = ib + 1; g < G; ++g) {
        const double v = prof[g];
        if (v != v) continue;
        if (v < thr) break;
        in = g;
    }
    if (g < G) {
        const double f = (thr - prof[g]) / (prof[in] - prof[g]);
        hi = grid[g] + f * (grid[in] - grid[g]);
    } else {
        cens |= 2;
    }
    out[0] = lo;
    out[1] = hi;
    out[2] = grid[ib];
    out[3] = (double)cens;
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
const char *kernel_class_name(int c) {
    static const char *names[KC_COUNT] = {"boxcox", "omega_prep", "matern_table", "build", "potrf",
                                          "panel_trsm", "trailing_gemm", "finalize", "profile", "convert",
                                          "potrf_mixed", "panel_split", "trailing_split", "panel_split7",
                                          "trailing_split7", "fused_small"};
    return (c >= 0 && c < KC_COUNT) ? names[c] : "";
}

#define TIMED(cls, launch)                  \
    do {                                    \
        if (timer) timer->begin(cls, s);    \
        launch;                             \
        if (timer) timer->end(cls, s);      \
    } while (0)

// blocks per tile pair of k_min_dist2: enough pairs x splits to reach ~148 blocks
static unsigned min_dist_split(int64_t nt) {
    const int64_t pairs = nt * (nt + 1) / 2;
    return pairs >= 148 ? 1u : pairs >= 74 ? 2u : pairs >= 37 ? 4u : 8u;
}

cudaError_t launch_boxcox(int64_t n, int64_t n_pad, int p, int M, const double *y, const double *X,
                          const double *coords, const double *lam, double *Bt, double *sumlogy, cudaStream_t s,
                          KernelTimer *timer) {
    const int64_t total = (int64_t)(M + p) * n_pad;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    const int64_t nt = (n + 127) / 128;
    cudaError_t e = cudaMemsetAsync(sumlogy + 1, 0x7f, sizeof(double), s);   // 0x7f7f.. ~ 1.4e306
    if (e != cudaSuccess) return e;
    const int split = (int)min_dist_split(nt);
    const int64_t grid = blocks + 1 + nt * (nt + 1) / 2 * split;
    TIMED(KC_BOXCOX, (k_dataset_front<<<(unsigned)grid, 256, 0, s>>>(blocks, split, n, n_pad, p, M, y, X, lam, Bt,
                                                                     coords, sumlogy)));
    return cudaGetLastError();
}

cudaError_t launch_front(const BatchArgs &b, cudaStream_t s, FrontMode mode, bool build) {
    const int cnt = b.count;
    KernelTimer *timer = b.timer;
    const int f32 = mode == FRONT_DF_FAST ? 1 : 0;
    TIMED(KC_PREP, (k_omega_prep<<<cnt, 256, 0, s>>>(b.params, b.n, b.n_pad, b.coords, b.sumlogy, b.oconst,
                                                      b.coordT, b.ldv, b.pstatus, f32, nullptr, b.dcount)));
    const dim3 tg((TAB_NBUCKET + 31) / 32, cnt), bg((unsigned)b.tpo, cnt);
    if (b.owner) {   // slots with the same kappa share one table
        if (cnt <= TABLE_SHARE_SMALL) {
            k_table_share_small<<<1, TABLE_SHARE_SMALL, 0, s>>>(cnt, b.oconst, b.pstatus, b.owner, b.dcount);
        } else {
            k_table_owner<<<cnt, 256, 0, s>>>(cnt, b.oconst, b.pstatus, b.owner, b.dcount);
            k_table_union<<<cnt, 256, 0, s>>>(cnt, b.oconst, b.owner, b.dcount);
        }
    }
    if (f32 && !build) {   // the fused path: tables spread over more blocks, 8 lanes per node
        const dim3 tg4((TAB_NBUCKET + 3) / 4, cnt);
        TIMED(KC_TABLE, (k_matern_table<true, 4, 8><<<tg4, 4 * TAB_NC * 8, 0, s>>>(b.oconst, b.tab, b.owner)));
    } else if (f32) {
        TIMED(KC_TABLE, (k_matern_table<true><<<tg, 320, 0, s>>>(b.oconst, b.tab, b.owner, nullptr, b.dcount)));
        if (build)
            TIMED(KC_BUILD, (k_build_f32<<<bg, 256, 0, s>>>(b.nb, b.n, b.n_pad, b.q, b.tpo, b.tiles, b.oconst,
                                                             b.coordT, b.tab, b.Bt, b.owner)));
    } else if (!build) {   // the fused path: tables spread over more blocks, 4 lanes per node
        const dim3 tg4((TAB_NBUCKET + 3) / 4, cnt);
        TIMED(KC_TABLE, (k_matern_table<false, 4, 4><<<tg4, 4 * TAB_NC * 4, 0, s>>>(b.oconst, b.tab, b.owner)));
    } else {
        TIMED(KC_TABLE, (k_matern_table<false><<<tg, 320, 0, s>>>(b.oconst, b.tab, b.owner, nullptr, b.dcount)));
        if (mode == FRONT_DF)
            TIMED(KC_BUILD, (k_build<true><<<bg, 256, 0, s>>>(b.nb, b.n, b.n_pad, b.q, b.tpo, b.tiles, b.oconst,
                                                               b.coordT, b.tab, b.Bt, b.owner, b.dcount)));
        else
            TIMED(KC_BUILD, (k_build<false><<<bg, 256, 0, s>>>(b.nb, b.n, b.n_pad, b.q, b.tpo, b.tiles, b.oconst,
                                                                b.coordT, b.tab, b.Bt, b.owner, b.dcount)));
    }
    return cudaGetLastError();
}

// Dense row-major V (both triangles) of every point of a batch from its data
// tiles: one block per lower tile (I, J), I < nb; df = tiles hold hi/lo planes.
__global__ void __launch_bounds__(256) k_tiles_to_dense(int nb, int64_t n, int64_t tpo, const double *__restrict__ tiles,
                                                        int df, double *__restrict__ V) {
    const int w = blockIdx.y;
    const int t = blockIdx.x;
    int I = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    while (I * (I + 1) / 2 > t) --I;
    const int J = t - I * (I + 1) / 2;
    const double *T = tiles + ((int64_t)w * tpo + t) * NT;
    const float *TH = reinterpret_cast<const float *>(T), *TL = TH + NT;
    double *Vw = V + (int64_t)w * n * n;
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        const int r = e >> 7, c = e & (TB - 1);
        const int64_t i = (int64_t)I * TB + r, j = (int64_t)J * TB + c;
        if (i >= n || j >= n || j > i) continue;
        const double v = df ? (double)TH[e] + (double)TL[e] : T[e];
        Vw[i * n + j] = v;
        Vw[j * n + i] = v;
    }
}

cudaError_t launch_covariance(const BatchArgs &b, FrontMode mode, double *min_dist2, double *V, cudaStream_t s) {
    const int64_t nt = (b.n + 127) / 128;
    cudaError_t e = cudaMemsetAsync(min_dist2, 0x7f, sizeof(double), s);   // 0x7f7f.. ~ 1.4e306
    if (e != cudaSuccess) return e;
    k_min_dist2<<<dim3((unsigned)(nt * (nt + 1) / 2), min_dist_split(nt)), 256, 0, s>>>(b.n, b.coords, min_dist2);
    if ((e = launch_front(b, s, mode)) != cudaSuccess) return e;
    const unsigned data_tiles = (unsigned)((int64_t)b.nb * (b.nb + 1) / 2);
    k_tiles_to_dense<<<dim3(data_tiles, b.count), 256, 0, s>>>(b.nb, b.n, b.tpo, b.tiles, mode == FRONT_FP64 ? 0 : 1,
                                                                V);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const BatchArgs &b, cudaStream_t s) {
    const int cnt = b.count;
    KernelTimer *timer = b.timer;
    TIMED(KC_FINAL, (k_finalize<<<(cnt + 63) / 64, 64, 0, s>>>(
                        cnt, b.k0, b.M, b.p, b.n, b.nb, b.reml, b.tpo, b.tiles, b.ldv, b.pstatus,
                        b.sumlogy, b.lambdas, b.logL, b.sigma2, b.beta, b.logdet, b.ssq, b.status, b.out_index,
                        b.status_or, nullptr, b.dcount)));
    return cudaGetLastError();
}

cudaError_t launch_fp64_batch(const BatchArgs &b, cudaStream_t s) {
    // per function and device; cheap to repeat
    cudaError_t e = cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * PK * sizeof(double)));
    if (e != cudaSuccess) return e;
    const int cnt = b.count;
    KernelTimer *timer = b.timer;
    if ((e = launch_front(b, s, FRONT_FP64)) != cudaSuccess) return e;
    for (int J = 0; J < b.nb; ++J) {
        TIMED(KC_POTRF, (k_potrf<<<cnt, 256, 2 * PK * sizeof(double), s>>>(J, b.tpo, b.tiles, b.inv,
                                                                            b.ldv, b.pstatus, b.dcount)));
        const int m = b.nb - J;   // tile rows below the diagonal, RHS row included
        TIMED(KC_TRSM, (k_gemm_nt<0><<<dim3(m, cnt), 256, 0, s>>>(J, b.tpo, b.tiles, b.inv, b.nb, b.q, b.dcount)));
        TIMED(KC_GEMM, (k_gemm_nt<1><<<dim3(m * (m + 1) / 2, cnt), 256, 0, s>>>(J, b.tpo, b.tiles, b.inv, b.nb, b.q,
                                                                                    b.dcount)));
    }
    return launch_finalize(b, s);
}

cudaError_t launch_profile_max(const double *vals, int64_t G, int64_t SM, double *prof,
                               cudaStream_t s) {
    const int wpb = 8;
    k_profile_max<<<(unsigned)((G + wpb - 1) / wpb), 32 * wpb, 0, s>>>(vals, G, SM, prof);
    return cudaGetLastError();
}

cudaError_t launch_profile_ci(const double *grid, const double *prof, int64_t G, double half_q,
                              double *out, cudaStream_t s) {
    k_profile_ci<<<1, 32, 0, s>>>(grid, prof, G, half_q, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused evaluation of small datasets: one CTA per point (Step 3 items 1-4)
// ---------------------------------------------------------------------------
// For n + q <= FUSED_MAX_R the whole bordered matrix [[V, 0], [B^T, 0]] of
// R = n + q rows fits in shared memory as a packed lower triangle (row i at
// i (i + 1) / 2), so one CTA builds it (V from the point's rho table, exactly
// as k_build does, B^T from the Box-Cox rows), factors its first n columns
// right-looking in FP64 and leaves -B^T V^-1 B in its last q x q block: no
// 128-tile padding, no launch per tile step.  That block is written where the
// blocked path leaves it (the last diagonal tile of the point's tile array),
// so the same closed-form kernel finishes the point.  log|V| is the sum of the
// logs of the n pivots, reduced over the block.
// Threads per block (measured at n = 100: 256 -> 512 raised the FP64 kernel
// 3.9 %, 512 -> 768 the double-float kernel 1 %; more warps keep the four
// sub-partitions issuing between the per-column barriers)
constexpr int FUSED_THREADS = 512;      // FP64 kernel
constexpr int FUSED_DF_THREADS = 768;   // double-float kernel (dependent FP32 chains)

__global__ void __launch_bounds__(FUSED_THREADS, 1) k_fused_small(int64_t n, int64_t n_pad, int q, int nb, int64_t tpo,
                                                               double *__restrict__ tiles,
                                                               const double *__restrict__ oconst,
                                                               const double *__restrict__ coordT,
                                                               const double *__restrict__ tab,
                                                               const double *__restrict__ Bt,
                                                               const int *__restrict__ owner,
                                                               double *__restrict__ ldv, int *__restrict__ pstatus,
                                                               const int *__restrict__ gate) {
    extern __shared__ double A[];
    const int w = blockIdx.x;
    if (gate && !gate[w]) return;   // gated pass: only the flagged slots
    const int R = (int)n + q, nn = (int)n;
    const int64_t P = (int64_t)R * (R + 1) / 2;
    double *piv = A + P;   // the n pivots
    __shared__ int s_fail;
    __shared__ double red[FUSED_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = FUSED_THREADS / 32;
    if (pstatus[w] != PLK_POINT_OK) return;   // invalid parameters: the closed form writes NaN
    const double *oc = oconst + OC_N * (int64_t)w;
    const double nug = oc[OC_NUG], kap = oc[OC_KAPPA], logc = oc[OC_LOGC];
    const int ow = owner ? owner[w] : w;
    const int elo = (int)oconst[OC_N * (int64_t)ow + OC_ELO], ehi = (int)oconst[OC_N * (int64_t)ow + OC_EHI];
    const double *ca = coordT + (int64_t)w * 2 * n_pad;
    const double *cb = ca + n_pad;
    const double *tw = tab + (int64_t)ow * TAB_SIZE;
    // build: one warp per row, lanes along the row
    for (int i = warp; i < R; i += nw) {
        double *row = A + (int64_t)i * (i + 1) / 2;
        if (i < nn) {
            const double ai = ca[i], bi = cb[i];
            for (int k = lane; k <= i; k += 32) {
                double v;
                if (k == i) {
                    v = 1.0 + nug;
                } else {
                    const double da = ai - ca[k], db = bi - cb[k];
                    v = rho_table(tw, fma(da, da, db * db), kap, logc, elo, ehi);
                }
                row[k] = v;
            }
        } else {
            const double *br = Bt + (int64_t)(i - nn) * n_pad;
            for (int k = lane; k <= i; k += 32) row[k] = k < nn ? br[k] : 0.0;
        }
    }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    // Right-looking Cholesky of the first n columns, two per step: warp 0
    // factors columns j and j + 1 (pivot, scale, column j applied to column
    // j + 1, pivot, scale) while the block waits, then every warp applies both
    // columns to the rows and columns beyond them (each entry's two updates in
    // column order, as a column-by-column factorisation would).  FP64 issues
    // at 0.5 DFMA per clock per SM sub-partition here, so a look-ahead (warp 0
    // factoring the next pair beside the others' update) gains nothing: its
    // dependent chain waits behind its partner warp's FMAs (measured slower).
    auto col = [&](int r, int c) -> double & { return A[(int64_t)r * (r + 1) / 2 + c]; };
    for (int j = 0; j < nn; j += 2) {
        const bool two = j + 1 < nn;
        if (warp == 0) {
            bool bad = false;
            for (int c = j; c <= (two ? j + 1 : j) && !bad; ++c) {
                if (c > j) {
                    // column j applied to column j + 1 (rows j + 1 ..): needs L_{j+1,j}
                    __syncwarp();
                    const double l1 = col(j + 1, j);
                    for (int i = j + 1 + lane; i < R; i += 32) col(i, j + 1) = fma(-col(i, j), l1, col(i, j + 1));
                    __syncwarp();
                }
                const double d = col(c, c);
                const bool ok = d > 0.0;
                // 1 / sqrt(d): FP32 estimate and two Newton steps in FP64 (from
                // ~2^-23 to full precision), or FP64 sqrt and division where d
                // is outside the FP32 range
                double r = 0.0;
                if (ok && d > 1e-30 && d < 1e30) {
                    r = (double)rsqrtf((float)d);
                    r = r * fma(-0.5 * d, r * r, 1.5);
                    r = r * fma(-0.5 * d, r * r, 1.5);
                } else if (ok) {
                    r = 1.0 / sqrt(d);
                }
                __syncwarp();
                if (lane == 0) {
                    piv[c] = d;
                    if (ok) col(c, c) = d * r;
                    else s_fail = 1;
                }
                bad = !ok;
                if (ok)
                    for (int i = c + 1 + lane; i < R; i += 32) col(i, c) *= r;
            }
        }
        __syncthreads();
        if (s_fail) break;
        const int k0 = two ? j + 2 : j + 1;
        for (int i = k0 + warp; i < R; i += nw) {
            double *row = A + (int64_t)i * (i + 1) / 2;
            const double a0 = row[j];
            if (two) {
                const double a1 = row[j + 1];
                for (int k = k0 + lane; k <= i; k += 32) {
                    const double *rk = A + (int64_t)k * (k + 1) / 2 + j;
                    row[k] = fma(-a1, rk[1], fma(-a0, rk[0], row[k]));
                }
            } else {
                for (int k = k0 + lane; k <= i; k += 32) row[k] = fma(-a0, col(k, j), row[k]);
            }
        }
        __syncthreads();
    }
    if (s_fail) {
        if (tid == 0) pstatus[w] = PLK_POINT_NOT_PD;
        return;
    }
    double ls = 0.0;
    for (int j = tid; j < nn; j += FUSED_THREADS) ls += log(piv[j]);
    for (int o = 16; o > 0; o >>= 1) ls += __shfl_xor_sync(0xffffffffu, ls, o);
    if (lane == 0) red[warp] = ls;
    // -B^T V^-1 B into the last diagonal tile, lower triangle
    double *S = tiles + ((int64_t)w * tpo + tile_index(nb, nb)) * NT;
    for (int e = tid; e < q * q; e += FUSED_THREADS) {
        const int a = e / q, c = e - a * q;
        if (c <= a) S[a * TB + c] = A[(int64_t)(nn + a) * (nn + a + 1) / 2 + nn + c];
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += red[k];
        ldv[w] = t;
    }
}

// The same fused evaluation in double-float FP32 arithmetic (two floats per
// value, ~2^-44 per operation; FP32 issues at ~68x the FP64 rate here), for
// the mixed precision: V from the first pass's double-float build of each
// entry (rho_entry_df on the double-float table), the L D L^T elimination of
// the bordered matrix in double-float, log|V| and sum 1/d_j of the pivots in FP64.
// A point whose a-posteriori bound FUSED_DF_EPS (1 + nu^2) sum 1/d_j exceeds
// the tolerance, or whose factorisation fails, is evaluated again by
// k_fused_small in FP64.
__device__ __forceinline__ void df_mul_f(float ah, float al, float bh, float bl, float &ph, float &pl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, e);
    e = __fmaf_rn(al, bh, e);
    fast_two_sum_f(p, e, ph, pl);
}
// a - x0 y0 - x1 y1 (x1 = y1 = 0 for one product), normalised
__device__ __forceinline__ float2 df_sub2(float2 a, float2 x0, float2 y0, float2 x1, float2 y1) {
    const float p0 = __fmul_rn(x0.x, y0.x), p1 = __fmul_rn(x1.x, y1.x);
    float e0 = __fmaf_rn(x0.x, y0.x, -p0), e1 = __fmaf_rn(x1.x, y1.x, -p1);
    e0 = __fmaf_rn(x0.x, y0.y, __fmaf_rn(x0.y, y0.x, e0));
    e1 = __fmaf_rn(x1.x, y1.y, __fmaf_rn(x1.y, y1.x, e1));
    float s, t, s2, t2;
    two_sum_f(a.x, -p0, s, t);
    two_sum_f(s, -p1, s2, t2);
    const float lo = __fadd_rn(__fsub_rn(__fsub_rn(a.y, e0), e1), __fadd_rn(t, t2));
    float h, l;
    fast_two_sum_f(s2, lo, h, l);
    return make_float2(h, l);
}

// a - x y, normalised
__device__ __forceinline__ float2 df_sub1(float2 a, float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, __fmaf_rn(x.y, y.x, e));
    float s, t;
    two_sum_f(a.x, -p, s, t);
    float h, l;
    fast_two_sum_f(s, __fadd_rn(__fsub_rn(a.y, e), t), h, l);
    return make_float2(h, l);
}
// 1 / d in double-float for d > 0: FP32 reciprocal r0 and one Newton step
// r0 + r0 (1 - d r0), the residual formed in double-float (1 - d_hi r0 is
// exact by Sterbenz; ~2^-46 overall)
__device__ __forceinline__ float2 df_rcp_f(float2 d) {
    const float r0 = __frcp_rn(d.x);
    const float p = __fmul_rn(d.x, r0), pe = __fmaf_rn(d.x, r0, -p);
    const float res = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(d.y, r0));
    float h, l;
    fast_two_sum_f(r0, __fmul_rn(r0, res), h, l);
    return make_float2(h, l);
}

__global__ void __launch_bounds__(FUSED_DF_THREADS, 1) k_fused_small_df(int64_t n, int64_t n_pad, int q, int nb,
                                                                     int64_t tpo, double *__restrict__ tiles,
                                                                     const double *__restrict__ oconst,
                                                                     const double *__restrict__ coordT,
                                                                     const double *__restrict__ tab,
                                                                     const double *__restrict__ Bt,
                                                                     const int *__restrict__ owner,
                                                                     double *__restrict__ ldv, int *__restrict__ pstatus,
                                                                     double *__restrict__ invsum, int64_t k0,
                                                                     double eps, double tol, double *err_bound,
                                                                     int *__restrict__ flags) {
    extern __shared__ float2 Af[];
    const int w = blockIdx.x;
    const int R = (int)n + q, nn = (int)n;
    const int64_t P = (int64_t)R * (R + 1) / 2;
    float2 *pv = Af + P;   // the n pivots
    __shared__ double red[FUSED_DF_THREADS / 32], red2[FUSED_DF_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = FUSED_DF_THREADS / 32;
    // the a-posteriori bound E = eps (1 + nu^2) sum 1/d_j of each point and
    // its re-evaluation flag (E > tol or a failed factorisation), by thread 0
    auto verdict = [&](double isum, bool not_pd) {
        invsum[w] = isum;
        const double E = eps * (1.0 + oconst[OC_N * (int64_t)w + OC_NUG]) * isum;
        if (err_bound) err_bound[k0 + w] = E;
        flags[w] = (not_pd || (pstatus[w] == PLK_POINT_OK && !(E <= tol))) ? 1 : 0;
    };
    if (pstatus[w] != PLK_POINT_OK) {   // invalid parameters: the closed form writes NaN
        if (tid == 0) verdict(0.0, false);
        return;
    }
    const double *oc = oconst + OC_N * (int64_t)w;
    const double nug = oc[OC_NUG], kap = oc[OC_KAPPA], logc = oc[OC_LOGC];
    const int ow = owner ? owner[w] : w;
    const int elo = (int)oconst[OC_N * (int64_t)ow + OC_ELO], ehi = (int)oconst[OC_N * (int64_t)ow + OC_EHI];
    const float *cf = reinterpret_cast<const float *>(coordT + (int64_t)w * 2 * n_pad);
    const float *tf = reinterpret_cast<const float *>(tab + (int64_t)ow * TAB_SIZE);
    float dgh, dgl;   // 1 + nu^2
    split_df_bits(1.0 + nug, dgh, dgl);
    auto at = [&](int r, int c) -> float2 & { return Af[(int64_t)r * (r + 1) / 2 + c]; };
    for (int i = warp; i < R; i += nw) {
        float2 *row = Af + (int64_t)i * (i + 1) / 2;
        if (i < nn) {
            const float aih = cf[i], ail = cf[n_pad + i], bih = cf[2 * n_pad + i], bil = cf[3 * n_pad + i];
            for (int k = lane; k <= i; k += 32) {
                float vh = dgh, vl = dgl;
                if (k != i)
                    rho_entry_df(aih, ail, bih, bil, cf[k], cf[n_pad + k], cf[2 * n_pad + k], cf[3 * n_pad + k], tf,
                                 elo, ehi, kap, logc, vh, vl);
                row[k] = make_float2(vh, vl);
            }
        } else {
            const double *br = Bt + (int64_t)(i - nn) * n_pad;
            for (int k = lane; k <= i; k += 32) {
                float h, l;
                split_df_bits(k < nn ? br[k] : 0.0, h, l);
                row[k] = make_float2(h, l);
            }
        }
    }
    __syncthreads();
    // L D L^T elimination of the first n columns, right-looking, two columns
    // (c, c + 1) per step and no square roots.  The pivots d_c are the squares
    // of the Cholesky factor's diagonal and the last q x q block ends as
    // -B^T V^-1 B, all that the closed form needs (L itself is never formed).
    // Columns c and c + 1 are read from contiguous copies that the owners of
    // their rows wrote in the previous step.  Every thread forms the 2 x 2
    // pivot block itself (a few FP32 operations, identical in all threads):
    //   d_c, m = A(c+1, c) / d_c, d_{c+1} = A(c+1, c+1) - m A(c+1, c);
    // then (a) column c + 1 takes column c, A'(i, c+1) = A(i, c+1) - m A(i, c),
    // one row per thread, and (b) after a barrier every entry takes both,
    //   A(i, k) -= (A(i, c) / d_c) A(k, c) + (A'(i, c+1) / d_{c+1}) A'(k, c+1),
    // the right-looking Cholesky's two updates in order, in L D L^T form.  Two
    // barriers per two columns; no warp factors a panel while the others wait,
    // and a failed pivot ends the loop in all threads at the same step.
    float2 *cb = pv + nn;   // [cur c | cur c+1 | next c | next c+1 | A'(., c+1)], R entries each
    for (int k = tid; k < R; k += FUSED_DF_THREADS) {
        const float2 *rowk = Af + (int64_t)k * (k + 1) / 2;
        cb[k] = rowk[0];
        if (k >= 1) cb[R + k] = rowk[1];
    }
    __syncthreads();
    bool fail = false;
    auto bad = [](float2 d) { return !(d.x > 0.0f && d.x < INFINITY); };
    int par = 0;   // which pair of copies holds the current columns
    int c = 0;
    for (; c + 1 < nn; c += 2, par ^= 1) {
        const float2 *c0 = cb + (2 * par) * R, *c1 = c0 + R;
        float2 *n0 = cb + (2 * (par ^ 1)) * R, *n1 = n0 + R, *c1p = cb + 4 * R;
        const float2 d0 = c0[c];
        if (bad(d0)) {
            fail = true;
            break;
        }
        const float2 r0 = df_rcp_f(d0);
        float2 m;
        df_mul_f(c0[c + 1].x, c0[c + 1].y, r0.x, r0.y, m.x, m.y);
        const float2 d1 = df_sub1(c1[c + 1], m, c0[c + 1]);
        if (bad(d1)) {
            fail = true;
            break;
        }
        const float2 r1 = df_rcp_f(d1);
        if (tid == 0) {
            pv[c] = d0;
            pv[c + 1] = d1;
        }
        for (int i = c + 2 + tid; i < R; i += FUSED_DF_THREADS) c1p[i] = df_sub1(c1[i], m, c0[i]);
        __syncthreads();
        for (int i = c + 2 + warp; i < R; i += nw) {
            float2 *row = Af + (int64_t)i * (i + 1) / 2;
            float2 s0, s1;
            df_mul_f(c0[i].x, c0[i].y, r0.x, r0.y, s0.x, s0.y);
            df_mul_f(c1p[i].x, c1p[i].y, r1.x, r1.y, s1.x, s1.y);
            int k = c + 2 + lane;
            if (k <= i) {   // the first entry: column c + 2 or c + 3, copied for the next step
                const float2 v = df_sub2(row[k], s0, c0[k], s1, c1p[k]);
                row[k] = v;
                if (k == c + 2) n0[i] = v;
                else if (k == c + 3) n1[i] = v;
                k += 32;
            }
            for (; k + 32 <= i; k += 64) {   // two independent entries per iteration
                const float2 u = df_sub2(row[k], s0, c0[k], s1, c1p[k]);
                const float2 v = df_sub2(row[k + 32], s0, c0[k + 32], s1, c1p[k + 32]);
                row[k] = u;
                row[k + 32] = v;
            }
            if (k <= i) row[k] = df_sub2(row[k], s0, c0[k], s1, c1p[k]);
        }
        __syncthreads();
    }
    if (!fail && c < nn) {   // odd n: the last column alone
        const float2 *c0 = cb + (2 * par) * R;
        const float2 d0 = c0[c];
        if (bad(d0)) {
            fail = true;
        } else {
            const float2 r0 = df_rcp_f(d0);
            if (tid == 0) pv[c] = d0;
            for (int i = c + 1 + warp; i < R; i += nw) {
                float2 *row = Af + (int64_t)i * (i + 1) / 2;
                float2 s0;
                df_mul_f(c0[i].x, c0[i].y, r0.x, r0.y, s0.x, s0.y);
                for (int k = c + 1 + lane; k <= i; k += 32) row[k] = df_sub1(row[k], s0, c0[k]);
            }
            __syncthreads();
        }
    }
    if (fail) {
        if (tid == 0) {
            pstatus[w] = PLK_POINT_NOT_PD;
            verdict(0.0, true);
        }
        return;
    }
    double ls = 0.0, is = 0.0;
    for (int j = tid; j < nn; j += FUSED_DF_THREADS) {
        const double d = (double)pv[j].x + (double)pv[j].y;
        ls += log(d);
        is += 1.0 / d;
    }
    for (int o = 16; o > 0; o >>= 1) {
        ls += __shfl_xor_sync(0xffffffffu, ls, o);
        is += __shfl_xor_sync(0xffffffffu, is, o);
    }
    if (lane == 0) {
        red[warp] = ls;
        red2[warp] = is;
    }
    double *S = tiles + ((int64_t)w * tpo + tile_index(nb, nb)) * NT;
    for (int e = tid; e < q * q; e += FUSED_DF_THREADS) {
        const int a = e / q, c = e - a * q;
        if (c <= a) {
            const float2 v = at(nn + a, nn + c);
            S[a * TB + c] = (double)v.x + (double)v.y;
        }
    }
    __syncthreads();
    if (tid == 0) {
        double t = 0.0, t2 = 0.0;
        for (int k = 0; k < nw; ++k) {
            t += red[k];
            t2 += red2[k];
        }
        ldv[w] = t;
        verdict(t2, false);
    }
}

cudaError_t launch_fused_df_batch(const BatchArgs &b, double *invsum, double eps, double tol, double *err_bound,
                                  int *flags, cudaStream_t s) {
    const size_t smem = fused_smem_bytes(b.n, b.q);
    cudaError_t e = cudaFuncSetAttribute(k_fused_small_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    KernelTimer *timer = b.timer;
    if ((e = launch_front(b, s, FRONT_DF_FAST, false)) != cudaSuccess) return e;
    TIMED(KC_FUSED, (k_fused_small_df<<<b.count, FUSED_DF_THREADS, smem, s>>>(b.n, b.n_pad, b.q, b.nb, b.tpo, b.tiles,
                                                                          b.oconst, b.coordT, b.tab, b.Bt, b.owner,
                                                                          b.ldv, b.pstatus, invsum, b.k0, eps, tol,
                                                                          err_bound, flags)));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_finalize(b, s);
}

size_t fused_smem_bytes(int64_t n, int q) {   // packed matrix, n pivots, five column copies
    const int64_t R = n + q;
    return sizeof(double) * (size_t)(R * (R + 1) / 2 + n + 5 * R);
}

bool fused_applies(int64_t n, int q) { return n + q <= FUSED_MAX_R; }

cudaError_t launch_fused_batch(const BatchArgs &b, cudaStream_t s) {
    const size_t smem = fused_smem_bytes(b.n, b.q);
    cudaError_t e = cudaFuncSetAttribute(k_fused_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    KernelTimer *timer = b.timer;
    if ((e = launch_front(b, s, FRONT_FP64, false)) != cudaSuccess) return e;
    TIMED(KC_FUSED, (k_fused_small<<<b.count, FUSED_THREADS, smem, s>>>(b.n, b.n_pad, b.q, b.nb, b.tpo, b.tiles,
                                                                       b.oconst, b.coordT, b.tab, b.Bt, b.owner,
                                                                       b.ldv, b.pstatus, nullptr)));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    return launch_finalize(b, s);
}

// The FP64 fused evaluation of the slots flagged in gate[w] (set by the
// double-float pass's bound kernel), in place, with every kernel launched over
// the whole batch and exiting for the other slots: no host read-back, so the
// double-float pass and its re-evaluation form one asynchronous sequence (and
// can be captured in a graph).  Tables are per slot (no sharing by kappa).
cudaError_t launch_fused_fp64_gated(const BatchArgs &b, const int *gate, double *err_bound, cudaStream_t s) {
    const size_t smem = fused_smem_bytes(b.n, b.q);
    cudaError_t e = cudaFuncSetAttribute(k_fused_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    KernelTimer *timer = b.timer;
    const int cnt = b.count;
    const int32_t sor = PLK_POINT_RETRIED | PLK_POINT_FP64;
    TIMED(KC_PREP, (k_omega_prep<<<cnt, 256, 0, s>>>(b.params, b.n, b.n_pad, b.coords, b.sumlogy, b.oconst, b.coordT,
                                                      b.ldv, b.pstatus, 0, gate)));
    const dim3 tg4((TAB_NBUCKET + 3) / 4, cnt);
    TIMED(KC_TABLE, (k_matern_table<false, 4, 4><<<tg4, 4 * TAB_NC * 4, 0, s>>>(b.oconst, b.tab, nullptr, gate)));
    TIMED(KC_FUSED, (k_fused_small<<<cnt, FUSED_THREADS, smem, s>>>(b.n, b.n_pad, b.q, b.nb, b.tpo, b.tiles, b.oconst,
                                                                   b.coordT, b.tab, b.Bt, nullptr, b.ldv, b.pstatus,
                                                                   gate)));
    TIMED(KC_FINAL, (k_finalize<<<(cnt + 63) / 64, 64, 0, s>>>(cnt, b.k0, b.M, b.p, b.n, b.nb, b.reml, b.tpo, b.tiles,
                                                                b.ldv, b.pstatus, b.sumlogy, b.lambdas, b.logL,
                                                                b.sigma2, b.beta, b.logdet, b.ssq, b.status,
                                                                b.out_index, sor, gate, nullptr, err_bound)));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// self-test of the double-float exp (one thread per argument)
// ---------------------------------------------------------------------------
__global__ void k_df_exp_selftest(int64_t count, const float *__restrict__ xh, const float *__restrict__ xl,
                                  float *__restrict__ yh, float *__restrict__ yl) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float h, l;
    df_exp(xh[i], xl[i], h, l);
    yh[i] = h;
    yl[i] = l;
}

cudaError_t launch_df_exp_selftest(int64_t count, const float *xh, const float *xl, float *yh, float *yl,
                                   cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = (count + 255) / 256;
    k_df_exp_selftest<<<(unsigned)blocks, 256, 0, s>>>(count, xh, xl, yh, yl);
    return cudaGetLastError();
}

}  // namespace plk
