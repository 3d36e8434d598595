// plk_mixed.cu -- mixed-precision factorisation on the tcgen05 tensor cores.
//
// The blocked right-looking Cholesky of the bordered matrix (Section 3.3,
// Step 3 items 2-4) with
//   * the diagonal tile factorised in double-float FP32 (5 slices) or FP64
//     (7 slices), its inverse's off-diagonal blocks in double-float at 5 slices,
//   * the panel solve  L_IJ = A_IJ L_JJ^-T  and the trailing update
//     A_IK -= L_IJ L_KJ^T  computed as exact products of bf16 "slices",
//   * the trailing matrix held as double-float (two FP32 planes per tile).
//
// Split products (after Ozaki, Ogita, Oishi & Rump, "Error-free transformations
// of matrix multiplication", Numer. Algorithms 59 (2012)): each row r of an
// operand X is written as X_r = 2^(e_r - 7) sum_j m_j 2^(-8 j) with integers
// |m_j| <= 128 and max_k |X_rk| < 2^e_r.  Every m_j 2^(-8j) is exact in bf16, every
// product of two of them is exact in FP32, and the sum over a 128-deep tile of
// the products of one group g = i + j (at most 3 * 128 * 2^14 < 2^24 in units of
// 2^(-8g)) is an exact FP32 integer multiple -- so the tensor core's FP32
// accumulators hold the groups g = 0, 1, 2 exactly.  Groups g >= 3 share one
// accumulator (their rounding is 2^-24 of a term already 2^-24 below group 0).
// The product is 2^(eA + eB - 14) (P0 + P1 + P2 + P3).  S = 5 slices keep
// about 39 bits of every row, S = 7 about 55; the double-float epilogue keeps
// about 48.
#include <cuda.h>   // CUtensorMap (the driver function is looked up at run time)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "plk.h"
#include "plk_common.cuh"
#include "plk_kernels.cuh"
#include "plk_tc.cuh"

namespace plk {

namespace {

constexpr int SBLK = 16384;   // one 128-row x 64-element bf16 block, 128-byte swizzle
constexpr int HBLK = SBLK / 2;  // rows 0..63 or 64..127 of a block: 8 KB, contiguous
constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 128);

__device__ __forceinline__ float pow2f(int e) {   // exact 2^e (0 below the normal range)
    if (e < -126) return 0.0f;
    if (e > 127) e = 127;
    return __int_as_float((e + 127) << 23);
}

__device__ __forceinline__ int row_exp(float maxabs) {   // e with maxabs < 2^e
    if (!(maxabs > 0.0f)) return -100;
    int e;
    frexpf(maxabs, &e);
    return e < -100 ? -100 : (e > 120 ? 120 : e);
}

// error-free sum a + b = s + e
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += x, renormalised
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    e = __fadd_rn(e, lo);
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

// (acc_h, acc_l) += x y for double-float x, y (x_lo y_lo dropped; acc_l not
// renormalised until df_norm)
__device__ __forceinline__ void df_fma_acc(float &ah, float &al, float2 x, float2 y) {
    const float p = __fmul_rn(x.x, y.x);
    float e = __fmaf_rn(x.x, y.x, -p);
    e = __fmaf_rn(x.x, y.y, e);
    e = __fmaf_rn(x.y, y.x, e);
    float s, es;
    two_sum(ah, p, s, es);
    ah = s;
    al = __fadd_rn(al, __fadd_rn(es, e));
}
__device__ __forceinline__ float2 df_norm(float h, float l) {
    const float s = __fadd_rn(h, l);
    return make_float2(s, __fsub_rn(l, __fsub_rn(s, h)));
}
// (h, l) renormalised without assuming |h| >= |l| (after a cancellation)
__device__ __forceinline__ float2 df_renorm(float h, float l) {
    float s, e;
    two_sum(h, l, s, e);
    return make_float2(s, e);
}

// Arithmetic of the diagonal-tile Cholesky (one template, two number types).
// FP64 for the 7-slice tier (its products keep ~2^-46 of each entry, so the
// factor must be better than double-float); double-float FP32 pairs (~2^-44
// per operation) for the 5-slice pass, whose products are only good to 2^-30.
struct ArithF64 {
    using T = double;
    double v;   // rank-32 accumulator
    static __device__ __forceinline__ T load(float h, float l) { return (double)h + (double)l; }
    static __device__ __forceinline__ double value(T x) { return x; }
    static __device__ __forceinline__ T rsqrt_(T d) { return rsqrt(d); }
    static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
    static __device__ __forceinline__ T fms(T a, T x, T y) { return fma(-x, y, a); }   // a - x y
    static __device__ __forceinline__ T recip(T x) { return 1.0 / x; }
    static __device__ __forceinline__ T zero_value() { return 0.0; }
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void fma_acc(T x, T y) { v = fma(x, y, v); }
    __device__ __forceinline__ T sub_from(T p) const { return p - v; }
};
struct ArithDF {
    using T = float2;
    float h, l;   // rank-32 accumulator, l renormalised in sub_from
    static __device__ __forceinline__ T load(float hi, float lo) { return make_float2(hi, lo); }
    static __device__ __forceinline__ double value(T x) { return (double)x.x + (double)x.y; }
    // d^(-1/2): FP32 estimate y, then one Newton step y (1 + r / 2) with the
    // residual r = 1 - d y^2 formed to ~2^-46 (y^2 and d_hi y^2 split exactly;
    // 1 - t is exact for t within a factor 2 of 1).  Relative error ~1.5 (2^-22)^2.
    // d <= 0 gives NaN (or inf at 0) as in FP64.
    static __device__ __forceinline__ T rsqrt_(T d) {
        const float y = rsqrtf(d.x);
        const float p = __fmul_rn(y, y);
        const float pe = __fmaf_rn(y, y, -p);
        const float t = __fmul_rn(d.x, p);
        const float te = __fmaf_rn(d.x, p, -t);
        float r = __fsub_rn(1.0f, t);
        r = __fsub_rn(r, __fmaf_rn(d.x, pe, __fmaf_rn(d.y, p, te)));
        return df_norm(y, __fmul_rn(__fmul_rn(y, r), 0.5f));
    }
    static __device__ __forceinline__ T mul(T a, T b) {   // a_lo b_lo dropped
        const float p = __fmul_rn(a.x, b.x);
        float e = __fmaf_rn(a.x, b.x, -p);
        e = __fmaf_rn(a.x, b.y, e);
        e = __fmaf_rn(a.y, b.x, e);
        return df_norm(p, e);
    }
    static __device__ __forceinline__ T fms(T a, T x, T y) {   // a - x y (x_lo y_lo dropped)
        const float p = __fmul_rn(x.x, y.x);
        float e = __fmaf_rn(x.x, y.x, -p);
        e = __fmaf_rn(x.x, y.y, e);
        e = __fmaf_rn(x.y, y.x, e);
        float s, es;
        two_sum(a.x, -p, s, es);
        return df_renorm(s, __fadd_rn(es, __fsub_rn(a.y, e)));
    }
    // 1 / x: FP32 reciprocal y, then y + y r with r = 1 - x y formed to ~2^-47
    // (x_hi y split exactly; 1 - x_hi y exact); relative error ~2^-46
    static __device__ __forceinline__ T recip(T x) {
        const float y = __frcp_rn(x.x);
        const float p = __fmul_rn(x.x, y);
        const float pe = __fmaf_rn(x.x, y, -p);
        float r = __fsub_rn(1.0f, p);
        r = __fsub_rn(r, __fmaf_rn(x.y, y, pe));
        return df_norm(y, __fmul_rn(y, r));
    }
    static __device__ __forceinline__ T zero_value() { return make_float2(0.0f, 0.0f); }
    __device__ __forceinline__ void zero() { h = l = 0.0f; }
    __device__ __forceinline__ void fma_acc(T x, T y) { df_fma_acc(h, l, x, y); }
    __device__ __forceinline__ T sub_from(T p) const {
        float s, es;
        two_sum(p.x, -h, s, es);
        return df_renorm(s, __fadd_rn(es, __fsub_rn(p.y, l)));
    }
};

// The S slice values m_j 2^(-8j) of the double-float value (hi, lo) of a row with
// exponent e.
template <int S>
__device__ __forceinline__ void slice_df(float hi, float lo, int e, float (&m)[S]) {
    const float sc = pow2f(7 - e);
    float th = hi * sc, tl = lo * sc;
    if constexpr (S == 5) {
        // Digits 0-2 from the high part alone (r - rint(r) and the scaling by
        // 256 are exact, |r| <= 128); the low part then joins the residual
        // with one rounding (at most 2^-17 of a unit of digit 3, 1/256 of the
        // last digit's own truncation), and digits 3-4 follow.  Digits 0-2 stay
        // within +-128 (their groups are exact in the accumulators); digit 3
        // may reach +-192, still exact in bf16, and only enters groups >= 3,
        // which share a rounded accumulator anyway.
        float r = th;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const float mi = rintf(r);
            m[j] = mi * pow2f(-8 * j);
            r = __fmul_rn(__fsub_rn(r, mi), 256.0f);
        }
        r = __fmaf_rn(tl, 16777216.0f, r);   // + tl 2^24
        const float m3 = rintf(r);
        m[3] = m3 * pow2f(-24);
        m[4] = rintf(__fmul_rn(__fsub_rn(r, m3), 256.0f)) * pow2f(-32);
    } else {
#pragma unroll
        for (int j = 0; j < S; ++j) {
            const float mi = rintf(th);
            m[j] = mi * pow2f(-8 * j);
            const float r = __fsub_rn(th, mi);
            float s_, e_;
            two_sum(r, tl, s_, e_);
            th = s_ * 256.0f;
            tl = e_ * 256.0f;
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);   // exact: values are bf16-representable
    return *reinterpret_cast<uint32_t *>(&v);
}

// Global slice image of one 128 x 128 operand: S x 2 swizzled blocks (K halves)
// then 128 int row exponents.
template <int S>
__host__ __device__ constexpr size_t img_bytes() {
    return (size_t)S * 2 * SBLK + 1024;
}

// Panel slot of one tile row: four 5-slice images (panels J with J % 4 = 0 .. 3;
// the trailing update of the data triangle applies up to four panels at once)
// or one 7-slice image.
constexpr size_t SLOT = 4 * img_bytes<5>() > img_bytes<7>() ? 4 * img_bytes<5>() : img_bytes<7>();

// Exponent shared by every row and panel of L (data rows): |L_rk| <= sqrt(V_rr)
// = sqrt(1 + nu^2), with a margin for the rounding of the computed factor.
__device__ __forceinline__ int common_exp(double nug) {
    return row_exp((float)sqrt(1.0 + nug) * (1.0f + 1.0f / 1024.0f));
}

// Exponent shared by all data rows of a Schur complement (the trailing matrix
// before a panel solve): |S_ij| <= sqrt(S_ii S_jj) <= 1 + nu^2.  Slicing with it
// instead of each row's own maximum adds an absolute error of 2^-40 (1 + nu^2)
// per entry, far below what the earlier trailing updates already left there.
__device__ __forceinline__ int common_exp_schur(double nug) {
    return row_exp((float)(1.0 + nug) * (1.0f + 1.0f / 1024.0f));
}

template <int S>
__device__ __forceinline__ void store_pair(uint8_t *img, int r, int k, const float (&m0)[S], const float (&m1)[S]) {
    const int h = k >> 6;
    const uint32_t off = tc::sw128_offset(r, k & 63);
#pragma unroll
    for (int j = 0; j < S; ++j)
        *reinterpret_cast<uint32_t *>(img + (size_t)(j * 2 + h) * SBLK + off) = pack_bf16x2(m0[j], m1[j]);
}

__device__ __forceinline__ uint8_t *align1024(uint8_t *p) {
    return reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// Issue the S-slice split products of one K half into the four accumulators.
template <int S>
__device__ __forceinline__ void issue_split_mmas(uint32_t tb, const uint8_t *sA, const uint8_t *sB, bool first_half) {
    // B slices are back to back (128 rows each): two adjacent slices whose
    // groups both have their own accumulator (g + 1 <= 3) go in one MMA of
    // N = 256 into two adjacent accumulators; the rest add into accumulator
    // min(g, 3) with N = 128.
    const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sA)), b0 = tc::sdesc_sw128(tc::smem_u32(sB));
#pragma unroll
    for (int i = 0; i < S; ++i) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = a0 + (uint64_t)((i * SBLK + kk * 32) >> 4);
#pragma unroll
            for (int j = 0; i + j < S;) {
                const int g = i + j;
                const uint64_t bd = b0 + (uint64_t)((j * SBLK + kk * 32) >> 4);
                const uint32_t accumulate = (first_half && kk == 0 && i == 0 && j <= 3) ? 0u : 1u;
                if (g + 1 <= 3 && g + 1 < S) {
                    tc::mma_bf16(tb + g * 128, ad, bd, tc::idesc_bf16_f32(128, 256), accumulate);
                    j += 2;
                } else {
                    tc::mma_bf16(tb + (g < 3 ? g : 3) * 128, ad, bd, IDESC, accumulate);
                    j += 1;
                }
            }
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// double-float planes -> FP64 (the last diagonal tile, read by the closed form)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_tile_to_fp64(int64_t tpo, int64_t tile, double *tiles, const int *__restrict__ dcount = nullptr) {
    if (beyond(dcount, (int)blockIdx.x)) return;
    double *T = tiles + ((int64_t)blockIdx.x * tpo + tile) * NT;
    const float *H = reinterpret_cast<const float *>(T);
    const float *L = H + NT;
    double v[NT / 256];
#pragma unroll
    for (int l = 0; l < NT / 256; ++l) {
        const int e = threadIdx.x + 256 * l;
        v[l] = (double)H[e] + (double)L[e];
    }
    __syncthreads();
#pragma unroll
    for (int l = 0; l < NT / 256; ++l) T[threadIdx.x + 256 * l] = v[l];
}

// ---------------------------------------------------------------------------
// Diagonal tile in FP64: L_JJ, W = L_JJ^-1 (sliced for the tensor cores),
// log-det and the pivot sum for the error bound.
// ---------------------------------------------------------------------------
// Row of the t-th entry of a packed lower triangle (t = r (r + 1) / 2 + c, c <= r).
__device__ __forceinline__ int tri_row(int t) {
    int r = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    if ((r + 1) * (r + 2) / 2 <= t) ++r;
    if (r * (r + 1) / 2 > t) --r;
    return r;
}

// Dynamic shared memory of k_potrf_mixed: the packed tile (66 KB) and three
// 32 x 32 FP64 temporaries (24 KB); two blocks share an SM.
constexpr int DB = 32;   // block size of the diagonal-tile factorisation

// eps of the error bound E = eps (1 + nu^2) sum_j 1 / d_j: relative
// perturbation of the updated entries.  Calibrated on the n = 4000 workload
// against the FP64 path: with these values the bound exceeded the measured
// |Delta l_p| on every point (5 slices: by >= 3x; 7 slices with all groups
// exact: by >= 4.7x, on points whose own FP64 result differs from the CPU
// oracle by up to 1e-4).
__host__ __device__ constexpr double mixed_eps(int S) {
    return S == 7 ? 1.4210854715202004e-14 /* 2^-46 */ : 9.313225746154785e-10 /* 2^-30 */;
}
constexpr size_t POTRF_MIXED_SMEM = (size_t)(PK + 3 * DB * DB) * sizeof(double);

// Cholesky of the tile in the packed lower triangle P (number type Ar::T) in
// 32-column panels, two columns per block barrier: each of warps 0-3 forms the
// pair's pivots itself (1/sqrt(d_j), L_{j+1,j}, d_{j+1} and its 1/sqrt: the
// same operations in every thread), then one thread per row scales its entry
// of column j, applies it to column j + 1 and scales that -- a row's
// operations exactly as a column-by-column factorisation orders them -- and,
// after the barrier, thread 0 writes the pair's diagonal entries while the
// block applies both columns to the rest of the panel; then the panel's
// rank-32 update of the trailing lower triangle in 4 x 4 register tiles.  A
// non-positive pivot leaves NaN behind it; the pivot itself is kept (piv) for
// the status.
template <class Ar>
__device__ __forceinline__ void chol_tile(typename Ar::T *__restrict__ P, typename Ar::T *col,
                                          typename Ar::T *col2, double *piv, int tid) {
    using T = typename Ar::T;
    for (int kb = 0; kb < TB; kb += DB) {
        const int kend = kb + DB - 1;
        for (int j = kb; j <= kend; j += 2) {
            // warps 0-3 (one per SM sub-partition; 128 threads cover the <= 126
            // rows): the FP64 instance issues the pivots' square roots once per
            // sub-partition, not per warp
            T d, rl, cj1, d2, rl2;
            if (tid < 128) {
                d = P[pk(j, j)];
                rl = Ar::rsqrt_(d);
                cj1 = Ar::mul(P[pk(j + 1, j)], rl);   // L_{j+1,j}
                d2 = Ar::fms(P[pk(j + 1, j + 1)], cj1, cj1);
                rl2 = Ar::rsqrt_(d2);
                const int i = j + 2 + tid;              // this thread's row
                if (i < TB) {
                    const T v = Ar::mul(P[pk(i, j)], rl);
                    P[pk(i, j)] = v;
                    col[i] = v;
                    const T v2 = Ar::mul(Ar::fms(P[pk(i, j + 1)], v, cj1), rl2);
                    P[pk(i, j + 1)] = v2;
                    col2[i] = v2;
                }
            }
            __syncthreads();
            if (tid == 0) {   // every thread has read the pair's entries
                piv[j] = Ar::value(d);
                piv[j + 1] = Ar::value(d2);
                P[pk(j, j)] = Ar::mul(d, rl);
                P[pk(j + 1, j)] = cj1;
                P[pk(j + 1, j + 1)] = Ar::mul(d2, rl2);
            }
            const int nk = kend - j - 1;   // panel columns right of j + 1
            if (nk == 0) __syncthreads();   // no panel update follows: publish thread 0's writes
            if (nk > 0) {
                // rows j+2 .. kend (k <= i: a triangle), then rows below the panel (all nk columns)
                const int tri = nk * (nk + 1) / 2;
                const int total = tri + (TB - 1 - kend) * nk;
                for (int t = tid; t < total; t += 256) {
                    int i, k;
                    if (t < tri) {
                        const int ii = tri_row(t);
                        i = j + 2 + ii;
                        k = j + 2 + (t - ii * (ii + 1) / 2);
                    } else {
                        const int t2 = t - tri, q = t2 / nk;
                        i = kend + 1 + q;
                        k = j + 2 + (t2 - q * nk);
                    }
                    P[pk(i, k)] = Ar::fms(Ar::fms(P[pk(i, k)], col[i], col[k]), col2[i], col2[k]);
                }
                __syncthreads();
            }
        }
        const int m = TB - 1 - kend;   // rank-32 update of the trailing lower triangle
        if (m > 0) {
            const int nbl = m / 4, nblocks = nbl * (nbl + 1) / 2;
            for (int bq = tid; bq < nblocks; bq += 256) {
                const int bi = tri_row(bq), bk = bq - bi * (bi + 1) / 2;
                const int i0 = kend + 1 + 4 * bi, k0 = kend + 1 + 4 * bk;
                int ra[4], rb[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    ra[r] = pk(i0 + r, 0);
                    rb[r] = pk(k0 + r, 0);
                }
                Ar acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c].zero();
#pragma unroll 4
                for (int q = kb; q <= kend; ++q) {
                    T x[4], y[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        x[r] = P[ra[r] + q];
                        y[r] = P[rb[r] + q];
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int c = 0; c < 4; ++c) acc[r][c].fma_acc(x[r], y[c]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (k0 + c <= i0 + r) P[ra[r] + k0 + c] = acc[r][c].sub_from(P[ra[r] + k0 + c]);
            }
            __syncthreads();
        }
    }
}

// Inverses of the four 32 x 32 diagonal blocks of L in place (block b by warps
// 2b, 2b+1, named barrier 1 + b), right-looking by rows: row k of W is final
// once rows < k are applied; column k of L is staged a step ahead (dlc)
// because its slots become W's.  rd receives 1 / L_jj.
template <class Ar>
__device__ __forceinline__ void inv_diag_blocks(typename Ar::T *__restrict__ P, typename Ar::T *rd,
                                                typename Ar::T (*dcol)[2][DB], typename Ar::T (*dlc)[2][DB], int tid) {
    using T = typename Ar::T;
    const int warp = tid >> 5;
    if (tid < TB) rd[tid] = Ar::recip(P[pk(tid, tid)]);
    __syncthreads();
    const int b = warp >> 1, lt = tid & 63, base = DB * b;
    if (lt < DB) dlc[b][0][lt] = P[pk(base + lt, base)];
    if (lt == 0) {
        P[pk(base, base)] = rd[base];
        dcol[b][0][0] = rd[base];
    }
    tc::named_sync(1 + b, 64);
    for (int k = 0; k < DB - 1; ++k) {
        const T *ck = dcol[b][k & 1], *lk = dlc[b][k & 1];
        T *cn = dcol[b][(k + 1) & 1], *ln = dlc[b][(k + 1) & 1];
        const int ncol = k + 1, cnt = (DB - 1 - k) * ncol;
        if (lt > k + 1 && lt < DB) ln[lt] = P[pk(base + lt, base + k + 1)];
        const T rn = rd[base + k + 1];
        for (int t = lt; t < cnt; t += 64) {
            const int ii = t / ncol, c = t - ii * ncol, i = k + 1 + ii;
            const int e = pk(base + i, base + c);
            const T acc = (c == k) ? Ar::zero_value() : P[e];   // slot (i, k) still holds L[i][k]
            T v = Ar::fms(acc, lk[i], ck[c]);
            if (ii == 0) {
                v = Ar::mul(v, rn);
                cn[c] = v;
            }
            P[e] = v;
        }
        if (lt == 0) {
            P[pk(base + k + 1, base + k + 1)] = rn;
            cn[k + 1] = rn;
        }
        tc::named_sync(1 + b, 64);
    }
    __syncthreads();
}

// FP64 issues at 1/68 of FP32 on this part, so the 5-slice pass keeps FP64
// out of the bulk of the work and the kernel blocks what remains:
// - Cholesky (chol_tile) in double-float FP32 at 5 slices, in FP64 at 7;
// - W = L^-1 in place: the four 32 x 32 diagonal blocks are inverted at once
//   (two warps each, right-looking by rows: row k of W is final once rows < k
//   are applied; column k of L is staged a step ahead because its slots become
//   W's), then the off-diagonal blocks column by column from the right:
//   W_bc = -(sum_{d=c+1..b} W_bd L_dc) W_cc, the sums first (into temporaries,
//   while L_dc is still intact), then the products with W_cc over L_bc.
template <int S>
__global__ void __launch_bounds__(256, 2) k_potrf_mixed(int J, int64_t tpo, double *__restrict__ tiles,
                                                        uint8_t *__restrict__ wimg, double *__restrict__ logdet,
                                                        double *__restrict__ invsum, int *__restrict__ pstatus,
                                                        const double *__restrict__ oconst, int *__restrict__ doomed,
                                                        double tol, const int *__restrict__ dcount = nullptr) {
    extern __shared__ double sm[];
    double *P = sm;                   // packed lower triangle: the tile, then L, then W = L^-1
    double *Tm = sm + PK;             // 3 x 32 x 32 temporaries of the block inverse
    __shared__ double col[TB];        // scaled column j of L
    __shared__ double col2[TB];       // scaled column j + 1 of L
    __shared__ double piv[TB];        // pivots d_j
    __shared__ double rd[TB];         // 1 / L[j][j]
    __shared__ double dcol[4][2][DB];   // per diagonal block: finished row k of W
    __shared__ double dlc[4][2][DB];    // per diagonal block: column k of L, staged
    __shared__ double red[2][4];
    const int w = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (doomed && doomed[w]) return;   // already bound for the 7-slice tier
    if (beyond(dcount, w)) return;
    double *T = tiles + ((int64_t)w * tpo + tile_index(J, J)) * NT;
    const float *H = reinterpret_cast<const float *>(T);
    const float *Lo = H + NT;
    if constexpr (S == 5) {
        // double-float Cholesky
        float2 *P2 = reinterpret_cast<float2 *>(P);
        for (int e = tid; e < NT; e += 256) {
            const int r = e >> 7, c = e & (TB - 1);
            if (c <= r) P2[pk(r, c)] = ArithDF::load(H[e], Lo[e]);
        }
        __syncthreads();
        chol_tile<ArithDF>(P2, reinterpret_cast<float2 *>(col), reinterpret_cast<float2 *>(col2), piv, tid);
    } else {
        for (int e = tid; e < NT; e += 256) {
            const int r = e >> 7, c = e & (TB - 1);
            if (c <= r) P[pk(r, c)] = ArithF64::load(H[e], Lo[e]);
        }
        __syncthreads();
        chol_tile<ArithF64>(P, col, col2, piv, tid);
    }
    // ---- W = L^-1 in place
    if constexpr (S == 5)
        inv_diag_blocks<ArithDF>(reinterpret_cast<float2 *>(P), reinterpret_cast<float2 *>(rd),
                                 reinterpret_cast<float2(*)[2][DB]>(dcol), reinterpret_cast<float2(*)[2][DB]>(dlc), tid);
    else
        inv_diag_blocks<ArithF64>(P, rd, dcol, dlc, tid);
    if constexpr (S == 5) {
        // 5 slices keep ~40 bits of L_JJ^-1: the off-diagonal blocks of the
        // inverse (most of its work) run in double-float FP32 arithmetic
        // (~2^-46 per product, FP32 issues at 68x the FP64 rate)
        float2 *P2 = reinterpret_cast<float2 *>(P);
        float2 *Tm2 = reinterpret_cast<float2 *>(Tm);
        const float2 z2 = make_float2(0.0f, 0.0f);
        for (int c = 2; c >= 0; --c) {
            const int nres = 3 - c;
            for (int u = tid; u < nres * 64; u += 256) {   // sums: T_bc = sum_d W_bd L_dc
                const int b = c + 1 + u / 64, bl = u & 63;
                const int i0 = 4 * (bl >> 3), k0 = 4 * (bl & 7);
                float ah[4][4], al[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) ah[r][cc] = al[r][cc] = 0.0f;
                int ra[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) ra[r] = pk(DB * b + i0 + r, 0);
                for (int d = c + 1; d <= b; ++d) {
                    const bool diag = (d == b);
                    const int qend = diag ? i0 + 3 : DB - 1;
                    for (int q = 0; q <= qend; ++q) {
                        float2 x[4], y[4];
                        const int rq = pk(DB * d + q, 0) + DB * c + k0;
#pragma unroll
                        for (int r = 0; r < 4; ++r) x[r] = (diag && q > i0 + r) ? z2 : P2[ra[r] + DB * d + q];
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) y[cc] = P2[rq + cc];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) df_fma_acc(ah[r][cc], al[r][cc], x[r], y[cc]);
                    }
                }
                float2 *Tb = Tm2 + (b - c - 1) * DB * DB;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) Tb[(i0 + r) * DB + k0 + cc] = df_norm(ah[r][cc], al[r][cc]);
            }
            __syncthreads();
            for (int u = tid; u < nres * 64; u += 256) {   // W_bc = -T_bc W_cc
                const int b = c + 1 + u / 64, bl = u & 63;
                const int i0 = 4 * (bl >> 3), k0 = 4 * (bl & 7);
                const float2 *Tb = Tm2 + (b - c - 1) * DB * DB;
                float ah[4][4], al[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) ah[r][cc] = al[r][cc] = 0.0f;
                for (int q = k0; q < DB; ++q) {
                    float2 x[4], y[4];
                    const int rq = pk(DB * c + q, 0) + DB * c + k0;
#pragma unroll
                    for (int r = 0; r < 4; ++r) x[r] = Tb[(i0 + r) * DB + q];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) y[cc] = (q >= k0 + cc) ? P2[rq + cc] : z2;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) df_fma_acc(ah[r][cc], al[r][cc], x[r], y[cc]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const float2 v = df_norm(ah[r][cc], al[r][cc]);
                        P2[pk(DB * b + i0 + r, DB * c + k0 + cc)] = make_float2(-v.x, -v.y);
                    }
            }
            __syncthreads();
        }
    } else {
        for (int c = 2; c >= 0; --c) {   // off-diagonal blocks of block column c, in 4 x 4 register tiles
            const int nres = 3 - c;
            for (int u = tid; u < nres * 64; u += 256) {   // sums: T_bc = sum_d W_bd L_dc
                const int b = c + 1 + u / 64, bl = u & 63;
                const int i0 = 4 * (bl >> 3), k0 = 4 * (bl & 7);
                double acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.0;
                int ra[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) ra[r] = pk(DB * b + i0 + r, 0);
                for (int d = c + 1; d <= b; ++d) {
                    const bool diag = (d == b);   // W_bb is lower triangular
                    const int qend = diag ? i0 + 3 : DB - 1;
                    for (int q = 0; q <= qend; ++q) {
                        double x[4], y[4];
                        const int rq = pk(DB * d + q, 0) + DB * c + k0;
#pragma unroll
                        for (int r = 0; r < 4; ++r) x[r] = (diag && q > i0 + r) ? 0.0 : P[ra[r] + DB * d + q];
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) y[cc] = P[rq + cc];
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) acc[r][cc] = fma(x[r], y[cc], acc[r][cc]);
                    }
                }
                double *Tb = Tm + (b - c - 1) * DB * DB;
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) Tb[(i0 + r) * DB + k0 + cc] = acc[r][cc];
            }
            __syncthreads();
            for (int u = tid; u < nres * 64; u += 256) {   // W_bc = -T_bc W_cc (W_cc lower triangular)
                const int b = c + 1 + u / 64, bl = u & 63;
                const int i0 = 4 * (bl >> 3), k0 = 4 * (bl & 7);
                const double *Tb = Tm + (b - c - 1) * DB * DB;
                double acc[4][4];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) acc[r][cc] = 0.0;
                for (int q = k0; q < DB; ++q) {
                    double x[4], y[4];
                    const int rq = pk(DB * c + q, 0) + DB * c + k0;
#pragma unroll
                    for (int r = 0; r < 4; ++r) x[r] = Tb[(i0 + r) * DB + q];
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) y[cc] = (q >= k0 + cc) ? P[rq + cc] : 0.0;
#pragma unroll
                    for (int r = 0; r < 4; ++r)
#pragma unroll
                        for (int cc = 0; cc < 4; ++cc) acc[r][cc] = fma(x[r], y[cc], acc[r][cc]);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) P[pk(DB * b + i0 + r, DB * c + k0 + cc)] = -acc[r][cc];
            }
            __syncthreads();
        }
    }
    // log|tile| and sum 1/d over the pivots
    {
        double a = 0.0, bsum = 0.0;
        if (tid < TB) {
            a = log(piv[tid]);
            bsum = 1.0 / piv[tid];
        }
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xffffffffu, a, o);
            bsum += __shfl_down_sync(0xffffffffu, bsum, o);
        }
        if (lane == 0 && warp < 4) {
            red[0][warp] = a;
            red[1][warp] = bsum;
        }
    }
    const bool bad = __syncthreads_or(tid < TB && !(piv[tid] > 0.0));
    const double *Wp = P;
    const float2 *W2 = reinterpret_cast<const float2 *>(P);   // S == 5: W as double-float pairs
    // slice the rows of W (B operand of the panel solve: C = A W^T)
    uint8_t *img = wimg + (int64_t)w * img_bytes<S>();
    int *exps = reinterpret_cast<int *>(img + (size_t)S * 2 * SBLK);
    for (int r = warp; r < TB; r += 8) {
        const int bi = pk(r, 0);
        float mx = 0.0f;
        for (int k = lane; k <= r; k += 32)
            mx = fmaxf(mx, fabsf(S == 5 ? W2[bi + k].x : __double2float_rn(Wp[bi + k])));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int e = row_exp(mx * (1.0f + 1.0f / 1024.0f));
        if (lane == 0) exps[r] = e;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int k = 64 * q + 2 * lane;
            float m0[S], m1[S];
            if constexpr (S == 5) {
                const float2 z2 = make_float2(0.0f, 0.0f);
                const float2 x0 = (k <= r) ? W2[bi + k] : z2;
                const float2 x1 = (k + 1 <= r) ? W2[bi + k + 1] : z2;
                slice_df<S>(x0.x, x0.y, e, m0);
                slice_df<S>(x1.x, x1.y, e, m1);
            } else {
                const double x0 = (k <= r) ? Wp[bi + k] : 0.0;
                const double x1 = (k + 1 <= r) ? Wp[bi + k + 1] : 0.0;
                const float h0 = __double2float_rn(x0), h1 = __double2float_rn(x1);
                slice_df<S>(h0, __double2float_rn(x0 - (double)h0), e, m0);
                slice_df<S>(h1, __double2float_rn(x1 - (double)h1), e, m1);
            }
            store_pair<S>(img, r, k, m0, m1);
        }
    }
    if (tid == 0) {
        double a = 0.0, bsum = 0.0;
        for (int q = 0; q < 4; ++q) {
            a += red[0][q];
            bsum += red[1][q];
        }
        logdet[w] += a;
        const double isum = invsum[w] + bsum;
        invsum[w] = isum;
        if (bad && pstatus[w] == PLK_POINT_OK) pstatus[w] = PLK_POINT_NOT_PD;
        // early verdict (the retry rule of the 5-slice pass, applied now): the
        // bound only grows with further pivots (all 1/d_j > 0 while the
        // factorisation holds), so a point past the tolerance, or one whose
        // factorisation failed, goes to the 7-slice tier whatever the remaining
        // panels give
        if (doomed) {
            const int st = pstatus[w];
            const double E = mixed_eps(S) * (1.0 + oconst[OC_N * (int64_t)w + OC_NUG]) * isum;
            if (st == PLK_POINT_NOT_PD || (st == PLK_POINT_OK && !(E <= tol))) doomed[w] = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Shared pieces of the two split-product kernels (512 threads = 16 warps).
// Warp w reads TMEM lanes 32 (w % 4) .. +31 (its rows) and columns
// 32 (w / 4) .. +31 of each accumulator.
// ---------------------------------------------------------------------------
constexpr int NTH = 512;

__device__ __forceinline__ void load_groups(uint32_t tb, int warp, int c0, uint32_t (&p0)[16], uint32_t (&p1)[16],
                                            uint32_t (&p2)[16], uint32_t (&p3)[16]) {
    const uint32_t a = tb + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * (warp >> 2) + c0;
    tc::tmem_ld16(a + 0 * 128, p0);
    tc::tmem_ld16(a + 1 * 128, p1);
    tc::tmem_ld16(a + 2 * 128, p2);
    tc::tmem_ld16(a + 3 * 128, p3);
    tc::tmem_wait_ld();
}

// Thread's value of the product at (row r, column c): double-float of
// 2^(ea + eb) (P0 + P1 + (P2 + P3)), ea + eb including the -14.
__device__ __forceinline__ void group_value(uint32_t p0, uint32_t p1, uint32_t p2, uint32_t p3, int e, float &hi,
                                            float &lo) {
    const float sc = pow2f(e);
    hi = __uint_as_float(p0) * sc;
    lo = 0.0f;
    df_add(hi, lo, __uint_as_float(p1) * sc);
    df_add(hi, lo, (__uint_as_float(p2) + __uint_as_float(p3)) * sc);
}

// ---------------------------------------------------------------------------
// Panel solve L_IJ = A_IJ W^T on the tensor cores; the result is only kept as
// the slice image of panel slot I (the A / B operand of the trailing update).
// ---------------------------------------------------------------------------
template <int S>
__global__ void __launch_bounds__(NTH, 1) k_trsm_split(int J, int nb, int64_t tpo, const double *__restrict__ tiles,
                                                       const uint8_t *__restrict__ wimg, uint8_t *__restrict__ pimg,
                                                       const double *__restrict__ oconst, const int *__restrict__ doomed,
                                                       int *__restrict__ err) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sbase = align1024(smraw);
    uint8_t *sA = sbase;             // S blocks of the current K half of A_IJ
    uint8_t *sW = sbase + S * SBLK;  // S blocks of the current K half of W
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ short sEA[TB], sEW[TB], sEO[TB];   // row exponents, |e| <= 120
    __shared__ int sMx[TB];                         // row max |value| as float bits (>= 0)
    __shared__ int s_ok;
    const int w = blockIdx.y, I = J + 1 + blockIdx.x;
    if (doomed && doomed[w]) return;   // already bound for the 7-slice tier
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float *H = reinterpret_cast<const float *>(tiles + ((int64_t)w * tpo + tile_index(I, J)) * NT);
    const float *Lo = H + NT;
    const uint8_t *wi = wimg + (int64_t)w * img_bytes<S>();
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
        s_ok = 1;
    }
    if (tid < TB) {
        sEW[tid] = (short)reinterpret_cast<const int *>(wi + (size_t)S * 2 * SBLK)[tid];
        sMx[tid] = 0;
    }
    __syncthreads();   // barriers initialised
    // the L_JJ^-1 slices of K half 0 load while A_IJ is scanned and sliced
    // (one copy per lane: a thread's copies run one after another)
    if (warp == 0) {
        if (lane == 0) tc::mbar_arrive_expect_tx(&bar_load, S * SBLK);
        __syncwarp();
        if (lane < S) tc::bulk_g2s(sW + lane * SBLK, wi + (size_t)(lane * 2) * SBLK, SBLK, &bar_load);
    }
    // row exponents of A_IJ: data rows share one; right-hand-side rows use
    // their own maximum (warp w scans rows 8w .. 8w + 7)
    const bool data_rows = I < nb;
    if (data_rows) {
        if (tid < TB) sEA[tid] = (short)common_exp_schur(oconst[OC_N * (int64_t)w + OC_NUG]);
    } else {
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int r = warp * 8 + rr;
            float mx = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) mx = fmaxf(mx, fabsf(H[r * TB + lane + 32 * q]));
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) sEA[r] = (short)row_exp(mx);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    uint32_t phase = 0;
    // df values of this thread's rows (8 rows, 2 columns each) for K half h
    float2 hv[8], lv[8];
    auto load_half = [&](int h) {
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int r = warp * 8 + rr;
            const int k = 64 * h + 2 * lane;
            hv[rr] = *reinterpret_cast<const float2 *>(H + r * TB + k);
            lv[rr] = *reinterpret_cast<const float2 *>(Lo + r * TB + k);
        }
    };
    load_half(0);
    for (int h = 0; h < 2; ++h) {
        // slice the K half h of A_IJ into shared memory
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int r = warp * 8 + rr;
            const int e = sEA[r];
            float m0[S], m1[S];
            slice_df<S>(hv[rr].x, lv[rr].x, e, m0);
            slice_df<S>(hv[rr].y, lv[rr].y, e, m1);
            const uint32_t off = tc::sw128_offset(r, 2 * lane);
#pragma unroll
            for (int j = 0; j < S; ++j) *reinterpret_cast<uint32_t *>(sA + j * SBLK + off) = pack_bf16x2(m0[j], m1[j]);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0 && s_ok) {
            bool ok = tc::mbar_wait(&bar_load, phase);
            if (!ok) tc::mbar_wait(&bar_load, phase);
            if (ok) {
                tc::fence_after_sync();
                issue_split_mmas<S>(tb, sA, sW, h == 0);
                tc::mma_commit(&bar_mma);
            } else {
                s_ok = 0;
                atomicExch(err, 1);
            }
        }
        if (h == 0) load_half(1);   // next K half's values arrive while the MMAs run
        if (tid == 0 && s_ok) {
            bool ok = tc::mbar_wait(&bar_mma, phase);
            if (!ok) tc::mbar_wait(&bar_mma, phase);
            if (!ok) {
                s_ok = 0;
                atomicExch(err, 1);
            }
        }
        phase ^= 1;
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (h == 0 && warp == 0 && s_ok) {   // shared A and W are free again: K half 1 of W
            if (lane == 0) tc::mbar_arrive_expect_tx(&bar_load, S * SBLK);
            __syncwarp();
            if (lane < S) tc::bulk_g2s(sW + lane * SBLK, wi + (size_t)(lane * 2 + 1) * SBLK, SBLK, &bar_load);
        }
    }
    const bool ok = s_ok != 0;
    const int r = 32 * (warp & 3) + lane;   // this thread's row, columns 32 (warp / 4) .. +31
    const int cb = 32 * (warp >> 2);
    if (ok && !data_rows) {
        float mx = 0.0f;
#pragma unroll 1
        for (int c0 = 0; c0 < 32; c0 += 16) {
            uint32_t p0[16], p1[16], p2[16], p3[16];
            load_groups(tb, warp, c0, p0, p1, p2, p3);
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                const float sc = pow2f(sEA[r] + sEW[cb + c0 + c] - 14);
                const float v = (__uint_as_float(p0[c]) + __uint_as_float(p1[c]) +
                                 (__uint_as_float(p2[c]) + __uint_as_float(p3[c]))) * sc;
                mx = fmaxf(mx, fabsf(v));
            }
        }
        atomicMax(&sMx[r], __float_as_int(mx));
    }
    __syncthreads();
    if (ok) {
        const float mx = __int_as_float(sMx[r]);
        // data rows: the common exponent (lets two panels share one accumulator);
        // right-hand-side rows: their own maximum
        const int eo = data_rows ? common_exp(oconst[OC_N * (int64_t)w + OC_NUG]) : row_exp(mx * (1.0f + 1.0f / 1024.0f));
        if (warp < 4) sEO[r] = (short)eo;
#pragma unroll 1
        for (int c0 = 0; c0 < 32; c0 += 16) {
            uint32_t p0[16], p1[16], p2[16], p3[16];
            load_groups(tb, warp, c0, p0, p1, p2, p3);
            // eight columns (one 16-byte chunk of the row) per slice and store:
            // the warp's 32 rows at one chunk hit 32 distinct banks per 8 lanes
#pragma unroll
            for (int c8 = 0; c8 < 16; c8 += 8) {
                uint32_t pk2[S][4];
#pragma unroll
                for (int c = 0; c < 8; c += 2) {
                    float m[2][S];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        float hi, lo;
                        const int cc = c8 + c + u;
                        group_value(p0[cc], p1[cc], p2[cc], p3[cc], sEA[r] + sEW[cb + c0 + cc] - 14, hi, lo);
                        slice_df<S>(hi, lo, eo, m[u]);
                    }
#pragma unroll
                    for (int j = 0; j < S; ++j) pk2[j][c >> 1] = pack_bf16x2(m[0][j], m[1][j]);
                }
                const int k = cb + c0 + c8;
                const uint32_t off = tc::sw128_offset(r, k & 63);
#pragma unroll
                for (int j = 0; j < S; ++j)
                    *reinterpret_cast<uint4 *>(sbase + (size_t)(j * 2 + (k >> 6)) * SBLK + off) =
                        make_uint4(pk2[j][0], pk2[j][1], pk2[j][2], pk2[j][3]);
            }
        }
    }
    __syncthreads();
    uint8_t *dst = pimg + ((int64_t)w * (nb + 1) + I) * SLOT + (size_t)(J & 3) * img_bytes<S>();
    if (ok) {
        const uint4 *src4 = reinterpret_cast<const uint4 *>(sbase);
        uint4 *dst4 = reinterpret_cast<uint4 *>(dst);
#pragma unroll 4
        for (int e = tid; e < S * 2 * SBLK / 16; e += NTH) dst4[e] = src4[e];
        if (tid < TB) reinterpret_cast<int *>(dst + (size_t)S * 2 * SBLK)[tid] = (int)sEO[tid];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ---------------------------------------------------------------------------
// Persistent, pipelined trailing update with S = 5 or 7 slices.  One CTA per
// SM walks the work items (omega, tile (I, K), column half) of one step.
// Roles:
//   warp 0     producer: bulk copies of the B half-rows (all S slices of one K
//              half, double-buffered) and of the A slices (one slice of one K
//              half per stage, NA-stage ring);
//   warp 1     MMA issue.  S = 5: groups 0, 1, 2 and 3+ in two alternating
//              TMEM accumulator sets (2 sets x 4 groups x 64 columns = 512);
//              S = 7: the 7 groups each exact in one set (7 x 64 columns);
//   warp 2     TMEM allocation;
//   warps 4-11 epilogue: the half tile of C (double-float planes) arrives by
//              TMA (tensor map over the tile array, 128-byte swizzle) while
//              the item's MMAs run; each thread subtracts its row's TMEM
//              values in shared memory and one thread stores the half tile
//              back by TMA (with two sets, while the MMAs of the next item
//              run).
// Barrier use u of a slot completes phase u; a waiter for use u waits for
// parity (u & 1); the producer reusing a slot for use u >= 1 first waits for
// the consumer's release of use u - 1.
// ---------------------------------------------------------------------------
// Wait-cycle counters of the 5-slice trailing update, compiled in only with
// -DPLK_PIPE_COUNTERS (a diagnostic build of the library): per launch mode
// (0 triangle, 1 column, 2 right-hand-side row), summed over thread blocks,
// [0] cycles of the block's work loop, [1] items, [2] MMA warp waiting for a
// free accumulator set, [3] ... for B, [4] ... for an A stage, [5] epilogue
// waiting for the item's MMAs, [6] ... for its C half tile, [7] ... for the
// previous stores to read the C buffer, [8] epilogue update (TMEM to C).
#ifdef PLK_PIPE_COUNTERS
constexpr int PIPE_NCOUNT = 9;
__device__ unsigned long long g_pipe_counters[3][PIPE_NCOUNT];
#define PIPE_TIMED(k, expr)                                   \
    ([&]() {                                                  \
        const long long _t0 = clock64();                      \
        const auto _r = (expr);                               \
        pc[k] += (unsigned long long)(clock64() - _t0);       \
        return _r;                                            \
    }())
#else
#define PIPE_TIMED(k, expr) (expr)
#endif

namespace pipe {
constexpr int NTHP = 384;                   // warps 0-3 roles, warps 4-11 epilogue
constexpr int NEPI = NTHP - 128;
constexpr uint32_t IDESC_N64 = tc::idesc_bf16_f32(128, 64);
constexpr int CBOX = TB * 32 * 4;   // one tensor-map box: 128 rows x 32 floats (128-byte swizzle)
template <int S>
struct Cfg {
    static constexpr int NSET = (S == 5) ? 2 : 1;          // TMEM accumulator sets
    static constexpr int NA = (S == 5) ? 5 : 3;            // A stages
    static constexpr int BBUF = S * HBLK;                  // one K half of 64 B rows, S slices
    static constexpr int OFF_A = 2 * BBUF;
    static constexpr int OFF_C = OFF_A + NA * SBLK;        // C half tile: 4 boxes of 128 x 32 floats
    static constexpr int SMEM = OFF_C + 4 * CBOX + 1024;
};
}  // namespace pipe

// Item sets: mode 0 = the triangle Klo <= K <= I <= Ihi; mode 1 = the column
// K = Klo, Klo <= I <= Ihi; mode 2 = the row I = Ihi, Klo <= K <= Ihi.  Each
// item applies P (1 to 4)
// consecutive panels, the p-th in sub-slot (sub0 + p) % 4; with P >= 2 both
// operands use the common exponent (data rows only; 5 slices only).  The
// FP32 accumulators of groups 0-2 stay exact up to K = 4 x 128: with every
// data row of L bounded by sqrt(1 + nu^2) < 2^e (Cauchy-Schwarz over the
// leading digits), group 2's sums stay below 2^23.2 units.
template <int S, bool RT = false>
__global__ void __launch_bounds__(pipe::NTHP, 1) k_trail_pipe(int mode, int Klo, int Ihi, int P, int sub0,
                                                             int nb, int cnt, int64_t tpo,
                                                             const __grid_constant__ CUtensorMap tmapC,
                                                             const __grid_constant__ CUtensorMap tmapR, int qr,
                                                             const uint8_t *__restrict__ pimg,
                                                             const double *__restrict__ oconst,
                                                             const int *__restrict__ doomed, int *__restrict__ err,
                                                             const int *__restrict__ dcount = nullptr) {
    using namespace pipe;
    constexpr int NSET = Cfg<S>::NSET, NA = Cfg<S>::NA, BBUF = Cfg<S>::BBUF, OFF_A = Cfg<S>::OFF_A,
                  OFF_C = Cfg<S>::OFF_C;
    extern __shared__ uint8_t smraw[];
    uint8_t *sbase = align1024(smraw);
    __shared__ uint64_t bFull[2], bEmpty[2], aFull[NA], aEmpty[NA], accFull[2], accEmpty[2], cFull, drain;
    __shared__ uint32_t tmem_base;
    __shared__ short sEA[TB], sEB[64];
    __shared__ int s_err, s_stop;
    volatile int *verr = &s_err;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int m = Ihi - Klo + 1;
    const int T = (mode == 0) ? m * (m + 1) / 2 : m;
    // RT (5 slices, mode 2 only): the right-hand-side row runs transposed, one
    // item per tile (I = nb, K) with the tile of L_K (128 rows) as the M
    // operand and the right-hand-side image's first NR rows (qr rounded up to
    // 32; M + p <= 64 keeps NR <= 64) as B, so that C(nb, K)^T -= L_K R^T: its
    // q <= 64 live rows cost N = NR columns instead of M = 128 rows twice.  A
    // template argument, so that the other item sets compile without it.
    constexpr bool rt = RT && S == 5;
    const int NH = rt ? 1 : 2;             // items per tile (column halves)
    const int NR = (qr + 31) & ~31;
    if (dcount) cnt = min(cnt, *dcount);   // a compacted batch: its live slots only
    const int64_t items = (int64_t)cnt * T * NH;
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&bFull[i], S);   // one arrival (with its bytes) per slice lane
            tc::mbar_init(&bEmpty[i], 1);
            tc::mbar_init(&accFull[i], 1);
            tc::mbar_init(&accEmpty[i], 1);
        }
        for (int i = 0; i < NA; ++i) {
            tc::mbar_init(&aFull[i], 1);
            tc::mbar_init(&aEmpty[i], 1);
        }
        tc::mbar_init(&drain, 1);
        tc::mbar_init(&cFull, 1);
        tc::fence_mbar_init();
        s_err = 0;
    }
    if (warp == 2) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
#ifdef PLK_PIPE_COUNTERS
    const long long pc_start = clock64();
    unsigned long long pc[PIPE_NCOUNT] = {0};
#endif

    auto decode = [&](int64_t it, int &w, int &I, int &K, int &ch) {
        w = (int)(it / (NH * T));
        const int rem = (int)(it - (int64_t)w * NH * T);
        ch = (NH == 2) ? rem & 1 : 0;
        const int t = (NH == 2) ? rem >> 1 : rem;
        if (mode == 0) {
            decode_trailing(t, Klo - 1, I, K);
        } else if (mode == 1) {
            K = Klo;
            I = Klo + t;
        } else {
            I = Ihi;
            K = Klo + t;
        }
    };
    auto image = [&](int w, int R, int p) {
        return pimg + ((int64_t)w * (nb + 1) + R) * SLOT + (size_t)((sub0 + p) & 3) * img_bytes<S>();
    };

    if (warp == 0) {
        // Copies run from independent lanes with no warp-wide sync in between:
        // a lane that issues a bulk copy stalls until the copy is under way, so
        // one thread (or lanes that reconverge after each copy) would serialise
        // them.  Lane s < NA owns A ring stage s; lane 8 + j loads B slice j.
        const bool a_lane = lane < NA, b_lane = lane >= 8 && lane < 8 + S;
        if (a_lane || b_lane) {
            uint32_t acnt = 0, bcnt = 0;
            bool stop = false;
            for (int64_t it = blockIdx.x; it < items && !stop; it += gridDim.x) {
                int w, I, K, ch;
                decode(it, w, I, K, ch);
                if (doomed && doomed[w]) continue;
                for (int ph = 0; ph < 2 * P && !stop; ++ph) {
                    const int h = ph & 1;
                    const uint8_t *ia = image(w, rt ? K : I, ph >> 1), *ib = image(w, rt ? I : K, ph >> 1);
                    const int bs = bcnt & 1;
                    const uint32_t bu = bcnt >> 1;
                    ++bcnt;
                    if (b_lane) {
                        const int j = lane - 8;
                        if (*verr || (bu > 0 && !tc::mbar_wait(&bEmpty[bs], (bu - 1) & 1))) {
                            *verr = 1;
                            stop = true;
                            break;
                        }
                        // B slice j: rows 64 ch .. +63 of the K tile, or the first
                        // NR rows of the right-hand-side image (slices NR rows apart)
                        const uint32_t bb = rt ? (uint32_t)NR * 128u : (uint32_t)HBLK;
                        tc::mbar_arrive_expect_tx(&bFull[bs], bb);
                        tc::bulk_g2s(sbase + bs * BBUF + j * bb, ib + (size_t)(j * 2 + h) * SBLK + ch * HBLK, bb,
                                     &bFull[bs]);
                    }
                    for (int i = 0; i < S; ++i, ++acnt) {
                        const int as = acnt % NA;
                        if (!a_lane || as != lane) continue;
                        const uint32_t au = acnt / NA;
                        if (*verr || (au > 0 && !tc::mbar_wait(&aEmpty[as], (au - 1) & 1))) {
                            *verr = 1;
                            stop = true;
                            break;
                        }
                        tc::mbar_arrive_expect_tx(&aFull[as], SBLK);
                        tc::bulk_g2s(sbase + OFF_A + as * SBLK, ia + (size_t)(i * 2 + h) * SBLK, SBLK, &aFull[as]);
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            uint32_t acnt = 0, bcnt = 0, tcnt = 0;
            bool issued = false;
            for (int64_t it = blockIdx.x; it < items && !*verr; it += gridDim.x) {
                if (doomed && doomed[(int)(it / (NH * T))]) continue;
                const int set = (NSET == 2) ? (int)(tcnt & 1) : 0;
                const uint32_t tu = (NSET == 2) ? tcnt >> 1 : tcnt;
                if (tu > 0 && !PIPE_TIMED(2, tc::mbar_wait(&accEmpty[set], (tu - 1) & 1))) { *verr = 1; break; }
                tc::fence_after_sync();
                const uint32_t dacc = tb + set * 256;
                for (int ph = 0; ph < 2 * P && !*verr; ++ph) {
                    const int h = ph;   // first K half of the first panel starts the accumulators
                    const int bs = bcnt & 1;
                    if (!PIPE_TIMED(3, tc::mbar_wait(&bFull[bs], (bcnt >> 1) & 1))) { *verr = 1; break; }
                    ++bcnt;
                    const uint64_t b0 = tc::sdesc_sw128(tc::smem_u32(sbase + bs * BBUF));
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        const int as = acnt % NA;
                        if (!PIPE_TIMED(4, tc::mbar_wait(&aFull[as], (acnt / NA) & 1))) { *verr = 1; break; }
                        ++acnt;
                        tc::fence_after_sync();
                        const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sbase + OFF_A + as * SBLK));
                        // The B slices sit back to back (64 rows each), so slices
                        // j = 0 .. 3 - i, whose groups g = i + j are 0..3, go in one
                        // MMA of N = 64 (4 - i) into accumulators i .. 3; slice 4 - i
                        // (group 4) adds into accumulator 3.  Descriptor address
                        // fields count 16 bytes: +2 per 16-element K step.
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = a0 + 2 * kk, bk = b0 + 2 * kk;
                            const uint32_t acc = (h == 0 && kk == 0 && i == 0) ? 0u : 1u;
                            // Where one A slice feeds two MMAs, the first keeps it in
                            // the tensor core's collector buffer and the second takes it
                            // from there: A is read from shared memory once per K step.
                            if (S == 5 && rt && NR == 32) {
                                // five 32-column accumulators (group g at column 32 g):
                                // B slices 0 .. 4 - i in one MMA into groups i .. 4
                                tc::mma_bf16(dacc + 32 * i, ad, bk, tc::idesc_bf16_f32(128, 32 * (5 - i)), acc);
                            } else if (S == 5 && rt) {
                                // NR = 64: the half-tile group layout with 64-column
                                // accumulators (groups 0-3; group 4 into 3), B slices
                                // 64 rows apart
                                const uint32_t nrd = (uint32_t)NR * 128u >> 4;
                                if (i < 4) {
                                    tc::mma_bf16_ca<tc::Collector::FILL>(dacc + NR * i, ad, bk,
                                                                         tc::idesc_bf16_f32(128, NR * (4 - i)), acc);
                                    tc::mma_bf16_ca<tc::Collector::LASTUSE>(dacc + 3 * NR, ad, bk + (4 - i) * nrd,
                                                                            tc::idesc_bf16_f32(128, NR), 1u);
                                } else {
                                    tc::mma_bf16(dacc + 3 * NR, ad, bk, tc::idesc_bf16_f32(128, NR), 1u);
                                }
                            } else if (S == 5) {
                                if (i < 4) {
                                    tc::mma_bf16_ca<tc::Collector::FILL>(dacc + 64 * i, ad, bk,
                                                                         tc::idesc_bf16_f32(128, 64 * (4 - i)), acc);
                                    tc::mma_bf16_ca<tc::Collector::LASTUSE>(
                                        dacc + 3 * 64, ad, bk + (uint64_t)(((4 - i) * HBLK) >> 4), IDESC_N64, 1u);
                                } else {
                                    tc::mma_bf16(dacc + 3 * 64, ad, bk + (uint64_t)(((4 - i) * HBLK) >> 4), IDESC_N64, 1u);
                                }
                            } else {
                                // every group exact: slices j = 0 .. S-1-i into accumulators
                                // i .. S-1, at most four slices (N = 256) per MMA
                                const int nj = S - i, n1 = nj < 4 ? nj : 4;
                                if (nj > 4) {
                                    tc::mma_bf16_ca<tc::Collector::FILL>(dacc + 64 * i, ad, bk,
                                                                         tc::idesc_bf16_f32(128, 64 * n1), acc);
                                    tc::mma_bf16_ca<tc::Collector::LASTUSE>(dacc + 64 * (i + 4), ad,
                                                                            bk + (uint64_t)((4 * HBLK) >> 4),
                                                                            tc::idesc_bf16_f32(128, 64 * (nj - 4)), acc);
                                } else {
                                    tc::mma_bf16(dacc + 64 * i, ad, bk, tc::idesc_bf16_f32(128, 64 * n1), acc);
                                }
                            }
                        }
                        issued = true;
                        tc::mma_commit(&aEmpty[as]);   // the A stage is free once these MMAs finish
                    }
                    tc::mma_commit(&bEmpty[bs]);
                }
                tc::mma_commit(&accFull[set]);
                ++tcnt;
            }
            // let every issued MMA finish before the accumulators are released
            if (issued) {
                tc::mma_commit(&drain);
                if (!tc::mbar_wait(&drain, 0)) tc::mbar_wait(&drain, 0);
            }
        }
    } else if (warp >= 4) {
        const int et = tid - 128;            // 0..NEPI-1
        const int r = 32 * (warp & 3) + lane;   // this thread's row (its TMEM lane)
        const int q = (warp - 4) >> 2;       // columns 32 q .. 32 q + 31 of the half: box q
        uint8_t *sC = sbase + OFF_C;         // boxes [H, q = 0 | H, q = 1 | L, q = 0 | L, q = 1]
        float4 *rowH = reinterpret_cast<float4 *>(sC + q * CBOX + r * 128);
        float4 *rowL = reinterpret_cast<float4 *>(sC + (2 + q) * CBOX + r * 128);
        const int sw = r & 7;                // 16-byte chunk k of the row sits at k ^ (r % 8)
        uint32_t tcnt = 0;
        bool c_pending = false;              // loads issued and not yet waited for
        for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
            int w, I, K, ch;
            decode(it, w, I, K, ch);
            if (doomed && doomed[w]) continue;
            // rows of the tile in the tensor map: H plane T*256 .. +127, L plane T*256+128 .. +255
            const int yH = (int)(((int64_t)w * tpo + tile_index(I, K)) * 256);
            // a tile of the right-hand-side row holds M + p <= 64 non-zero rows:
            // only its first qr rows (M + p rounded up to 8) are read, updated
            // and written back, through the map with qr-row boxes
            const bool rhs = I == nb;
            const int rows = rhs ? qr : TB;
            const CUtensorMap *tm = rhs ? &tmapR : &tmapC;
            if (et == 0) {
                // the previous item's stores have read the buffer: load this item's half tile
                PIPE_TIMED(7, (tc::bulk_wait_read_all(), 0));
                if (rt) {   // the whole tile width: boxes [H, 32 b | L, 32 b], qr rows each
                    tc::mbar_arrive_expect_tx(&cFull, 8 * qr * 128);
#pragma unroll
                    for (int bx = 0; bx < 8; ++bx)
                        tc::tma_load_2d(sC + bx * qr * 128, tm, 32 * (bx & 3), yH + 128 * (bx >> 2), &cFull);
                } else {
                    tc::mbar_arrive_expect_tx(&cFull, 4 * rows * 128);
#pragma unroll
                    for (int bx = 0; bx < 4; ++bx)
                        tc::tma_load_2d(sC + bx * CBOX, tm, 64 * ch + 32 * (bx & 1), yH + 128 * (bx >> 1), &cFull);
                }
                c_pending = true;
            }
            if (P >= 2) {
                const short ec = (short)common_exp(oconst[OC_N * (int64_t)w + OC_NUG]);
                if (et < TB) sEA[et] = ec;
                else if (et < TB + 64) sEB[et - TB] = ec;
            } else {
                const uint8_t *ia = image(w, rt ? K : I, 0), *ib = image(w, rt ? I : K, 0);
                if (et < TB) sEA[et] = (short)reinterpret_cast<const int *>(ia + (size_t)S * 2 * SBLK)[et];
                else if (et < TB + 64)
                    sEB[et - TB] = (short)reinterpret_cast<const int *>(ib + (size_t)S * 2 * SBLK)[64 * ch + et - TB];
            }
            const int set = (NSET == 2) ? (int)(tcnt & 1) : 0;
            if (et == 0) {   // one thread waits and decides for all
                const bool ok = PIPE_TIMED(5, tc::mbar_wait(&accFull[set], ((NSET == 2) ? tcnt >> 1 : tcnt) & 1)) &&
                                PIPE_TIMED(6, tc::mbar_wait(&cFull, tcnt & 1));
#ifdef PLK_PIPE_COUNTERS
                pc[1] += 1;
#endif
                if (ok) c_pending = false;
                if (!ok) *verr = 1;
                s_stop = (!ok || *verr) ? 1 : 0;
            }
            tc::named_sync(1, NEPI);       // exponents and C visible; stop decision uniform
            if (s_stop) break;
            tc::fence_after_sync();
#ifdef PLK_PIPE_COUNTERS
            const long long pc_upd = clock64();
#endif
            if (rt) {
                // transposed right-hand-side item: this thread's TMEM lane r is
                // column r of the C tile; warps 4-7 take rows 0-7, 16-23, ...,
                // warps 8-11 rows 8-15, 24-31, ... (qr is a multiple of 8)
                const uint32_t a = tb + set * 256 + ((uint32_t)(32 * (warp & 3)) << 16);
                const int ea = sEA[r] - 14;
                float *cH = reinterpret_cast<float *>(sC + (r >> 5) * qr * 128);
                float *cL = reinterpret_cast<float *>(sC + (4 + (r >> 5)) * qr * 128);
                const int kc = (r & 31) >> 2, kw = r & 3;
#pragma unroll 1
                for (int rb = 8 * q; rb < qr; rb += 16) {
                    uint32_t p0[8], p1[8], p2[8], p3[8], p4[8];
                    tc::tmem_ld8(a + 0 * NR + rb, p0);
                    tc::tmem_ld8(a + 1 * NR + rb, p1);
                    tc::tmem_ld8(a + 2 * NR + rb, p2);
                    tc::tmem_ld8(a + 3 * NR + rb, p3);
                    if (NR == 32) tc::tmem_ld8(a + 4 * NR + rb, p4);   // group 4's own accumulator
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const int rr = rb + c;
                        // groups 3 and 4 summed in FP32, as one shared accumulator would
                        const uint32_t g3 =
                            NR == 32 ? __float_as_uint(__uint_as_float(p3[c]) + __uint_as_float(p4[c])) : p3[c];
                        float dh, dl;
                        group_value(p0[c], p1[c], p2[c], g3, ea + sEB[rr], dh, dl);
                        const int x = rr * 32 + ((kc ^ (rr & 7)) << 2) + kw;
                        float h = cH[x], l = cL[x];
                        df_add(h, l, -dh);
                        df_add(h, l, -dl);
                        cH[x] = h;
                        cL[x] = l;
                    }
                }
            } else if (32 * (warp & 3) < rows) {   // warps whose rows all lie beyond an RHS tile's rows skip
                const uint32_t a = tb + set * 256 + ((uint32_t)(32 * (warp & 3)) << 16) + 32 * q;
                const int ea = sEA[r] - 14;
                const short *eb = sEB + 32 * q;
#pragma unroll 1
                for (int c0 = 0; c0 < 32; c0 += 16) {
                    float dh[16], dl[16];
                    if (S == 5) {
                        uint32_t p0[16], p1[16], p2[16], p3[16];
                        tc::tmem_ld16(a + 0 * 64 + c0, p0);
                        tc::tmem_ld16(a + 1 * 64 + c0, p1);
                        tc::tmem_ld16(a + 2 * 64 + c0, p2);
                        tc::tmem_ld16(a + 3 * 64 + c0, p3);
                        tc::tmem_wait_ld();
#pragma unroll
                        for (int c = 0; c < 16; ++c) group_value(p0[c], p1[c], p2[c], p3[c], ea + eb[c0 + c], dh[c], dl[c]);
                    } else {
#pragma unroll 1
                        for (int g = 0; g < S; ++g) {
                            uint32_t pg[16];
                            tc::tmem_ld16(a + g * 64 + c0, pg);
                            tc::tmem_wait_ld();
#pragma unroll
                            for (int c = 0; c < 16; ++c) {
                                const float v = __uint_as_float(pg[c]) * pow2f(ea + eb[c0 + c]);
                                if (g == 0) {
                                    dh[c] = v;
                                    dl[c] = 0.0f;
                                } else {
                                    df_add(dh[c], dl[c], v);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int k4 = 0; k4 < 4; ++k4) {
                        const int kc = ((c0 >> 2) + k4) ^ sw;
                        float4 h = rowH[kc], l = rowL[kc];
                        df_add(h.x, l.x, -dh[4 * k4 + 0]);
                        df_add(h.x, l.x, -dl[4 * k4 + 0]);
                        df_add(h.y, l.y, -dh[4 * k4 + 1]);
                        df_add(h.y, l.y, -dl[4 * k4 + 1]);
                        df_add(h.z, l.z, -dh[4 * k4 + 2]);
                        df_add(h.z, l.z, -dl[4 * k4 + 2]);
                        df_add(h.w, l.w, -dh[4 * k4 + 3]);
                        df_add(h.w, l.w, -dl[4 * k4 + 3]);
                        rowH[kc] = h;
                        rowL[kc] = l;
                    }
                }
            }
            tc::fence_proxy_async();        // these writes are read by the TMA store
            tc::fence_before_sync();
            tc::named_sync(1, NEPI);
#ifdef PLK_PIPE_COUNTERS
            pc[8] += (unsigned long long)(clock64() - pc_upd);
#endif
            if (et == 0) {
                tc::mbar_arrive(&accEmpty[set]);   // the MMA warp may reuse this set
                if (rt) {
#pragma unroll
                    for (int bx = 0; bx < 8; ++bx)
                        tc::tma_store_2d(tm, 32 * (bx & 3), yH + 128 * (bx >> 2), sC + bx * qr * 128);
                } else {
#pragma unroll
                    for (int bx = 0; bx < 4; ++bx)
                        tc::tma_store_2d(tm, 64 * ch + 32 * (bx & 1), yH + 128 * (bx >> 1), sC + bx * CBOX);
                }
                tc::bulk_commit();
            }
            ++tcnt;
        }
        if (et == 0) {
            tc::bulk_wait_all();
            if (c_pending) tc::mbar_wait(&cFull, tcnt & 1);   // error exit: let the loads land first
        }
    }
    __syncthreads();
#ifdef PLK_PIPE_COUNTERS
    if (S == 5 && (tid == 32 || tid == 128) && mode >= 0 && mode < 3) {   // the MMA thread, the epilogue's first
        if (tid == 32) {
            atomicAdd(&g_pipe_counters[mode][0], (unsigned long long)(clock64() - pc_start));
            for (int k = 2; k <= 4; ++k) atomicAdd(&g_pipe_counters[mode][k], pc[k]);
        } else {
            atomicAdd(&g_pipe_counters[mode][1], pc[1]);
            for (int k = 5; k <= 8; ++k) atomicAdd(&g_pipe_counters[mode][k], pc[k]);
        }
    }
#endif
    if (*verr && tid == 0) atomicExch(err, 1);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 2) tc::tmem_dealloc(tb, 512);
}

// ---------------------------------------------------------------------------
// 7-slice variants with every group exact: the 128 x 128 result is produced as
// two 128 x 64 column halves; each half keeps the 7 groups g = 0..6 in their
// own 64-column TMEM accumulators (448 columns), so no group is rounded before
// the double-float epilogue.  Used for the re-evaluation of points whose
// 5-slice error bound was too large.
// ---------------------------------------------------------------------------
constexpr int S7 = 7;

__device__ __forceinline__ void issue_exact_mmas7(uint32_t tb, const uint8_t *sA, const uint8_t *sB, bool first_half) {
    // B slices are back to back (64 rows each): slices j = 0 .. 6 - i go into
    // accumulators i .. 6 in at most two MMAs of N <= 256.
    const uint64_t a0 = tc::sdesc_sw128(tc::smem_u32(sA)), b0 = tc::sdesc_sw128(tc::smem_u32(sB));
#pragma unroll
    for (int i = 0; i < S7; ++i) {
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = a0 + (uint64_t)((i * SBLK + kk * 32) >> 4), bk = b0 + 2 * kk;
            const uint32_t accumulate = (first_half && kk == 0 && i == 0) ? 0u : 1u;
            const int nj = S7 - i, n1 = nj < 4 ? nj : 4;
            tc::mma_bf16(tb + i * 64, ad, bk, tc::idesc_bf16_f32(128, 64 * n1), accumulate);
            if (nj > 4)
                tc::mma_bf16(tb + (i + 4) * 64, ad, bk + (uint64_t)((4 * HBLK) >> 4),
                             tc::idesc_bf16_f32(128, 64 * (nj - 4)), accumulate);
        }
    }
}

// double-float of 2^e sum_g P_g over the 7 exact groups at column c of this
// thread's row (16 columns per call); warp w: lanes 32 (w % 4), columns cb..cb+15
__device__ __forceinline__ void exact_values7(uint32_t tb, int warp, int cb, const short *eB, int ea, float (&hi)[16],
                                              float (&lo)[16]) {
    const uint32_t a = tb + ((uint32_t)(32 * (warp & 3)) << 16) + cb;
#pragma unroll 1
    for (int g = 0; g < S7; ++g) {
        uint32_t pg[16];
        tc::tmem_ld16(a + g * 64, pg);
        tc::tmem_wait_ld();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float v = __uint_as_float(pg[c]) * pow2f(ea + eB[c]);
            if (g == 0) {
                hi[c] = v;
                lo[c] = 0.0f;
            } else {
                df_add(hi[c], lo[c], v);
            }
        }
    }
}

// Panel solve with 7 exact groups: the two column halves of L_IJ are written
// as double-float planes into the panel slot (scratch), then every row is
// sliced with its exponent over all 128 columns and the image replaces the
// scratch.
__global__ void __launch_bounds__(NTH, 1) k_trsm_split7x(int J, int nb, int64_t tpo, const double *__restrict__ tiles,
                                                         const uint8_t *__restrict__ wimg, uint8_t *__restrict__ pimg,
                                                         int *__restrict__ err, const int *__restrict__ dcount = nullptr) {
    extern __shared__ uint8_t smraw[];
    uint8_t *sbase = align1024(smraw);
    uint8_t *sA = sbase;
    uint8_t *sW = sbase + S7 * SBLK;
    __shared__ uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_base;
    __shared__ short sEA[TB], sEW[TB], sEO[TB];
    __shared__ int sMx[TB];
    __shared__ int s_ok;
    const int w = blockIdx.y, I = J + 1 + blockIdx.x;
    if (beyond(dcount, w)) return;   // before any barrier or TMEM allocation
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float *H = reinterpret_cast<const float *>(tiles + ((int64_t)w * tpo + tile_index(I, J)) * NT);
    const float *Lo = H + NT;
    const uint8_t *wi = wimg + (int64_t)w * img_bytes<S7>();
    uint8_t *slot = pimg + ((int64_t)w * (nb + 1) + I) * SLOT;
    float *scH = reinterpret_cast<float *>(slot);   // scratch planes of L_IJ (128 KB < slot)
    float *scL = scH + NT;
    if (warp == 0) {
        tc::tmem_alloc(&tmem_base, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar_load, 1);
        tc::mbar_init(&bar_mma, 1);
        tc::fence_mbar_init();
        s_ok = 1;
    }
    if (tid < TB) {
        sEW[tid] = (short)reinterpret_cast<const int *>(wi + (size_t)S7 * 2 * SBLK)[tid];
        sMx[tid] = 0;
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
        const int r = warp * 8 + rr;
        float mx = 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) mx = fmaxf(mx, fabsf(H[r * TB + lane + 32 * q]));
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) sEA[r] = (short)row_exp(mx);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tb = tmem_base;
    uint32_t phase = 0;
    for (int ch = 0; ch < 2; ++ch) {
        for (int h = 0; h < 2; ++h) {
#pragma unroll 2
            for (int rr = 0; rr < 8; ++rr) {
                const int r = warp * 8 + rr;
                const int k = 64 * h + 2 * lane;
                const float2 hv = *reinterpret_cast<const float2 *>(H + r * TB + k);
                const float2 lv = *reinterpret_cast<const float2 *>(Lo + r * TB + k);
                float m0[S7], m1[S7];
                slice_df<S7>(hv.x, lv.x, sEA[r], m0);
                slice_df<S7>(hv.y, lv.y, sEA[r], m1);
                const uint32_t off = tc::sw128_offset(r, 2 * lane);
#pragma unroll
                for (int j = 0; j < S7; ++j)
                    *reinterpret_cast<uint32_t *>(sA + j * SBLK + off) = pack_bf16x2(m0[j], m1[j]);
            }
            tc::fence_proxy_async();
            __syncthreads();
            if (warp == 0 && s_ok) {   // one copy per lane: a thread's copies run one after another
                if (lane == 0) tc::mbar_arrive_expect_tx(&bar_load, S7 * HBLK);
                __syncwarp();
                if (lane < S7)
                    tc::bulk_g2s(sW + lane * HBLK, wi + (size_t)(lane * 2 + h) * SBLK + ch * HBLK, HBLK, &bar_load);
            }
            if (tid == 0 && s_ok) {
                bool ok = tc::mbar_wait(&bar_load, phase);
                if (!ok) tc::mbar_wait(&bar_load, phase);
                if (ok) {
                    tc::fence_after_sync();
                    issue_exact_mmas7(tb, sA, sW, h == 0);
                    tc::mma_commit(&bar_mma);
                    ok = tc::mbar_wait(&bar_mma, phase);
                    if (!ok) tc::mbar_wait(&bar_mma, phase);
                }
                if (!ok) {
                    s_ok = 0;
                    atomicExch(err, 1);
                }
            }
            phase ^= 1;
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
        }
        if (s_ok) {
            const int r = 32 * (warp & 3) + lane;
            const int cb = 16 * (warp >> 2);
            float hi[16], lo[16];
            exact_values7(tb, warp, cb, sEW + 64 * ch + cb, sEA[r] - 14, hi, lo);
            float mx = 0.0f;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                scH[r * TB + 64 * ch + cb + c] = hi[c];
                scL[r * TB + 64 * ch + cb + c] = lo[c];
                mx = fmaxf(mx, fabsf(hi[c]));
            }
            atomicMax(&sMx[r], __float_as_int(mx));
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    const bool ok = s_ok != 0;
    if (ok) {
        // slice: thread handles row r = tid / 4, columns 32 (tid % 4) .. +31
        const int r = tid >> 2, c0 = 32 * (tid & 3);
        const int eo = row_exp(__int_as_float(sMx[r]) * (1.0f + 1.0f / 1024.0f));
        if ((tid & 3) == 0) sEO[r] = (short)eo;
#pragma unroll 1
        for (int c = 0; c < 32; c += 2) {
            float m0[S7], m1[S7];
            slice_df<S7>(scH[r * TB + c0 + c], scL[r * TB + c0 + c], eo, m0);
            slice_df<S7>(scH[r * TB + c0 + c + 1], scL[r * TB + c0 + c + 1], eo, m1);
            store_pair<S7>(sbase, r, c0 + c, m0, m1);
        }
    }
    __syncthreads();   // all scratch reads done before the image overwrites it
    if (ok) {
        const uint4 *src4 = reinterpret_cast<const uint4 *>(sbase);
        uint4 *dst4 = reinterpret_cast<uint4 *>(slot);
#pragma unroll 4
        for (int e = tid; e < S7 * 2 * SBLK / 16; e += NTH) dst4[e] = src4[e];
        if (tid < TB) reinterpret_cast<int *>(slot + (size_t)S7 * 2 * SBLK)[tid] = (int)sEO[tid];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tb, 512);
}

// ---------------------------------------------------------------------------
// Error bound and retry flags
// ---------------------------------------------------------------------------
// E = eps_S * (1 + nu^2) * sum_j 1/d_j, d_j the pivots: a first-order bound on
// |Delta log|V|| from a relative perturbation eps_S of each updated entry.
__global__ void k_mixed_bound(int count, int64_t k0, double eps, double tol, int flag_not_pd, int keep_doomed,
                              const double *__restrict__ oconst, const double *__restrict__ invsum,
                              const int *__restrict__ pstatus, const int *__restrict__ out_index, double *err_bound,
                              int *flags, const int *__restrict__ dcount = nullptr) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= count) return;
    if (beyond(dcount, w)) {   // not a live slot: nothing to re-evaluate
        flags[w] = 0;
        return;
    }
    const double E = eps * (1.0 + oconst[OC_N * w + OC_NUG]) * invsum[w];
    const int64_t k = out_index ? (int64_t)out_index[w] : k0 + w;
    if (err_bound) err_bound[k] = E;
    const int st = pstatus[w];
    // a point marked by the early verdict stopped part-way: its status and
    // results are incomplete, it is re-evaluated in any case
    const bool doomed = keep_doomed && flags[w];
    flags[w] = (doomed || (flag_not_pd && st == PLK_POINT_NOT_PD) || (st == PLK_POINT_OK && !(E <= tol))) ? 1 : 0;
}

// Stream compaction of the flagged slots of a batch, in slot order, by one
// block: out_idx[j] = the j-th flagged slot w's output row (map[w], or k0 + w
// without a map), *out_count = their number.  Only slots below *live (when
// given) are considered.  The mixed path's retry tiers run over these lists
// with no host read-back of the flags.
__global__ void __launch_bounds__(1024) k_compact_flags(int count, const int *__restrict__ flags,
                                                        const int *__restrict__ live, int64_t k0,
                                                        const int *__restrict__ map, int *__restrict__ out_idx,
                                                        int *__restrict__ out_count) {
    __shared__ int wsum[32];
    __shared__ int s_base, s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n = live ? min(count, *live) : count;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < n; c0 += 1024) {
        const int w = c0 + tid;
        const int f = (w < n && flags[w]) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        const int before = __popc(bal & ((1u << lane) - 1u));   // flagged lanes below this one
        if (lane == 0) wsum[warp] = __popc(bal);
        __syncthreads();
        if (warp == 0) {   // exclusive prefix over the 32 warps
            const int v = wsum[lane];
            int incl = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            wsum[lane] = incl - v;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (f) out_idx[s_base + wsum[warp] + before] = map ? map[w] : (int)(k0 + w);
        __syncthreads();
        if (tid == 0) s_base += s_total;
        __syncthreads();
    }
    if (tid == 0) *out_count = s_base;
}

cudaError_t pipe_counters(unsigned long long *out, int reset) {
#ifdef PLK_PIPE_COUNTERS
    cudaError_t e = cudaMemcpyFromSymbol(out, g_pipe_counters, sizeof(g_pipe_counters));
    if (e == cudaSuccess && reset) {
        static const unsigned long long zero[3 * PIPE_NCOUNT] = {};
        e = cudaMemcpyToSymbol(g_pipe_counters, zero, sizeof(zero));
    }
    return e;
#else
    (void)out;
    (void)reset;
    return cudaErrorNotSupported;
#endif
}

// The IF condition of a graph's conditional node from a device-side count
// (one thread): the node's body runs only where *count > 0.
__global__ void k_set_condition(cudaGraphConditionalHandle h, const int *__restrict__ count) {
    if (threadIdx.x == 0) cudaGraphSetConditional(h, *count > 0 ? 1u : 0u);
}

cudaError_t launch_set_condition(cudaGraphConditionalHandle h, const int *count, cudaStream_t s) {
    k_set_condition<<<1, 32, 0, s>>>(h, count);
    return cudaGetLastError();
}

cudaError_t launch_compact_flags(int count, const int *flags, const int *live, int64_t k0, const int *map,
                                 int *out_idx, int *out_count, cudaStream_t s) {
    k_compact_flags<<<1, 1024, 0, s>>>(count, flags, live, k0, map, out_idx, out_count);
    return cudaGetLastError();
}

__global__ void k_scatter_value(int count, const int *__restrict__ idx, double v, double *out, const int *__restrict__ dcount = nullptr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count && !beyond(dcount, t)) out[idx[t]] = v;
}

__global__ void k_gather_params(int count, const int *__restrict__ idx, const double *__restrict__ params,
                                double *__restrict__ out, const int *__restrict__ dcount = nullptr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count * 5 || beyond(dcount, t / 5)) return;
    out[t] = params[(int64_t)idx[t / 5] * 5 + t % 5];
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t mixed_img_bytes(int S) { return S == 5 ? img_bytes<5>() : img_bytes<7>(); }
size_t mixed_slot_bytes() { return SLOT; }

static int num_sms() {
    int dev = 0, n = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

#define TIMED(cls, launch)               \
    do {                                 \
        if (timer) timer->begin(cls, s); \
        launch;                          \
        if (timer) timer->end(cls, s);   \
    } while (0)

// Tensor map over the batch's tile array seen as float rows of 128: tile T
// (global index w * tpo + t) holds its H plane in rows 256 T .. 256 T + 127 and
// its L plane in the next 128 rows.  Box: 32 floats x 128 rows, 128-byte
// swizzle (the trailing update's C half tile is four boxes).
static cudaError_t make_tile_map(CUtensorMap *m, double *tiles, int count, int64_t tpo, int box_rows = TB) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return cudaErrorNotSupported;
    const int64_t rows = (int64_t)count * tpo * 256;
    if (rows > (int64_t)INT32_MAX) return cudaErrorInvalidValue;   // row coordinates are 32-bit
    const cuuint64_t dims[2] = {(cuuint64_t)TB, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)TB * sizeof(float)};
    const cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, tiles, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int S>
static cudaError_t launch_mixed_steps(const BatchArgs &b, const MixedArgs &x, cudaStream_t s) {
    KernelTimer *timer = b.timer;
    const int cnt = b.count, nb = b.nb;
    const int smem_split = 2 * S * SBLK + 1024;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_potrf_mixed<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)POTRF_MIXED_SMEM)) != cudaSuccess)
        return e;
    cudaMemsetAsync(x.invsum, 0, sizeof(double) * cnt, s);
    // 5-slice pass with the early verdict: flags marks the points already bound
    // for the 7-slice tier (the bound kernel keeps the marks)
    int *doomed = (S == 5 && x.early) ? x.flags : nullptr;
    if (doomed) cudaMemsetAsync(doomed, 0, sizeof(int) * cnt, s);
    CUtensorMap tmapC, tmapR;
    const int qr = std::min(TB, (b.q + 7) / 8 * 8);   // rows of a right-hand-side tile that can be non-zero
    if ((e = make_tile_map(&tmapC, b.tiles, cnt, b.tpo)) != cudaSuccess) return e;
    if ((e = make_tile_map(&tmapR, b.tiles, cnt, b.tpo, qr)) != cudaSuccess) return e;
    const int sms = num_sms();
    if constexpr (S == 7) {
        if ((e = cudaFuncSetAttribute(k_trsm_split7x, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_split)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_trail_pipe<7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      pipe::Cfg<7>::SMEM)) != cudaSuccess)
            return e;
        for (int J = 0; J < nb; ++J) {
            TIMED(KC_POTRF_MIXED, (k_potrf_mixed<S><<<cnt, 256, POTRF_MIXED_SMEM, s>>>(
                                      J, b.tpo, b.tiles, x.wimg, b.ldv, x.invsum, b.pstatus, b.oconst, nullptr, x.tol,
                                      b.dcount)));
            const int m = nb - J;
            TIMED(KC_TRSM_SPLIT7, (k_trsm_split7x<<<dim3(m, cnt), NTH, smem_split, s>>>(J, nb, b.tpo, b.tiles, x.wimg,
                                                                                      x.pimg, x.err, b.dcount)));
            // trailing triangle J+1 <= K <= I <= nb (data rows and the right-hand-side row)
            const int64_t items = (int64_t)cnt * (m * (m + 1) / 2) * 2;
            const int grid = (int)std::min<int64_t>(items, sms);
            TIMED(KC_GEMM_SPLIT7, (k_trail_pipe<7><<<grid, pipe::NTHP, pipe::Cfg<7>::SMEM, s>>>(
                                      0, J + 1, nb, 1, 0, nb, cnt, b.tpo, tmapC, tmapR, qr, x.pimg, b.oconst, nullptr,
                                      x.err, b.dcount)));
        }
    } else {
        if ((e = cudaFuncSetAttribute(k_trsm_split<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_split)) !=
            cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(k_trail_pipe<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      pipe::Cfg<5>::SMEM)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_trail_pipe<5, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      pipe::Cfg<5>::SMEM)) != cudaSuccess)
            return e;
        auto trail = [&](int mode, int Klo, int Ihi, int P, int sub0) {
            const int m = Ihi - Klo + 1;
            if (m <= 0) return;
            const int64_t T = (mode == 0) ? (int64_t)m * (m + 1) / 2 : m;
            const int64_t items = (int64_t)cnt * T * (mode == 2 ? 1 : 2);   // mode 2: whole tiles
            const int grid = (int)std::min<int64_t>(items, sms);
            auto *kern = (mode == 2) ? k_trail_pipe<5, true> : k_trail_pipe<5, false>;   // mode 2 transposed
            TIMED(KC_GEMM_SPLIT, (kern<<<grid, pipe::NTHP, pipe::Cfg<5>::SMEM, s>>>(
                                     mode, Klo, Ihi, P, sub0, nb, cnt, b.tpo, tmapC, tmapR, qr, x.pimg, b.oconst, doomed,
                                     x.err, nullptr)));
        };
        auto factor_panel = [&](int J) {
            TIMED(KC_POTRF_MIXED, (k_potrf_mixed<S><<<cnt, 256, POTRF_MIXED_SMEM, s>>>(
                                      J, b.tpo, b.tiles, x.wimg, b.ldv, x.invsum, b.pstatus, b.oconst, doomed, x.tol)));
            TIMED(KC_TRSM_SPLIT, (k_trsm_split<S><<<dim3(nb - J, cnt), NTH, smem_split, s>>>(
                                     J, nb, b.tpo, b.tiles, x.wimg, x.pimg, b.oconst, doomed, x.err)));
        };
        // Panels in groups of up to four: before panel J is factored, its tile
        // column's data rows receive the group's earlier panels in one launch
        // (one read-modify-write per tile); after it, the right-hand-side row
        // (K = J + 1 .. nb, own exponents) receives panel J; after the group,
        // the data triangle beyond it receives all of the group's panels at
        // once (K = 512 in one accumulator set: one read-modify-write of every
        // trailing tile per four panels).
        constexpr int GP = 4;
        for (int J0 = 0; J0 < nb; J0 += GP) {
            const int G = std::min(GP, nb - J0), Jend = J0 + G;   // panels J0 .. Jend - 1
            for (int J = J0; J < Jend; ++J) {
                if (J > J0) trail(1, J, nb - 1, J - J0, J0 & 3);   // column J with panels J0 .. J - 1
                factor_panel(J);
                trail(2, J + 1, nb, 1, J & 3);                      // RHS row with panel J, incl. the corner
            }
            trail(0, Jend, nb - 1, G, J0 & 3);                      // data triangle with the group's panels
        }
    }
    TIMED(KC_CONVERT, (k_tile_to_fp64<<<cnt, 256, 0, s>>>(b.tpo, tile_index(nb, nb), b.tiles, b.dcount)));
    return cudaGetLastError();
}

cudaError_t launch_mixed_batch(const BatchArgs &b, const MixedArgs &x, int S, cudaStream_t s) {
    // double-float tiles: FP32 pair arithmetic for the 5-slice pass, FP64 for
    // the 7-slice tier (whose 2^-46 products need entries good to ~1e-16)
    cudaError_t e = launch_front(b, s, S == 5 ? FRONT_DF_FAST : FRONT_DF);
    if (e != cudaSuccess) return e;
    return launch_mixed_back(b, x, S, s);
}

cudaError_t launch_mixed_back(const BatchArgs &b, const MixedArgs &x, int S, cudaStream_t s) {
    cudaError_t e = (S == 7) ? launch_mixed_steps<7>(b, x, s) : launch_mixed_steps<5>(b, x, s);
    if (e != cudaSuccess) return e;
    if ((e = launch_finalize(b, s)) != cudaSuccess) return e;
    const double eps = mixed_eps(S);
    k_mixed_bound<<<(b.count + 127) / 128, 128, 0, s>>>(b.count, b.k0, eps, x.tol, S == 5 ? 1 : 0,
                                                       S == 5 && x.early ? 1 : 0, b.oconst, x.invsum, b.pstatus,
                                                       b.out_index, x.err_bound, x.flags, b.dcount);
    return cudaGetLastError();
}

// Self-test of the bounded waits: thread 0 waits on a barrier that nothing
// completes, with the same bounded wait the tensor-core kernels use; when it
// gives up, the kernel records the failure in *err and returns.
__global__ void k_wait_selftest(uint32_t max_iter, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, max_iter)) atomicExch(err, 1);
}

cudaError_t launch_wait_selftest(uint32_t max_iter, int *err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(max_iter, err);
    return cudaGetLastError();
}

cudaError_t launch_scatter_value(int count, const int *idx, double v, double *out, cudaStream_t s,
                                 const int *dcount) {
    k_scatter_value<<<(count + 127) / 128, 128, 0, s>>>(count, idx, v, out, dcount);
    return cudaGetLastError();
}

cudaError_t launch_gather_params(int count, const int *idx, const double *params, double *out, cudaStream_t s,
                                 const int *dcount) {
    k_gather_params<<<(count * 5 + 255) / 256, 256, 0, s>>>(count, idx, params, out, dcount);
    return cudaGetLastError();
}

}  // namespace plk
