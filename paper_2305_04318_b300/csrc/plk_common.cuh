// plk_common.cuh -- layout constants and small device helpers shared by the
// CUDA kernels of libplk (the B300 profile-likelihood library).
//
// Data layout of one parameter point omega in a batch workspace:
//   The bordered matrix  A = [[V, 0], [B^T, 0]]  of size (N + TB) x (N + TB), where
//   N = n rounded up to a multiple of the tile size TB, V = R(omega) + nu^2 I
//   (padded with the identity), and B = [y'(lambda_1) ... y'(lambda_M) | X] is the
//   n x q right-hand side (q = M + p <= TB) placed as q rows of the last tile row.
//   Only the lower-triangular tiles are stored, tile-major: tile (I, J), J <= I,
//   is TB x TB doubles, row-major, at index I (I + 1) / 2 + J.
//   Factoring the first N columns (right-looking blocked Cholesky) leaves
//     L             in the data tiles        (V = L L^T, Section 3.3 Step 3 item 2)
//     W^T = B^T L^-T in the last tile row     (W = L^-1 B, item 3)
//     -B^T V^-1 B    in the last diagonal tile (ssqYX of Table 1, item 4)
//   so the triangular solve and the cross-products come out of the same trailing
//   updates as the factorisation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace plk {

constexpr int TB = 128;                 // tile edge
constexpr int NT = TB * TB;             // doubles per tile
constexpr int PK = TB * (TB + 1) / 2;   // packed lower triangle of one tile

// Per-omega constants (10 doubles): kappa, nu^2, log c_kappa, sqrt(8 kappa),
// cos phi_A, sin phi_A, sqrt(8 kappa)/phi_X, sqrt(8 kappa)/phi_Y, and the
// octaves [e_lo, e_hi) of w = u^2 that the point's site pairs can reach (the
// rho table is built and read there only).
constexpr int OC_KAPPA = 0, OC_NUG = 1, OC_LOGC = 2, OC_S8K = 3, OC_COS = 4, OC_SIN = 5,
              OC_IA = 6, OC_IB = 7, OC_ELO = 8, OC_EHI = 9, OC_N = 10;

// Piecewise-polynomial table of rho as a function of w = u^2 = 8 kappa d^2.
// Octaves [2^e, 2^(e+1)) for e in [TAB_ELO, TAB_EHI), each cut into TAB_S equal
// sub-intervals; on each, a degree TAB_NC-1 polynomial in the local variable
// t in [-1, 1) (monomial coefficients of the Chebyshev interpolant).
constexpr int TAB_ELO = -40;
constexpr int TAB_EHI = 14;
constexpr int TAB_SB = 3;               // log2 of sub-intervals per octave
constexpr int TAB_S = 1 << TAB_SB;
constexpr int TAB_NC = 10;              // coefficients per sub-interval
constexpr int TAB_NBUCKET = (TAB_EHI - TAB_ELO) * TAB_S;
constexpr int TAB_SIZE = TAB_NBUCKET * TAB_NC;
// Float layout of one sub-interval (first pass of the mixed path): the TAB_DF
// leading coefficients as (hi, lo) pairs, the rest as single floats, padded to
// TAB_F32 floats (64 bytes: two 32-byte vector loads).
constexpr int TAB_DF = 4;
constexpr int TAB_F32 = 16;
static_assert(2 * TAB_DF + (TAB_NC - TAB_DF) <= TAB_F32, "float table layout");
static_assert(TAB_NBUCKET * TAB_F32 * 4 <= TAB_SIZE * 8, "float table fits the per-point region");

// Fixed trapezoid grid used by the table builder for u <= TAB_USPLIT.
constexpr double QH = 0.125;
constexpr int QNODES = 256;
constexpr double TAB_USPLIT = 16.0;

__host__ __device__ inline int64_t tile_index(int I, int J) {
    return (int64_t)I * (I + 1) / 2 + J;
}
__host__ __device__ inline int64_t tiles_per_omega(int nb) {  // nb data tile rows + 1 RHS row
    return (int64_t)(nb + 1) * (nb + 2) / 2;
}
__device__ inline int pk(int r, int c) { return r * (r + 1) / 2 + c; }

// (I, K) of the t-th trailing tile J+1 <= K <= I <= nb at step J.
__device__ inline void decode_trailing(int t, int J, int &I, int &K) {
    int ir = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while ((ir + 1) * (ir + 2) / 2 <= t) ++ir;
    while (ir * (ir + 1) / 2 > t) --ir;
    I = J + 1 + ir;
    K = J + 1 + (t - ir * (ir + 1) / 2);
}

// A batch whose points were compacted on the device (the mixed path's retry
// tiers) is launched over its upper bound of slots; slots at or beyond the
// device-side count *dcount return at once (dcount NULL: every slot is live).
__device__ __forceinline__ bool beyond(const int *dcount, int w) { return dcount && w >= *dcount; }

}  // namespace plk
