// plk_kernels.cuh -- launchers of the CUDA kernels (internal to libplk).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace plk {

// Kernel classes for the optional per-launch event timing.
enum KernelClass { KC_BOXCOX = 0, KC_PREP, KC_TABLE, KC_BUILD, KC_POTRF, KC_TRSM, KC_GEMM, KC_FINAL,
                   KC_PROFILE, KC_CONVERT, KC_POTRF_MIXED, KC_TRSM_SPLIT, KC_GEMM_SPLIT, KC_TRSM_SPLIT7, KC_GEMM_SPLIT7, KC_FUSED, KC_COUNT };
const char *kernel_class_name(int c);

// Records a CUDA event pair around a launch on its stream (see plk_api.cu).
struct KernelTimer {
    virtual void begin(int cls, cudaStream_t s) = 0;
    virtual void end(int cls, cudaStream_t s) = 0;
    virtual ~KernelTimer() {}
};

// One batch of `count` parameter points of one dataset.  Per-point arrays
// (oconst, coordT, tab, tiles, inv, ldv, pstatus) are indexed by the point's
// position w in the batch; outputs by its global index k0 + w.
struct BatchArgs {
    int count;
    int64_t k0;
    int64_t n, n_pad;
    int nb, q, p, M, reml;
    int64_t tpo;
    const double *params;    // count x 5 (already offset to the batch)
    const double *coords;    // n x 2
    const double *lambdas;   // M
    const double *Bt;        // q x n_pad
    const double *sumlogy;   // 2: sum log y, smallest squared site distance
    double *oconst;          // count x OC_N
    double *coordT;          // count x 2 x n_pad
    double *tab;             // count x TAB_SIZE
    double *tiles;           // count x tpo x NT
    double *inv;             // count x NT
    double *ldv;             // count
    int *pstatus;            // count
    double *logL, *sigma2, *beta, *logdet;
    double *ssq = nullptr;   // K x q x q (Table 1 ssqYX), may be NULL
    int32_t *status;
    KernelTimer *timer = nullptr;
    const int *out_index = nullptr;   // when set, batch slot w writes output row out_index[w]
    int32_t status_or = 0;            // bits OR-ed into every written status
    int *owner = nullptr;             // count: slot whose rho table this slot reads (NULL: its own)
    const int *dcount = nullptr;      // device: live slots 0 .. *dcount - 1 of the count (NULL: all)
};

// Sets the calling thread's message returned by plk_last_error().
void set_last_error(const char *msg);

cudaError_t launch_boxcox(int64_t n, int64_t n_pad, int p, int M, const double *y, const double *X,
                          const double *coords, const double *lam, double *Bt, double *sumlogy, cudaStream_t s,
                          KernelTimer *timer = nullptr);
cudaError_t launch_fp64_batch(const BatchArgs &b, cudaStream_t s);
// pieces of the batch pipeline shared with the mixed path
// prep, table, build: FP64 tiles; double-float planes evaluated in FP64 (the
// mixed path's 7-slice tier); double-float planes evaluated in FP32 pair
// arithmetic (the mixed path's 5-slice pass)
enum FrontMode { FRONT_FP64 = 0, FRONT_DF = 1, FRONT_DF_FAST = 2 };
cudaError_t launch_front(const BatchArgs &b, cudaStream_t s, FrontMode mode, bool build = true);
// Small datasets (n + q <= FUSED_MAX_R): the whole point in one CTA (build,
// FP64 Cholesky of the bordered matrix, closed form), in either precision
constexpr int FUSED_MAX_R = 224;
bool fused_applies(int64_t n, int q);
size_t fused_smem_bytes(int64_t n, int q);
cudaError_t launch_fused_batch(const BatchArgs &b, cudaStream_t s);
// the same in double-float FP32 (mixed precision); invsum[w] = sum_j 1/d_j of
// the pivots (for the a-posteriori bound), 0 for points that failed
// ... with each point's bound eps (1 + nu^2) sum 1/d_j into err_bound (may be
// NULL) and its re-evaluation flag (bound above tol, or a failed
// factorisation) into flags
cudaError_t launch_fused_df_batch(const BatchArgs &b, double *invsum, double eps, double tol, double *err_bound,
                                  int *flags, cudaStream_t s);
// the FP64 fused evaluation of the slots w with gate[w] != 0 (device flags),
// in place (status bits RETRIED | FP64, err_bound 0), without a host read-back
cudaError_t launch_fused_fp64_gated(const BatchArgs &b, const int *gate, double *err_bound, cudaStream_t s);
// relative perturbation of V's entries in the double-float fused Cholesky
// (bound E = FUSED_DF_EPS (1 + nu^2) sum_j 1 / d_j)
constexpr double FUSED_DF_EPS = 1.4551915228366852e-11;   // 2^-36
// closed form (beta, sigma^2, l_p, Table-1 cross-products) from the last
// diagonal tile of every point of the batch
cudaError_t launch_finalize(const BatchArgs &b, cudaStream_t s);
// smallest squared site distance into *min_dist2, the front in `mode`, then
// the dense n x n matrices V of the batch into V (count x n x n)
cudaError_t launch_covariance(const BatchArgs &b, FrontMode mode, double *min_dist2, double *V, cudaStream_t s);   // closed form from FP64 tile (nb, nb)
// Buffers of the mixed-precision path (per batch slot w unless noted).
struct MixedArgs {
    uint8_t *wimg;       // count x img: slices of L_JJ^-1
    uint8_t *pimg;       // count x (nb + 1) x img: slices of the current panel
    double *invsum;      // count: sum of 1 / pivot
    int *flags;          // count: 1 = re-evaluate with 7 slices
    int *err;            // 1: set by a kernel whose bounded wait gave up
    double *err_bound;   // K (global output, may be NULL)
    double tol;          // retry when the bound exceeds this
    int early;           // 5-slice pass: stop work on a point once its partial bound exceeds tol
};
size_t mixed_img_bytes(int S);
size_t mixed_slot_bytes();   // panel slot of one tile row
cudaError_t launch_mixed_batch(const BatchArgs &b, const MixedArgs &x, int S, cudaStream_t s);
// the batch after launch_front(b, s, FRONT_DF or FRONT_DF_FAST): factorisation, closed form, error bound
cudaError_t launch_mixed_back(const BatchArgs &b, const MixedArgs &x, int S, cudaStream_t s);
// Wait-cycle counters of the 5-slice trailing update (3 launch modes x 9;
// cudaErrorNotSupported unless built with -DPLK_PIPE_COUNTERS)
cudaError_t pipe_counters(unsigned long long *out, int reset);
// sets the graph conditional h to (*count > 0) on the device
cudaError_t launch_set_condition(cudaGraphConditionalHandle h, const int *count, cudaStream_t s);
// out_idx[j] = output row of the j-th slot w < min(count, *live) with flags[w]
// set (map[w], or k0 + w), *out_count = their number; one block, slot order
cudaError_t launch_compact_flags(int count, const int *flags, const int *live, int64_t k0, const int *map,
                                 int *out_idx, int *out_count, cudaStream_t s);
// dcount (device, optional): only entries 0 .. *dcount - 1 of the count
cudaError_t launch_gather_params(int count, const int *idx, const double *params, double *out, cudaStream_t s,
                                 const int *dcount = nullptr);
// one block whose bounded wait on a barrier that nothing completes gives up and sets *err
cudaError_t launch_wait_selftest(uint32_t max_iter, int *err, cudaStream_t s);
// yh + yl = exp(xh + xl) by the double-float exp of the first-pass rho table
cudaError_t launch_df_exp_selftest(int64_t count, const float *xh, const float *xl, float *yh, float *yl,
                                   cudaStream_t s);
cudaError_t launch_scatter_value(int count, const int *idx, double v, double *out, cudaStream_t s,
                                 const int *dcount = nullptr);

cudaError_t launch_profile_max(const double *vals, int64_t G, int64_t SM, double *prof,
                               cudaStream_t s);
cudaError_t launch_profile_ci(const double *grid, const double *prof, int64_t G, double half_q,
                              double *out, cudaStream_t s);

}  // namespace plk
