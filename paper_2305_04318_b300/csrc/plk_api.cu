// plk_api.cu -- host side of the C ABI declared in include/plk.h.
//
// Stateless evaluation (plk_eval_device) lays out a caller-provided workspace
// and enqueues the kernel pipeline batch by batch.  The context API keeps
// datasets resident in a device arena, admits jobs by the arena bytes their
// batches need, and runs a scheduler thread that launches batches of any active
// job on a pool of streams (continuous batching: a job submitted while others
// are running gets the next free stream slot and arena space; results are
// independent of the mix because each point's arithmetic order depends only on
// its own data).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <random>
#include <string>
#include <thread>
#include <vector>

#include "plk.h"
#include "plk_common.cuh"
#include "plk_kernels.cuh"

using namespace plk;

// Points per part of the mixed path's overlapped first pass (two diagonal-tile
// blocks per SM of a 148-SM B300); a build-time constant.
#ifndef PLK_MIXED_PART
#define PLK_MIXED_PART 296
#endif

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static plk_status fail(plk_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return s;
}

static plk_status cuda_fail(cudaError_t e, const char *where) {
    return fail(PLK_E_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

extern "C" const char *plk_last_error(void) { return g_err.c_str(); }

void plk::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

// ---------------------------------------------------------------------------
// workspace layout
// ---------------------------------------------------------------------------
namespace {

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

struct Layout {
    int64_t n = 0, n_pad = 0;
    int nb = 0, q = 0, p = 0, M = 0, batch = 0;
    int64_t tpo = 0;
    size_t off_Bt = 0, off_sumlog = 0, off_oc = 0, off_coordT = 0, off_tab = 0, off_tiles = 0,
           off_inv = 0, off_ldv = 0, off_pst = 0, off_owner = 0, total = 0;
    // mixed precision only
    bool mixed = false;
    size_t img = 0, off_wimg = 0, off_pimg = 0, off_invsum = 0, off_flags = 0, off_idx = 0,
           off_cparams = 0, off_err = 0, off_idx2 = 0, off_cnt = 0;
};

bool sizes_ok(int64_t n, int32_t p, int32_t M) {
    return n > 0 && p >= 1 && p <= 16 && M >= 1 && M + p <= 64 && n > p;
}

bool make_layout(int64_t n, int32_t p, int32_t M, int32_t batch, Layout &L, int precision = PLK_FP64) {
    if (!sizes_ok(n, p, M) || batch < 1 || batch > 65535) return false;   // batch is a grid dimension
    if (precision != PLK_FP64 && precision != PLK_MIXED) return false;
    L.n = n;
    L.p = p;
    L.M = M;
    L.q = M + p;
    L.batch = batch;
    L.nb = (int)((n + TB - 1) / TB);
    L.n_pad = (int64_t)L.nb * TB;
    L.tpo = tiles_per_omega(L.nb);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.off_Bt = take(sizeof(double) * (size_t)L.q * L.n_pad);
    L.off_sumlog = take(2 * sizeof(double));   // sum log y, smallest squared site distance
    L.off_oc = take(sizeof(double) * OC_N * (size_t)batch);
    L.off_coordT = take(sizeof(double) * 2 * (size_t)L.n_pad * batch);
    L.off_tab = take(sizeof(double) * (size_t)TAB_SIZE * batch);
    L.off_tiles = take(sizeof(double) * (size_t)NT * L.tpo * batch);
    L.off_inv = take(sizeof(double) * (size_t)NT * batch);
    L.off_ldv = take(sizeof(double) * (size_t)batch);
    L.off_pst = take(sizeof(int) * (size_t)batch);
    L.off_owner = take(sizeof(int) * (size_t)batch);
    if (precision == PLK_MIXED) {
        L.mixed = true;
        L.img = align_up(mixed_img_bytes(7));   // L_JJ^-1 image, sized for the 7-slice pass
        L.off_wimg = take(L.img * batch);
        L.off_pimg = take(align_up(mixed_slot_bytes()) * (size_t)(L.nb + 1) * batch);
        L.off_invsum = take(sizeof(double) * (size_t)batch);
        L.off_flags = take(sizeof(int) * (size_t)batch);
        L.off_idx = take(sizeof(int) * (size_t)batch);
        L.off_cparams = take(sizeof(double) * 5 * (size_t)batch);
        L.off_err = take(sizeof(int));
        L.off_idx2 = take(sizeof(int) * (size_t)batch);   // the FP64 tier's points
        L.off_cnt = take(2 * sizeof(int));                 // device-side counts of the two tiers
    }
    L.total = off;
    return true;
}

int default_batch(int64_t n, int64_t K) {
    // enough points in flight to fill 148 SMs in the per-tile kernels while
    // keeping the workspace modest: ~8 GB of tiles
    Layout L;
    if (!make_layout(n, 1, 1, 1, L)) return 1;
    const double per = (double)L.tpo * NT * sizeof(double);
    int64_t b = (int64_t)(8e9 / per);
    b = std::max<int64_t>(1, std::min<int64_t>(b, 296));
    if (K > 0) b = std::min<int64_t>(b, K);
    return (int)b;
}

template <class T>
T *at(void *base, size_t off) {
    return reinterpret_cast<T *>(static_cast<char *>(base) + off);
}

}  // namespace

extern "C" size_t plk_eval_workspace_bytes(int64_t n, int32_t p, int32_t M, int32_t batch,
                                           int32_t precision) {
    Layout L;
    if (!make_layout(n, p, M, batch, L, precision)) return 0;
    return L.total;
}

// ---------------------------------------------------------------------------
// optional per-launch event timing
// ---------------------------------------------------------------------------
namespace {
class EventTimer : public KernelTimer {
  public:
    void begin(int cls, cudaStream_t s) override {
        std::lock_guard<std::mutex> lk(mu_);
        Pending p;
        p.cls = cls;
        p.a = get();
        p.b = get();
        cudaEventRecord(p.a, s);
        open_[s] = p;
    }
    void end(int cls, cudaStream_t s) override {
        std::lock_guard<std::mutex> lk(mu_);
        auto it = open_.find(s);
        if (it == open_.end()) return;
        cudaEventRecord(it->second.b, s);
        pending_.push_back(it->second);
        open_.erase(it);
    }
    void collect(double *ms, int64_t *cnt, int n, bool reset) {
        std::lock_guard<std::mutex> lk(mu_);
        for (auto &p : pending_) {
            float t = 0.f;
            cudaEventSynchronize(p.b);
            cudaEventElapsedTime(&t, p.a, p.b);
            tot_[p.cls] += t;
            num_[p.cls] += 1;
            pool_.push_back(p.a);
            pool_.push_back(p.b);
        }
        pending_.clear();
        for (int c = 0; c < n && c < KC_COUNT; ++c) {
            if (ms) ms[c] = tot_[c];
            if (cnt) cnt[c] = num_[c];
        }
        if (reset)
            for (int c = 0; c < KC_COUNT; ++c) tot_[c] = 0.0, num_[c] = 0;
    }

  private:
    struct Pending {
        int cls;
        cudaEvent_t a, b;
    };
    cudaEvent_t get() {
        if (!pool_.empty()) {
            cudaEvent_t e = pool_.back();
            pool_.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    std::mutex mu_;
    std::vector<cudaEvent_t> pool_;
    std::vector<Pending> pending_;
    std::map<cudaStream_t, Pending> open_;
    double tot_[KC_COUNT] = {};
    int64_t num_[KC_COUNT] = {};
};
EventTimer g_timer;
}  // namespace

extern "C" plk_status plk_kernel_timing(double *total_ms, int64_t *launches, int32_t n_classes,
                                        int32_t reset, int32_t *n_defined) {
    if (n_classes < 0) return fail(PLK_E_INVALID, "n_classes < 0");
    g_timer.collect(total_ms, launches, n_classes, reset != 0);
    if (n_defined) *n_defined = KC_COUNT;
    return PLK_OK;
}

extern "C" const char *plk_kernel_class_name(int32_t c) { return kernel_class_name(c); }

// Mixed precision: 5-slice pass over the batch, then (unless PLK_FLAG_NO_RETRY)
// a 7-slice pass over the points whose error bound exceeded the tolerance or
// whose factorisation failed.  Deciding the retry set reads the flags back, so
// this synchronizes the stream once per batch.
// bound on |Delta log L| above which a mixed-precision point is re-evaluated
static std::atomic<double> g_mixed_tol{1e-3};

// Slots [off, off + cnt) of a mixed batch as a batch of their own.
static void sub_batch(const BatchArgs &b, const MixedArgs &x, int off, int cnt, BatchArgs &bo, MixedArgs &xo) {
    bo = b;
    xo = x;
    bo.count = cnt;
    bo.k0 = b.k0 + off;
    bo.params = b.params + 5 * (size_t)off;
    bo.oconst = b.oconst + (size_t)OC_N * off;
    bo.coordT = b.coordT + (size_t)2 * b.n_pad * off;
    bo.tab = b.tab + (size_t)TAB_SIZE * off;
    bo.tiles = b.tiles + (size_t)b.tpo * NT * off;
    bo.inv = b.inv + (size_t)NT * off;
    bo.ldv = b.ldv + off;
    bo.pstatus = b.pstatus + off;
    bo.owner = b.owner ? b.owner + off : nullptr;
    xo.wimg = x.wimg + mixed_img_bytes(5) * (size_t)off;   // slot stride of the 5-slice pass
    xo.pimg = x.pimg + mixed_slot_bytes() * (size_t)(b.nb + 1) * off;
    xo.invsum = x.invsum + off;
    xo.flags = x.flags + off;
}

// Streams of the calling thread on the current device, created on first use
// and kept for the thread's lifetime: hi at the highest priority (the
// factorisation), lo at the lowest (the overlapped build), re at the lowest
// (the 7-slice re-evaluation of finished parts), cp for reading flags back.
// With the build and the re-evaluation on low-priority streams, the block
// scheduler hands freed SM resources to the factorisation kernels first.
struct AuxStreams {
    cudaStream_t hi = nullptr, lo = nullptr, re = nullptr, cp = nullptr;
};
static AuxStreams aux_streams() {
    struct Table {
        std::map<int, AuxStreams> m;
        ~Table() {
            for (auto &kv : m)
                for (cudaStream_t x : {kv.second.hi, kv.second.lo, kv.second.re, kv.second.cp})
                    if (x) cudaStreamDestroy(x);
        }
    };
    thread_local Table t;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return {};
    auto it = t.m.find(dev);
    if (it != t.m.end()) return it->second;
    int least = 0, greatest = 0;
    AuxStreams st;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return {};
    const bool ok = cudaStreamCreateWithPriority(&st.hi, cudaStreamNonBlocking, greatest) == cudaSuccess &&
                    cudaStreamCreateWithPriority(&st.lo, cudaStreamNonBlocking, least) == cudaSuccess &&
                    cudaStreamCreateWithPriority(&st.re, cudaStreamNonBlocking, least) == cudaSuccess &&
                    cudaStreamCreateWithFlags(&st.cp, cudaStreamNonBlocking) == cudaSuccess;
    if (!ok) {
        for (cudaStream_t x : {st.hi, st.lo, st.re, st.cp})
            if (x) cudaStreamDestroy(x);
        return {};
    }
    t.m[dev] = st;
    return st;
}

// Launches the sequence `enqueue` puts on stream s as one CUDA graph: the
// sequence is captured from s (thread-local capture mode, so other threads'
// CUDA calls are unaffected), and the executable graph this thread keeps for s
// is updated in place when the capture has the same topology (only kernel
// arguments changed, as between batches of one shape), else instantiated anew.
template <class F>
static cudaError_t launch_as_graph(cudaStream_t s, F &&enqueue) {
    struct Cache {
        std::map<std::pair<int, cudaStream_t>, cudaGraphExec_t> m;
        ~Cache() {
            for (auto &kv : m)
                if (kv.second) cudaGraphExecDestroy(kv.second);
        }
    };
    thread_local Cache cache;
    if (s == nullptr || s == cudaStreamLegacy) return enqueue();   // the legacy stream cannot be captured
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    const cudaError_t le = enqueue();
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(s, &g);
    if (le != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return le != cudaSuccess ? le : e;
    }
    cudaGraphExec_t &x = cache.m[{dev, s}];
    if (x) {
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(x, g, &info) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaGraphExecDestroy(x);
            x = nullptr;
        }
    }
    if (!x) e = cudaGraphInstantiate(&x, g, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(x, s);
    cudaGraphDestroy(g);
    return e;
}

static bool use_graph(int flags) { return (flags & PLK_FLAG_GRAPH) && !(flags & PLK_FLAG_KERNEL_TIMING); }

// A stream of this thread for capturing conditional bodies (created outside
// any capture, on first use per device).
static cudaStream_t body_stream() {
    thread_local std::map<int, cudaStream_t> m;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    cudaStream_t &x = m[dev];
    if (!x && cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) x = nullptr;
    return x;
}

// Inside a capture of s: the work `body` enqueues on the stream it is given
// becomes the body of a conditional node that runs only when *count > 0 at
// that point of the graph (the condition is set on the device by a one-thread
// kernel), so a device-side count decides without a host read-back.
template <class F>
static cudaError_t enqueue_if_positive(cudaStream_t s, const int *count, F &&body) {
    cudaStream_t bs = body_stream();
    if (!bs) return cudaErrorNotReady;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd);
    if (e != cudaSuccess) return e;
    if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureUnmatched;
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) return e;
    if ((e = launch_set_condition(h, count, s)) != cudaSuccess) return e;
    if ((e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd)) != cudaSuccess) return e;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, edges, nd, &p)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies)) !=
        cudaSuccess)
        return e;
    if ((e = cudaStreamBeginCaptureToGraph(bs, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
        return e;
    const cudaError_t le = body(bs);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(bs, &out);
    return le != cudaSuccess ? le : e;
}
// Small datasets go through the fused one-CTA-per-point kernel in either
// precision (FP64 there costs less than the tiled tensor-core path).
static bool use_fused(int64_t n, int q, int flags) { return fused_applies(n, q) && !(flags & PLK_FLAG_NO_FUSED); }

// 5-slice pass over the batch.  With `overlap` and enough points, the batch is
// cut into parts of about 296 points (two diagonal-tile blocks per SM); the
// front of every part after the first (prep, table, build: FP64 pipe, no
// shared memory) runs on a low-priority stream beside the factorisations of
// the earlier parts (tensor cores) on a high-priority stream, so only the first
// part's build is exposed.  The work is forked from `s` onto the two internal
// streams and joined back into `s`.
constexpr int kOverlapMin = 256, kPart = PLK_MIXED_PART;
static int first_pass_parts(int count) { return std::max(2, (count + kPart - 1) / kPart); }

// part_done (optional): one event per part, recorded on the factorisation
// stream when that part's pass (closed form and error bound included) is done;
// the caller destroys them.
static cudaError_t mixed_first_pass(const BatchArgs &b, const MixedArgs &x, bool overlap, cudaStream_t s,
                                    std::vector<cudaEvent_t> *part_done = nullptr) {
    const AuxStreams st = overlap && b.count >= kOverlapMin ? aux_streams() : AuxStreams{};
    if (!st.hi) return launch_mixed_batch(b, x, 5, s);
    const int nparts = first_pass_parts(b.count);
    std::vector<cudaEvent_t> ev(nparts + 2, nullptr);   // [0] fork, [1 + p] front of part p done, [nparts + 1] join
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < ev.size() && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    auto part = [&](int p, BatchArgs &bp, MixedArgs &xp) {
        const int lo = (int)((int64_t)b.count * p / nparts), hi = (int)((int64_t)b.count * (p + 1) / nparts);
        sub_batch(b, x, lo, hi - lo, bp, xp);
    };
    bool forked = false;
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st.hi, ev[0], 0);
    forked = e == cudaSuccess;
    for (int p = 0; p < nparts && e == cudaSuccess; ++p) {   // fronts: part 0 on hi, the rest on lo
        BatchArgs bp;
        MixedArgs xp;
        part(p, bp, xp);
        cudaStream_t fs = p == 0 ? st.hi : st.lo;
        if (p == 1) e = cudaStreamWaitEvent(st.lo, ev[1], 0);
        if (e == cudaSuccess) e = launch_front(bp, fs, FRONT_DF_FAST);
        if (e == cudaSuccess) e = cudaEventRecord(ev[1 + p], fs);
    }
    for (int p = 0; p < nparts && e == cudaSuccess; ++p) {   // factorisations, in order, on hi
        BatchArgs bp;
        MixedArgs xp;
        part(p, bp, xp);
        if (p > 0) e = cudaStreamWaitEvent(st.hi, ev[1 + p], 0);
        if (e == cudaSuccess) e = launch_mixed_back(bp, xp, 5, st.hi);
        if (e == cudaSuccess && part_done) {
            cudaEvent_t d = nullptr;
            e = cudaEventCreateWithFlags(&d, cudaEventDisableTiming);
            if (e == cudaSuccess) part_done->push_back(d);
            if (e == cudaSuccess) e = cudaEventRecord(d, st.hi);
        }
    }
    if (forked) {   // join, also after a failed launch: nothing may run on past `s`
        cudaEventRecord(ev[nparts], st.lo);
        cudaStreamWaitEvent(st.hi, ev[nparts], 0);
        const cudaError_t j = cudaEventRecord(ev[nparts + 1], st.hi);
        const cudaError_t k = j == cudaSuccess ? cudaStreamWaitEvent(s, ev[nparts + 1], 0) : j;
        if (e == cudaSuccess) e = k;
    }
    for (auto &v : ev)
        if (v) cudaEventDestroy(v);   // released once the recorded work completes
    return e;
}

// FP64 tier: the points idx (global indices) re-evaluated in FP64, in slots
// 0 .. of the batch workspace (every earlier pass of the batch has finished).
static plk_status fp64_tier(const BatchArgs &b, const Layout &L, void *ws, const double *params_all,
                            double *err_bound, const std::vector<int> &idx2, cudaStream_t s) {
    if (idx2.empty()) return PLK_OK;
    int *d_idx = at<int>(ws, L.off_idx);
    double *d_par = at<double>(ws, L.off_cparams);
    cudaError_t e = cudaMemcpyAsync(d_idx, idx2.data(), sizeof(int) * idx2.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_gather_params((int)idx2.size(), d_idx, params_all, d_par, s);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 retry gather");
    BatchArgs f = b;
    f.count = (int)idx2.size();
    f.params = d_par;
    f.out_index = d_idx;
    f.status_or = PLK_POINT_RETRIED | PLK_POINT_FP64;
    e = launch_fp64_batch(f, s);
    if (e == cudaSuccess && err_bound) e = launch_scatter_value(f.count, d_idx, 0.0, err_bound, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // idx2 must outlive its copy
    if (e != cudaSuccess) return cuda_fail(e, "fp64 retry");
    return PLK_OK;
}

// The 5-slice pass in parts (mixed_first_pass) with the 7-slice tier
// pipelined behind it: as soon as a part is done, its flags are read back and
// its points bound for 7 slices are re-evaluated on the low-priority stream,
// in that part's own workspace slots, while the later parts' passes run on
// the high-priority stream (the re-evaluation fills the SMs their
// latency-bound diagonal-tile and panel kernels leave idle).  The FP64 tier,
// if any point needs it, follows once everything else is done.  Results are
// those of the sequential order: every point's arithmetic depends only on its
// own data.
static plk_status run_mixed_pipelined(const BatchArgs &b, const Layout &L, void *ws, const MixedArgs &x,
                                      const double *params_all, int flags, double *err_bound, cudaStream_t s) {
    const AuxStreams st = aux_streams();
    const int nparts = first_pass_parts(b.count);
    std::vector<cudaEvent_t> done;
    cudaEvent_t joined = nullptr;
    auto cleanup = [&]() {
        for (cudaEvent_t ev : done) cudaEventDestroy(ev);
        if (joined) cudaEventDestroy(joined);
    };
    cudaError_t e = cudaMemsetAsync(x.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = mixed_first_pass(b, x, true, s, &done);
    if (e == cudaSuccess && (int)done.size() != nparts) e = cudaErrorInvalidValue;
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "mixed batch launch");
    }
    int *d_idx = at<int>(ws, L.off_idx);
    double *d_par = at<double>(ws, L.off_cparams);
    std::vector<std::vector<int>> idx(nparts);   // kept until the copies from them are done
    std::vector<int> h;
    int dev_err = 0;
    bool retried = false;
    for (int p = 0; p < nparts && e == cudaSuccess; ++p) {
        const int lo = (int)((int64_t)b.count * p / nparts), cnt = (int)((int64_t)b.count * (p + 1) / nparts) - lo;
        h.assign(cnt + 1, 0);
        e = cudaStreamWaitEvent(st.cp, done[p], 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), x.flags + lo, sizeof(int) * cnt, cudaMemcpyDeviceToHost, st.cp);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data() + cnt, x.err, sizeof(int), cudaMemcpyDeviceToHost, st.cp);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st.cp);   // waits for part p only
        if (e != cudaSuccess) break;
        if (h[cnt]) dev_err = 1;
        for (int w = 0; w < cnt; ++w)
            if (h[w]) idx[p].push_back((int)(b.k0 + lo + w));
        if (idx[p].empty() || dev_err) continue;
        BatchArgs r;
        MixedArgs xr;
        sub_batch(b, x, lo, (int)idx[p].size(), r, xr);
        r.params = d_par + 5 * (size_t)lo;
        r.out_index = d_idx + lo;
        r.status_or = PLK_POINT_RETRIED;
        e = cudaStreamWaitEvent(st.re, done[p], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_idx + lo, idx[p].data(), sizeof(int) * idx[p].size(), cudaMemcpyHostToDevice, st.re);
        if (e == cudaSuccess) e = launch_gather_params(r.count, d_idx + lo, params_all, d_par + 5 * (size_t)lo, st.re);
        if (e == cudaSuccess) e = launch_mixed_batch(r, xr, 7, st.re);
        retried = true;
    }
    // join the re-evaluation back into s, also after a failed launch
    cudaError_t j = cudaEventCreateWithFlags(&joined, cudaEventDisableTiming);
    if (j == cudaSuccess) j = cudaEventRecord(joined, st.re);
    if (j == cudaSuccess) j = cudaStreamWaitEvent(s, joined, 0);
    if (e == cudaSuccess) e = j;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "mixed batch");
    }
    std::vector<int> idx2;
    if (retried && !dev_err) {
        for (int p = 0; p < nparts && e == cudaSuccess; ++p) {
            if (idx[p].empty()) continue;
            const int lo = (int)((int64_t)b.count * p / nparts), m = (int)idx[p].size();
            h.assign(m + 1, 0);
            e = cudaMemcpyAsync(h.data(), x.flags + lo, sizeof(int) * m, cudaMemcpyDeviceToHost, st.cp);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h.data() + m, x.err, sizeof(int), cudaMemcpyDeviceToHost, st.cp);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st.cp);
            if (e == cudaSuccess && h[m]) dev_err = 1;
            if (!(flags & PLK_FLAG_NO_FP64_TIER))
                for (int w = 0; w < m; ++w)
                    if (h[w]) idx2.push_back(idx[p][w]);
        }
    }
    cleanup();
    if (e != cudaSuccess) return cuda_fail(e, "mixed retry");
    if (dev_err) return fail(PLK_E_TIMEOUT, "a tensor-core wait gave up (device error flag set)");
    return fp64_tier(b, L, ws, params_all, err_bound, idx2, s);
}

static plk_status run_mixed_batch(BatchArgs b, const Layout &L, void *ws, const double *params_all, int flags,
                                  double *err_bound, bool overlap, cudaStream_t s) {
    MixedArgs x;
    x.wimg = at<uint8_t>(ws, L.off_wimg);
    x.pimg = at<uint8_t>(ws, L.off_pimg);
    x.invsum = at<double>(ws, L.off_invsum);
    x.flags = at<int>(ws, L.off_flags);
    x.err = at<int>(ws, L.off_err);
    x.err_bound = err_bound;
    x.tol = g_mixed_tol.load();
    // without the retry the caller gets every point's 5-slice result
    x.early = (flags & (PLK_FLAG_NO_RETRY | PLK_FLAG_FULL_FIRST_PASS)) ? 0 : 1;
    if ((flags & PLK_FLAG_PIPELINED_RETRY) && overlap && b.count >= kOverlapMin && !use_graph(flags) &&
        !(flags & PLK_FLAG_NO_RETRY) && aux_streams().re)
        return run_mixed_pipelined(b, L, ws, x, params_all, flags, err_bound, s);
    // The batch up to its 7-slice tier is one asynchronous sequence (one CUDA
    // graph with PLK_FLAG_GRAPH): the 5-slice pass; on the device, the
    // compaction of the points whose bound it flags and the gather of their
    // parameters; the 7-slice pass over them, launched over the batch's slots
    // with the device-side count deciding which are live; the compaction of the
    // points still flagged.  No decision reads the flags back.  As a graph,
    // the FP64 pass over those points is the body of a conditional node that
    // runs only when their count is positive (set on the device).  Eagerly,
    // the one read at the end takes the device error flag (a tensor-core wait
    // that gave up) and that count, and in the rare batch where it is not
    // zero the FP64 pass follows over exactly those points (launched
    // unconditionally over the whole batch, it would cost ~2 % of a step in
    // empty thread blocks).
    int *d_idx = at<int>(ws, L.off_idx), *d_idx2 = at<int>(ws, L.off_idx2), *d_cnt = at<int>(ws, L.off_cnt);
    double *d_par = at<double>(ws, L.off_cparams);
    const bool fp64_tier = !(flags & (PLK_FLAG_NO_RETRY | PLK_FLAG_NO_FP64_TIER));
    // a graph only where launch_as_graph captures (not on the legacy stream)
    const bool graph = use_graph(flags) && s != nullptr && s != cudaStreamLegacy;
    auto seq = [&]() {
        cudaError_t e = cudaMemsetAsync(x.err, 0, sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 2 * sizeof(int), s);
        if (e == cudaSuccess) e = mixed_first_pass(b, x, overlap, s);
        if (e != cudaSuccess || (flags & PLK_FLAG_NO_RETRY)) return e;
        e = launch_compact_flags(b.count, x.flags, nullptr, b.k0, nullptr, d_idx, d_cnt, s);
        if (e == cudaSuccess) e = launch_gather_params(b.count, d_idx, params_all, d_par, s, d_cnt);
        if (e != cudaSuccess) return e;
        BatchArgs r = b;
        r.params = d_par;
        r.out_index = d_idx;
        r.status_or = PLK_POINT_RETRIED;
        r.dcount = d_cnt;
        e = launch_mixed_batch(r, x, 7, s);   // flags[j] <- the 7-slice verdict of live slot j
        if (e == cudaSuccess && fp64_tier)
            e = launch_compact_flags(b.count, x.flags, d_cnt, 0, d_idx, d_idx2, d_cnt + 1, s);
        if (e == cudaSuccess && fp64_tier && graph)   // the FP64 tier inside the graph, run if its count > 0
            e = enqueue_if_positive(s, d_cnt + 1, [&](cudaStream_t bs) {
                BatchArgs f = b;
                f.params = d_par;
                f.out_index = d_idx2;
                f.status_or = PLK_POINT_RETRIED | PLK_POINT_FP64;
                f.dcount = d_cnt + 1;
                cudaError_t fe = launch_gather_params(b.count, d_idx2, params_all, d_par, bs, d_cnt + 1);
                if (fe == cudaSuccess) fe = launch_fp64_batch(f, bs);
                if (fe == cudaSuccess && err_bound) fe = launch_scatter_value(b.count, d_idx2, 0.0, err_bound, bs, d_cnt + 1);
                return fe;
            });
        return e;
    };
    if (graph) {   // create the helper streams outside the capture
        if (overlap) aux_streams();
        body_stream();
    }
    cudaError_t e = graph ? launch_as_graph(s, seq) : seq();
    if (e != cudaSuccess) return cuda_fail(e, "mixed batch launch");
    int h[3] = {0, 0, 0};   // error flag, counts of the 7-slice and FP64 tiers
    e = cudaMemcpyAsync(h, x.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h + 1, d_cnt, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "mixed batch");
    if (h[0]) return fail(PLK_E_TIMEOUT, "a tensor-core wait gave up (device error flag set)");
    if (!fp64_tier || graph || h[2] == 0) return PLK_OK;   // in a graph the tier has run already
    BatchArgs f = b;
    f.count = h[2];
    f.params = d_par;
    f.out_index = d_idx2;
    f.status_or = PLK_POINT_RETRIED | PLK_POINT_FP64;
    e = launch_gather_params(f.count, d_idx2, params_all, d_par, s);
    if (e == cudaSuccess) e = launch_fp64_batch(f, s);
    if (e == cudaSuccess && err_bound) e = launch_scatter_value(f.count, d_idx2, 0.0, err_bound, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "fp64 retry");
    return PLK_OK;
}

// Mixed precision on a small dataset: the fused kernel in double-float FP32
// over the batch, its a-posteriori bound per point, then (unless
// PLK_FLAG_NO_RETRY) the fused FP64 kernel on the points whose bound exceeded
// the tolerance or whose factorisation failed (status bits RETRIED | FP64,
// err_bound 0), gated on the device by the bound's flags: one asynchronous
// sequence with no host read-back (a CUDA graph with PLK_FLAG_GRAPH).
static plk_status run_fused_mixed_batch(BatchArgs b, const Layout &L, void *ws, int flags, double *err_bound,
                                        cudaStream_t s) {
    double *invsum = at<double>(ws, L.off_invsum);
    int *fl = at<int>(ws, L.off_flags);
    auto seq = [&]() {
        cudaError_t e = launch_fused_df_batch(b, invsum, FUSED_DF_EPS, g_mixed_tol.load(), err_bound, fl, s);
        if (e == cudaSuccess && !(flags & PLK_FLAG_NO_RETRY)) e = launch_fused_fp64_gated(b, fl, err_bound, s);
        return e;
    };
    const cudaError_t e = use_graph(flags) ? launch_as_graph(s, seq) : seq();
    if (e != cudaSuccess) return cuda_fail(e, "fused mixed batch");
    return PLK_OK;
}

// Enqueue the whole evaluation on `s` given a laid-out workspace.
static plk_status run_eval(const plk_eval_args *a, int reml, int flags, const Layout &L, void *ws,
                           cudaStream_t s) {
    KernelTimer *timer = (flags & PLK_FLAG_KERNEL_TIMING) ? &g_timer : nullptr;
    const bool fused = use_fused(a->n, L.q, flags);
    cudaError_t e = launch_boxcox(a->n, L.n_pad, a->p, a->M, a->y, a->X, a->coords, a->lambdas,
                                  at<double>(ws, L.off_Bt), at<double>(ws, L.off_sumlog), s, timer);
    if (e != cudaSuccess) return cuda_fail(e, "boxcox launch");
    for (int64_t k0 = 0; k0 < a->K; k0 += L.batch) {
        BatchArgs b;
        b.count = (int)std::min<int64_t>(L.batch, a->K - k0);
        b.k0 = k0;
        b.n = a->n;
        b.n_pad = L.n_pad;
        b.nb = L.nb;
        b.q = L.q;
        b.p = a->p;
        b.M = a->M;
        b.reml = reml;
        b.tpo = L.tpo;
        b.params = a->params + 5 * k0;
        b.coords = a->coords;
        b.lambdas = a->lambdas;
        b.Bt = at<double>(ws, L.off_Bt);
        b.sumlogy = at<double>(ws, L.off_sumlog);
        b.oconst = at<double>(ws, L.off_oc);
        b.coordT = at<double>(ws, L.off_coordT);
        b.tab = at<double>(ws, L.off_tab);
        b.tiles = at<double>(ws, L.off_tiles);
        b.inv = at<double>(ws, L.off_inv);
        b.ldv = at<double>(ws, L.off_ldv);
        b.pstatus = at<int>(ws, L.off_pst);
        b.owner = at<int>(ws, L.off_owner);
        b.logL = a->logL;
        b.sigma2 = a->sigma2;
        b.beta = a->beta;
        b.logdet = a->logdet;
        b.ssq = a->ssq_yx;
        b.status = a->status;
        b.timer = timer;
        if (fused && L.mixed) {
            plk_status st = run_fused_mixed_batch(b, L, ws, flags, a->err_bound, s);
            if (st != PLK_OK) return st;
        } else if (fused) {
            e = use_graph(flags) ? launch_as_graph(s, [&]() { return launch_fused_batch(b, s); })
                                 : launch_fused_batch(b, s);
            if (e != cudaSuccess) return cuda_fail(e, "fused batch launch");
        } else if (L.mixed) {
            plk_status st = run_mixed_batch(b, L, ws, a->params, flags, a->err_bound, true, s);
            if (st != PLK_OK) return st;
        } else {
            e = use_graph(flags) ? launch_as_graph(s, [&]() { return launch_fp64_batch(b, s); })
                                 : launch_fp64_batch(b, s);
            if (e != cudaSuccess) return cuda_fail(e, "batch launch");
        }
    }
    if (!L.mixed && a->err_bound) {
        e = cudaMemsetAsync(a->err_bound, 0, sizeof(double) * a->K, s);
        if (e != cudaSuccess) return cuda_fail(e, "err_bound");
    }
    return PLK_OK;
}

static plk_status check_args(const plk_eval_args *a) {
    if (!a) return fail(PLK_E_INVALID, "args is NULL");
    if (!sizes_ok(a->n, a->p, a->M))
        return fail(PLK_E_INVALID, "invalid sizes n=%lld p=%d M=%d (need n > p >= 1, p <= 16, M >= 1, M+p <= 64)",
                    (long long)a->n, a->p, a->M);
    if (a->K < 0) return fail(PLK_E_INVALID, "K < 0");
    if (!a->coords || !a->y || !a->X || !a->lambdas || (a->K > 0 && !a->params))
        return fail(PLK_E_INVALID, "NULL input pointer");
    return PLK_OK;
}

extern "C" plk_status plk_eval_device(const plk_eval_args *args, const plk_options *opts,
                                      void *workspace, size_t workspace_bytes, void *stream) {
    plk_status st = check_args(args);
    if (st != PLK_OK) return st;
    const int prec = opts ? opts->precision : PLK_FP64;
    if (prec != PLK_FP64 && prec != PLK_MIXED) return fail(PLK_E_INVALID, "unknown precision %d", prec);
    int batch = (opts && opts->batch > 0) ? opts->batch : default_batch(args->n, args->K);
    Layout L;
    if (!make_layout(args->n, args->p, args->M, batch, L, prec))
        return fail(PLK_E_INVALID, "batch %d outside [1, 65535]", batch);
    if (!workspace || workspace_bytes < L.total)
        return fail(PLK_E_NOMEM, "workspace of %zu bytes < %zu needed for batch %d", workspace_bytes,
                    L.total, batch);
    if (reinterpret_cast<uintptr_t>(workspace) % ALIGN != 0)
        return fail(PLK_E_INVALID, "workspace must be 256-byte aligned");
    if (args->K == 0) return PLK_OK;
    return run_eval(args, opts ? opts->reml : 0, opts ? opts->flags : 0, L, workspace,
                    static_cast<cudaStream_t>(stream));
}

extern "C" plk_status plk_build_covariance_device(const double *coords, int64_t n, const double *params, int64_t K,
                                                  int32_t mode, double *V, void *workspace, size_t workspace_bytes,
                                                  void *stream) {
    if (!coords || !params || !V) return fail(PLK_E_INVALID, "NULL pointer");
    if (n < 2 || K < 1 || K > 65535) return fail(PLK_E_INVALID, "need n >= 2 and 1 <= K <= 65535");
    if (mode < 0 || mode > 2) return fail(PLK_E_INVALID, "unknown build mode %d", mode);
    Layout L;
    if (!make_layout(n, 1, 1, (int32_t)K, L, PLK_FP64)) return fail(PLK_E_INVALID, "invalid sizes");
    if (!workspace || workspace_bytes < L.total)
        return fail(PLK_E_NOMEM, "workspace of %zu bytes < %zu needed", workspace_bytes, L.total);
    if (reinterpret_cast<uintptr_t>(workspace) % ALIGN != 0)
        return fail(PLK_E_INVALID, "workspace must be 256-byte aligned");
    BatchArgs b{};
    b.count = (int)K;
    b.k0 = 0;
    b.n = n;
    b.n_pad = L.n_pad;
    b.nb = L.nb;
    b.q = 0;   // no right-hand-side rows: the build reads no B^T
    b.p = 1;
    b.M = 1;
    b.tpo = L.tpo;
    b.params = params;
    b.coords = coords;
    b.Bt = at<double>(workspace, L.off_Bt);
    b.sumlogy = at<double>(workspace, L.off_sumlog);
    b.oconst = at<double>(workspace, L.off_oc);
    b.coordT = at<double>(workspace, L.off_coordT);
    b.tab = at<double>(workspace, L.off_tab);
    b.tiles = at<double>(workspace, L.off_tiles);
    b.inv = at<double>(workspace, L.off_inv);
    b.ldv = at<double>(workspace, L.off_ldv);
    b.pstatus = at<int>(workspace, L.off_pst);
    b.owner = at<int>(workspace, L.off_owner);
    const FrontMode fm = mode == 0 ? FRONT_FP64 : (mode == 1 ? FRONT_DF_FAST : FRONT_DF);
    cudaError_t e = launch_covariance(b, fm, at<double>(workspace, L.off_sumlog) + 1, V,
                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PLK_OK : cuda_fail(e, "covariance build");
}

// ---------------------------------------------------------------------------
// profile reduction, CI
// ---------------------------------------------------------------------------
extern "C" double plk_chi2_1_quantile(double level) {
    // c = z^2 with P(|Z| <= z) = level, i.e. erf(z / sqrt 2) = level; Newton on erf
    // from a bisection start.
    if (!(level > 0.0) || !(level < 1.0)) return NAN;
    double lo = 0.0, hi = 40.0;
    for (int i = 0; i < 80; ++i) {
        double mid = 0.5 * (lo + hi);
        if (std::erf(mid / std::sqrt(2.0)) < level) lo = mid; else hi = mid;
    }
    double z = 0.5 * (lo + hi);
    for (int i = 0; i < 3; ++i) {
        const double f = std::erfc(z / std::sqrt(2.0)) - (1.0 - level);
        const double df = -std::sqrt(2.0 / M_PI) * std::exp(-0.5 * z * z);
        if (df == 0.0) break;
        z -= f / df;
    }
    return z * z;
}

extern "C" plk_status plk_profile_max_device(const double *vals, int64_t G, int64_t SM, double *prof,
                                             void *stream) {
    if (G < 0 || SM < 1 || (G > 0 && (!vals || !prof))) return fail(PLK_E_INVALID, "bad profile_max args");
    if (G == 0) return PLK_OK;
    cudaError_t e = launch_profile_max(vals, G, SM, prof, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PLK_OK : cuda_fail(e, "profile_max");
}

extern "C" plk_status plk_profile_ci_device(const double *grid, const double *prof, int64_t G,
                                            double level, double *out, void *stream) {
    if (G < 1 || !grid || !prof || !out || !(level > 0.0 && level < 1.0))
        return fail(PLK_E_INVALID, "bad profile_ci args");
    cudaError_t e = launch_profile_ci(grid, prof, G, 0.5 * plk_chi2_1_quantile(level), out,
                                      static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? PLK_OK : cuda_fail(e, "profile_ci");
}

extern "C" plk_status plk_profile_ci(const double *grid, const double *profile_logL, int64_t G, double level,
                                     double *lo, double *hi, double *argmax, int32_t *censored) {
    if (G < 1 || !grid || !profile_logL || !(level > 0.0 && level < 1.0))
        return fail(PLK_E_INVALID, "bad profile_ci args");
    double *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(double) * (2 * (size_t)G + 4));
    if (e != cudaSuccess) return cuda_fail(e, "profile_ci cudaMalloc");
    double out[4];
    e = cudaMemcpy(d, grid, sizeof(double) * G, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + G, profile_logL, sizeof(double) * G, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_profile_ci(d, d + G, G, 0.5 * plk_chi2_1_quantile(level), d + 2 * G, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * G, sizeof out, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "profile_ci");
    if (lo) *lo = out[0];
    if (hi) *hi = out[1];
    if (argmax) *argmax = out[2];
    if (censored) *censored = out[3] == out[3] ? (int32_t)out[3] : 0;
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// context API
// ---------------------------------------------------------------------------
namespace {

// First-fit sub-allocator over one device arena (256-byte granules).
class Arena {
  public:
    void init(char *base, size_t size) {
        base_ = base;
        size_ = size;
        free_.clear();
        free_[0] = size;
        used_ = high_ = 0;
    }
    char *alloc(size_t bytes) {
        bytes = align_up(std::max<size_t>(bytes, 1));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                live_[off] = bytes;
                used_ += bytes;
                high_ = std::max(high_, used_);
                return base_ + off;
            }
        }
        return nullptr;
    }
    void release(char *p) {
        if (!p) return;
        size_t off = p - base_;
        auto it = live_.find(off);
        if (it == live_.end()) return;
        size_t len = it->second;
        live_.erase(it);
        used_ -= len;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && off + len == nx->first) {
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                pv->second += len;
                return;
            }
        }
        free_[off] = len;
    }
    size_t size() const { return size_; }
    size_t used() const { return used_; }
    size_t high() const { return high_; }

  private:
    char *base_ = nullptr;
    size_t size_ = 0, used_ = 0, high_ = 0;
    std::map<size_t, size_t> free_, live_;
};

struct Dataset {
    int64_t n = 0;
    int32_t p = 0;
    double *coords = nullptr, *y = nullptr, *X = nullptr;
    int active_jobs = 0;
};

struct Job {
    plk_job id = 0;
    plk_dataset ds = 0;
    int64_t K = 0;
    int32_t M = 0, p = 0;
    int64_t n = 0;
    plk_options opts{};
    std::vector<double> params, lambdas;
    // device buffers (from the arena): inputs, outputs
    char *dev = nullptr;
    double *d_params = nullptr, *d_lam = nullptr, *d_logL = nullptr, *d_s2 = nullptr,
           *d_beta = nullptr, *d_ld = nullptr, *d_bt = nullptr, *d_slog = nullptr;
    int32_t *d_st = nullptr;
    cudaEvent_t ready = nullptr;   // B^T and sum log y computed
    int batch = 1;
    int64_t next_k = 0;      // first point not yet launched
    int inflight = 0;
    bool started = false, done = false, failed = false, cancelled = false;
    std::string error;
    std::vector<double> logL, s2, beta, ld;
    std::vector<int32_t> st;
    double t_submit = 0, t_start = 0, t_done = 0;
    std::vector<double> item_s;   // wall time of every batch, launch to completion
};

struct Item {
    Job *job;
    Dataset *ds;
    int64_t k0;
    int count;
    char *ws;
};

}  // namespace

struct plk_ctx {
    int device = 0;
    char *arena_base = nullptr;
    bool own_arena = false;
    Arena arena;
    std::vector<cudaStream_t> streams;
    bool own_streams = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::map<plk_dataset, std::unique_ptr<Dataset>> datasets;
    std::map<plk_job, std::unique_ptr<Job>> jobs;
    std::deque<Job *> order;   // submission order of unfinished jobs
    plk_dataset next_ds = 1;
    plk_job next_job = 1;
    bool stop = false;
    std::vector<std::thread> workers;   // one per stream
    // autotuned points per scheduled batch: (half-octave bucket of n, precision) -> (batch, points/s)
    std::map<std::pair<int, int>, std::pair<int, double>> tuned;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    // host executor (plk_create_with_evaluator): batches run on the worker
    // threads through host_fn, all buffers in host memory
    bool host = false;
    plk_host_eval_fn host_fn = nullptr;
    void *host_user = nullptr;
    // host-side fault hooks (plk_inject_fault): counts of events still to fail
    int fault_arena = 0, fault_item = 0, fault_drop = 0;
    FILE *metrics = nullptr;   // per-job JSON lines (plk_set_metrics_log)
    int policy = PLK_SCHED_FIFO;   // which job's batch a free stream takes next
};

namespace {

size_t job_io_bytes(int64_t K, int32_t M, int32_t p, int64_t n) {
    size_t b = 0;
    b += align_up(sizeof(double) * 5 * K);
    b += align_up(sizeof(double) * M);
    b += align_up(sizeof(double) * K * M) * 2;
    b += align_up(sizeof(double) * K * M * p);
    b += align_up(sizeof(double) * 2 * K);
    b += align_up(sizeof(int32_t) * K);
    b += align_up(sizeof(double) * (size_t)(M + p) * ((n + TB - 1) / TB * TB));   // B^T rows
    b += align_up(sizeof(double));
    return b;
}

// Per-batch workspace without the shared dataset part (B^T, sum log y live in the job).
size_t item_bytes(int64_t n, int32_t p, int32_t M, int count, int precision) {
    Layout L;
    make_layout(n, p, M, count, L, precision);
    return L.total;
}

// Start a job: allocate its I/O, upload inputs, compute B^T once.  Caller holds mu.
bool start_job(plk_ctx *c, Job *j, cudaStream_t s) {
    size_t bytes = job_io_bytes(j->K, j->M, j->p, j->n);
    j->dev = c->arena.alloc(bytes);
    if (!j->dev) return false;
    char *q = j->dev;
    auto take = [&](size_t b) {
        char *r = q;
        q += align_up(b);
        return r;
    };
    j->d_params = (double *)take(sizeof(double) * 5 * j->K);
    j->d_lam = (double *)take(sizeof(double) * j->M);
    j->d_logL = (double *)take(sizeof(double) * j->K * j->M);
    j->d_s2 = (double *)take(sizeof(double) * j->K * j->M);
    j->d_beta = (double *)take(sizeof(double) * j->K * j->M * j->p);
    j->d_ld = (double *)take(sizeof(double) * 2 * j->K);
    j->d_st = (int32_t *)take(sizeof(int32_t) * j->K);
    const int64_t n_pad = (j->n + TB - 1) / TB * TB;
    j->d_bt = (double *)take(sizeof(double) * (size_t)(j->M + j->p) * n_pad);
    j->d_slog = (double *)take(2 * sizeof(double));
    Dataset *d = c->datasets[j->ds].get();
    if (c->host) {   // the evaluator forms the Box-Cox columns itself
        std::memcpy(j->d_params, j->params.data(), sizeof(double) * 5 * j->K);
        std::memcpy(j->d_lam, j->lambdas.data(), sizeof(double) * j->M);
        j->started = true;
        j->t_start = c->now();
        return true;
    }
    cudaMemcpyAsync(j->d_params, j->params.data(), sizeof(double) * 5 * j->K, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(j->d_lam, j->lambdas.data(), sizeof(double) * j->M, cudaMemcpyHostToDevice, s);
    cudaError_t e = launch_boxcox(j->n, n_pad, j->p, j->M, d->y, d->X, d->coords, j->d_lam, j->d_bt, j->d_slog, s);
    if (e != cudaSuccess) {
        j->failed = true;
        j->error = cudaGetErrorString(e);
    }
    cudaEventCreateWithFlags(&j->ready, cudaEventDisableTiming);
    cudaEventRecord(j->ready, s);
    j->started = true;
    j->t_start = c->now();
    return true;
}

// Runs one batch of a job on stream s and waits for it (called without the
// context lock).  Returns an error message, empty on success.
std::string run_item(plk_ctx *c, Job *j, Item &it, cudaStream_t s) {
    if (c->host) {
        const int64_t k0 = it.k0;
        const int r = c->host_fn(c->host_user, j->n, j->p, it.ds->coords, it.ds->y, it.ds->X, j->d_params + 5 * k0,
                                 it.count, j->d_lam, j->M, j->d_logL + k0 * j->M, j->d_s2 + k0 * j->M,
                                 j->d_beta + k0 * j->M * j->p, j->d_ld + 2 * k0, j->d_st + k0);
        return r == 0 ? std::string() : std::string("evaluator returned ") + std::to_string(r);
    }
    Layout L;
    make_layout(j->n, j->p, j->M, it.count, L, j->opts.precision);
    Dataset *d = it.ds;
    BatchArgs b;
    b.count = it.count;
    b.k0 = it.k0;
    b.n = j->n;
    b.n_pad = L.n_pad;
    b.nb = L.nb;
    b.q = L.q;
    b.p = j->p;
    b.M = j->M;
    b.reml = j->opts.reml;
    b.tpo = L.tpo;
    b.params = j->d_params + 5 * it.k0;
    b.coords = d->coords;
    b.lambdas = j->d_lam;
    b.Bt = j->d_bt;
    b.sumlogy = j->d_slog;
    b.oconst = at<double>(it.ws, L.off_oc);
    b.coordT = at<double>(it.ws, L.off_coordT);
    b.tab = at<double>(it.ws, L.off_tab);
    b.tiles = at<double>(it.ws, L.off_tiles);
    b.inv = at<double>(it.ws, L.off_inv);
    b.ldv = at<double>(it.ws, L.off_ldv);
    b.pstatus = at<int>(it.ws, L.off_pst);
    b.owner = at<int>(it.ws, L.off_owner);
    b.logL = j->d_logL;
    b.sigma2 = j->d_s2;
    b.beta = j->d_beta;
    b.logdet = j->d_ld;
    b.status = j->d_st;
    cudaStreamWaitEvent(s, j->ready, 0);   // the job's B^T may come from another stream
    std::string err;
    if (use_fused(j->n, L.q, j->opts.flags) && L.mixed) {
        plk_status st = run_fused_mixed_batch(b, L, it.ws, j->opts.flags, nullptr, s);
        if (st == PLK_OK && cudaStreamSynchronize(s) != cudaSuccess) st = PLK_E_CUDA;
        if (st != PLK_OK) err = plk_last_error();
    } else if (use_fused(j->n, L.q, j->opts.flags)) {
        cudaError_t e = use_graph(j->opts.flags) ? launch_as_graph(s, [&]() { return launch_fused_batch(b, s); })
                                                 : launch_fused_batch(b, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) err = cudaGetErrorString(e);
    } else if (L.mixed) {
        plk_status st = run_mixed_batch(b, L, it.ws, j->d_params, j->opts.flags, nullptr, true, s);
        if (st != PLK_OK) err = plk_last_error();
    } else {
        cudaError_t e = use_graph(j->opts.flags) ? launch_as_graph(s, [&]() { return launch_fp64_batch(b, s); })
                                                 : launch_fp64_batch(b, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) err = cudaGetErrorString(e);
    }
    return err;
}

void write_metrics(plk_ctx *c, const Job *j);

void finish_job(plk_ctx *c, Job *j) {
    // all items retired: read results back (synchronously on the job's last stream)
    const bool copy = !j->cancelled && !j->failed && j->dev;
    if (copy) {
        j->logL.resize(j->K * j->M);
        j->s2.resize(j->K * j->M);
        j->beta.resize(j->K * j->M * j->p);
        j->ld.resize(2 * j->K);
        j->st.resize(j->K);
    }
    cudaError_t e = cudaSuccess;
    if (copy && c->host && j->K > 0) {
        std::memcpy(j->logL.data(), j->d_logL, sizeof(double) * j->K * j->M);
        std::memcpy(j->s2.data(), j->d_s2, sizeof(double) * j->K * j->M);
        std::memcpy(j->beta.data(), j->d_beta, sizeof(double) * j->K * j->M * j->p);
        std::memcpy(j->ld.data(), j->d_ld, sizeof(double) * 2 * j->K);
        std::memcpy(j->st.data(), j->d_st, sizeof(int32_t) * j->K);
    } else if (copy && j->K > 0) {
        e = cudaMemcpy(j->logL.data(), j->d_logL, sizeof(double) * j->K * j->M, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(j->s2.data(), j->d_s2, sizeof(double) * j->K * j->M, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(j->beta.data(), j->d_beta, sizeof(double) * j->K * j->M * j->p, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(j->ld.data(), j->d_ld, sizeof(double) * 2 * j->K, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(j->st.data(), j->d_st, sizeof(int32_t) * j->K, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        j->failed = true;
        j->error = cudaGetErrorString(e);
    }
    c->arena.release(j->dev);
    j->dev = nullptr;
    if (j->ready) cudaEventDestroy(j->ready);
    j->ready = nullptr;
    c->datasets[j->ds]->active_jobs--;
    j->done = true;
    j->t_done = c->now();
    write_metrics(c, j);
}

// Wakes the threads waiting in plk_poll, unless a fault hook drops this
// notification (plk_poll then still sees the job done within its 50 ms
// re-check interval).  Caller holds mu.
void notify_done(plk_ctx *c) {
    if (c->fault_drop > 0) {
        c->fault_drop--;
        return;
    }
    c->cv_done.notify_all();
}

// Arena space for a batch's workspace; a fault hook can make the next
// allocations fail as if the arena were full.  Caller holds mu.
char *alloc_item(plk_ctx *c, size_t bytes) {
    if (c->fault_arena > 0) {
        c->fault_arena--;
        return nullptr;
    }
    return c->arena.alloc(bytes);
}

// One JSON line per finished job (plk_set_metrics_log).  Caller holds mu.
void write_metrics(plk_ctx *c, const Job *j) {
    if (!c->metrics) return;
    std::vector<double> it = j->item_s;
    std::sort(it.begin(), it.end());
    auto pct = [&](double q) { return it.empty() ? 0.0 : it[(size_t)std::min<double>(it.size() - 1, std::floor(q * it.size()))]; };
    double busy = 0.0;
    for (double v : it) busy += v;
    int64_t bad = 0, retried = 0, f64 = 0;
    for (int32_t v : j->st) {
        bad += (v & 15) != 0;
        retried += (v & PLK_POINT_RETRIED) != 0;
        f64 += (v & PLK_POINT_FP64) != 0;
    }
    const double run = j->t_done - j->t_start;
    const char *outcome = j->cancelled ? "cancelled" : j->failed ? "failed" : "ok";
    std::fprintf(c->metrics,
                 "{\"job\": %lld, \"dataset\": %lld, \"n\": %lld, \"p\": %d, \"M\": %d, \"K\": %lld, "
                 "\"precision\": \"%s\", \"reml\": %d, \"batch\": %d, \"items\": %zu, \"outcome\": \"%s\", "
                 "\"t_submit\": %.6f, \"t_start\": %.6f, \"t_done\": %.6f, \"queue_wait_s\": %.6f, "
                 "\"run_s\": %.6f, \"item_busy_s\": %.6f, \"item_ms_p50\": %.3f, \"item_ms_p99\": %.3f, "
                 "\"evals_per_s\": %.3f, \"points_not_ok\": %lld, \"points_retried\": %lld, "
                 "\"points_fp64\": %lld, \"arena_in_use\": %zu, \"arena_high_water\": %zu}\n",
                 (long long)j->id, (long long)j->ds, (long long)j->n, j->p, j->M, (long long)j->K,
                 j->opts.precision == PLK_MIXED ? "mixed" : "fp64", j->opts.reml, j->batch, it.size(), outcome,
                 j->t_submit, j->t_start, j->t_done, j->t_start - j->t_submit, run, busy, 1e3 * pct(0.5),
                 1e3 * pct(0.99), (run > 0.0 && !j->cancelled && !j->failed) ? (double)j->K / run : 0.0,
                 (long long)bad, (long long)retried, (long long)f64, c->arena.used(), c->arena.high());
    std::fflush(c->metrics);
}

// One worker per stream: take the next batch of the oldest job that has work
// left (admission: its workspace must fit in the arena; the batch shrinks until
// it does), run it, retire it.  Jobs submitted while others run are picked up
// as soon as a worker and arena space free up, so batches of different jobs
// overlap on the device.
void stream_worker(plk_ctx *c, int slot) {
    if (!c->host) cudaSetDevice(c->device);
    cudaStream_t s = c->host ? nullptr : c->streams[slot];
    std::unique_lock<std::mutex> lk(c->mu);
    while (true) {
        Job *pick = nullptr;
        for (Job *j : c->order) {
            if (!(j->next_k < j->K || (!j->started && j->K == 0))) continue;
            if (c->policy == PLK_SCHED_FIFO) {   // the oldest job with work left
                pick = j;
                break;
            }
            // largest first: the job with the largest dataset (cost per point ~ n^3), oldest on ties
            if (!pick || j->n > pick->n) pick = j;
        }
        if (!pick) {
            if (c->stop && c->order.empty()) break;
            c->cv_work.wait_for(lk, std::chrono::milliseconds(20));
            continue;
        }
        if (!pick->started) {
            if (!start_job(c, pick, s)) {   // no arena space for its inputs/outputs yet
                c->cv_work.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            if (pick->K == 0) {
                finish_job(c, pick);
                c->order.erase(std::find(c->order.begin(), c->order.end(), pick));
                notify_done(c);
                continue;
            }
        }
        int count = (int)std::min<int64_t>(pick->batch, pick->K - pick->next_k);
        char *ws = nullptr;
        while (count >= 1 &&
               !(ws = alloc_item(c, c->host ? (size_t)ALIGN * count
                                            : item_bytes(pick->n, pick->p, pick->M, count, pick->opts.precision))))
            count /= 2;
        if (!ws) {
            c->cv_work.wait_for(lk, std::chrono::milliseconds(2));
            continue;
        }
        Item it{pick, c->datasets[pick->ds].get(), pick->next_k, count, ws};
        pick->next_k += count;
        pick->inflight++;
        std::string err;
        if (c->fault_item > 0) {   // fault hook: this batch fails as a launch would
            c->fault_item--;
            err = "injected batch failure (fault hook)";
        } else {
            lk.unlock();
            const auto t0 = std::chrono::steady_clock::now();
            err = run_item(c, pick, it, s);
            const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            lk.lock();
            pick->item_s.push_back(dt);
        }
        if (!err.empty()) {
            pick->failed = true;
            pick->error = err;
            pick->next_k = pick->K;   // launch nothing more of a failed job
        }
        c->arena.release(ws);
        pick->inflight--;
        if (pick->inflight == 0 && pick->next_k >= pick->K && !pick->done) {
            finish_job(c, pick);
            c->order.erase(std::find(c->order.begin(), c->order.end(), pick));
            notify_done(c);
        }
        c->cv_work.notify_all();
    }
}

}  // namespace

namespace {
int n_bucket(int64_t n) { return (int)std::lround(2.0 * std::log2((double)std::max<int64_t>(n, 1))); }

// Points per batch for a job of K points on a dataset of n sites: the tuned
// value of the nearest tuned half-octave bucket (at most one bucket away),
// else the library default.  Caller holds mu.
int scheduled_batch(plk_ctx *c, int64_t n, int precision, int64_t K, int *tuned) {
    const int b = n_bucket(n);
    for (int d : {0, -1, 1}) {
        auto it = c->tuned.find({b + d, precision});
        if (it != c->tuned.end()) {
            if (tuned) *tuned = 1;
            return (int)std::max<int64_t>(1, std::min<int64_t>(it->second.first, std::max<int64_t>(K, 1)));
        }
    }
    if (tuned) *tuned = 0;
    return default_batch(n, K);
}
}  // namespace

extern "C" plk_status plk_create(plk_ctx **out, int device, void *arena, size_t arena_bytes,
                                 void *const *streams, int n_streams) {
    if (!out) return fail(PLK_E_INVALID, "out is NULL");
    if (arena_bytes < (1u << 20)) return fail(PLK_E_INVALID, "arena_bytes too small");
    if (n_streams < 1 || n_streams > 64) return fail(PLK_E_INVALID, "n_streams must be in [1, 64]");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(PLK_E_INVALID, "no device %d", device);
    if ((e = cudaSetDevice(device)) != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto c = std::make_unique<plk_ctx>();
    c->device = device;
    c->t0 = std::chrono::steady_clock::now();
    if (arena) {
        if (reinterpret_cast<uintptr_t>(arena) % ALIGN) return fail(PLK_E_INVALID, "arena must be 256-byte aligned");
        c->arena_base = static_cast<char *>(arena);
    } else {
        if ((e = cudaMalloc(&c->arena_base, arena_bytes)) != cudaSuccess) return cuda_fail(e, "cudaMalloc arena");
        c->own_arena = true;
    }
    c->arena.init(c->arena_base, arena_bytes / ALIGN * ALIGN);
    if (streams) {
        for (int i = 0; i < n_streams; ++i) c->streams.push_back(static_cast<cudaStream_t>(streams[i]));
    } else {
        for (int i = 0; i < n_streams; ++i) {
            cudaStream_t s;
            if ((e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking)) != cudaSuccess) return cuda_fail(e, "stream");
            c->streams.push_back(s);
        }
        c->own_streams = true;
    }
    for (int i = 0; i < (int)c->streams.size(); ++i) c->workers.emplace_back(stream_worker, c.get(), i);
    *out = c.release();
    return PLK_OK;
}

static bool all_finite(const double *p, int64_t m) {
    for (int64_t i = 0; i < m; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

extern "C" plk_status plk_create_dataset(plk_ctx *c, const double *coords, const double *y,
                                         const double *X, int64_t n, int32_t p, plk_dataset *out) {
    if (!c || !coords || !y || !X || !out) return fail(PLK_E_INVALID, "NULL argument");
    if (!(n > p && p >= 1 && p <= 16)) return fail(PLK_E_INVALID, "need n > p >= 1 and p <= 16");
    if (!all_finite(coords, 2 * n) || !all_finite(X, n * p) || !all_finite(y, n))
        return fail(PLK_E_INVALID, "non-finite input");
    for (int64_t i = 0; i < n; ++i)
        if (!(y[i] > 0.0)) return fail(PLK_E_INVALID, "y[%lld] = %g is not > 0", (long long)i, y[i]);
    if (!c->host) cudaSetDevice(c->device);
    std::lock_guard<std::mutex> lk(c->mu);
    auto d = std::make_unique<Dataset>();
    d->n = n;
    d->p = p;
    const size_t bc = align_up(sizeof(double) * 2 * n), by = align_up(sizeof(double) * n),
                 bx = align_up(sizeof(double) * n * p);
    char *m = c->arena.alloc(bc + by + bx);
    if (!m) return fail(PLK_E_NOMEM, "arena full: dataset needs %zu bytes", bc + by + bx);
    d->coords = (double *)m;
    d->y = (double *)(m + bc);
    d->X = (double *)(m + bc + by);
    cudaError_t e = cudaSuccess;
    if (c->host) {
        std::memcpy(d->coords, coords, sizeof(double) * 2 * n);
        std::memcpy(d->y, y, sizeof(double) * n);
        std::memcpy(d->X, X, sizeof(double) * n * p);
    }
    if (!c->host) e = cudaMemcpy(d->coords, coords, sizeof(double) * 2 * n, cudaMemcpyHostToDevice);
    if (!c->host && e == cudaSuccess) e = cudaMemcpy(d->y, y, sizeof(double) * n, cudaMemcpyHostToDevice);
    if (!c->host && e == cudaSuccess) e = cudaMemcpy(d->X, X, sizeof(double) * n * p, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        c->arena.release(m);
        return cuda_fail(e, "dataset upload");
    }
    *out = c->next_ds++;
    c->datasets[*out] = std::move(d);
    return PLK_OK;
}

extern "C" plk_status plk_submit_profile(plk_ctx *c, plk_dataset ds, const double *param_grid, int64_t K,
                                         const double *lambda_grid, int32_t M, const plk_options *opts,
                                         plk_job *out) {
    if (!c || !out || (K > 0 && !param_grid) || !lambda_grid) return fail(PLK_E_INVALID, "NULL argument");
    if (K < 0 || M < 1) return fail(PLK_E_INVALID, "need K >= 0 and M >= 1");
    if (!all_finite(lambda_grid, M)) return fail(PLK_E_INVALID, "non-finite lambda");
    plk_options o{};
    if (opts) o = *opts;
    if (o.precision != PLK_FP64 && o.precision != PLK_MIXED) return fail(PLK_E_INVALID, "unknown precision");
    std::unique_lock<std::mutex> lk(c->mu);
    auto dit = c->datasets.find(ds);
    if (dit == c->datasets.end()) return fail(PLK_E_INVALID, "unknown dataset %lld", (long long)ds);
    Dataset *d = dit->second.get();
    if (M + d->p > 64) return fail(PLK_E_INVALID, "M + p must be <= 64");
    const size_t need = job_io_bytes(K, M, d->p, d->n) + (c->host ? ALIGN : item_bytes(d->n, d->p, M, 1, o.precision));
    if (need > c->arena.size())
        return fail(PLK_E_NOMEM, "job needs at least %zu bytes, arena is %zu", need, c->arena.size());
    auto j = std::make_unique<Job>();
    j->id = c->next_job++;
    j->ds = ds;
    j->K = K;
    j->M = M;
    j->p = d->p;
    j->n = d->n;
    j->opts = o;
    j->params.assign(param_grid, param_grid + 5 * K);
    j->lambdas.assign(lambda_grid, lambda_grid + M);
    j->batch = o.batch > 0 ? std::min(o.batch, 65535) : scheduled_batch(c, d->n, o.precision, K, nullptr);
    j->t_submit = c->now();
    d->active_jobs++;
    *out = j->id;
    c->order.push_back(j.get());
    c->jobs[j->id] = std::move(j);
    c->cv_work.notify_all();
    return PLK_OK;
}

extern "C" plk_status plk_poll(plk_ctx *c, plk_job job, int32_t timeout_ms, double *logL,
                               double *sigma2, double *beta, double *logdet, int32_t *point_status,
                               double *t_submit, double *t_start, double *t_done) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    std::unique_lock<std::mutex> lk(c->mu);
    auto it = c->jobs.find(job);
    if (it == c->jobs.end()) return fail(PLK_E_INVALID, "unknown job %lld", (long long)job);
    Job *j = it->second.get();
    if (!j->done) {
        if (timeout_ms == 0) return fail(PLK_E_NOT_READY, "job %lld running", (long long)job);
        // wait in slices: a completion whose notification was lost is still
        // seen within one slice
        const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
        while (!j->done) {
            auto slice = std::chrono::steady_clock::now() + std::chrono::milliseconds(50);
            if (timeout_ms > 0 && deadline < slice) slice = deadline;
            c->cv_done.wait_until(lk, slice);
            if (!j->done && timeout_ms > 0 && std::chrono::steady_clock::now() >= deadline)
                return fail(PLK_E_NOT_READY, "job %lld running", (long long)job);
        }
    }
    if (j->cancelled) {
        c->jobs.erase(it);
        return fail(PLK_E_CANCELLED, "job %lld was cancelled", (long long)job);
    }
    if (j->failed) {
        std::string msg = j->error;
        c->jobs.erase(it);
        return fail(PLK_E_CUDA, "job failed: %s", msg.c_str());
    }
    if (logL) std::memcpy(logL, j->logL.data(), sizeof(double) * j->logL.size());
    if (sigma2) std::memcpy(sigma2, j->s2.data(), sizeof(double) * j->s2.size());
    if (beta) std::memcpy(beta, j->beta.data(), sizeof(double) * j->beta.size());
    if (logdet) std::memcpy(logdet, j->ld.data(), sizeof(double) * j->ld.size());
    if (point_status) std::memcpy(point_status, j->st.data(), sizeof(int32_t) * j->st.size());
    if (t_submit) *t_submit = j->t_submit;
    if (t_start) *t_start = j->t_start;
    if (t_done) *t_done = j->t_done;
    c->jobs.erase(it);
    return PLK_OK;
}

extern "C" plk_status plk_release_dataset(plk_ctx *c, plk_dataset ds) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->datasets.find(ds);
    if (it == c->datasets.end()) return fail(PLK_E_INVALID, "unknown dataset");
    if (it->second->active_jobs > 0) return fail(PLK_E_INVALID, "dataset has running jobs");
    c->arena.release((char *)it->second->coords);
    c->datasets.erase(it);
    return PLK_OK;
}

extern "C" plk_status plk_memory_stats(plk_ctx *c, size_t *in_use, size_t *high_water) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (in_use) *in_use = c->arena.used();
    if (high_water) *high_water = c->arena.high();
    return PLK_OK;
}

extern "C" plk_status plk_destroy(plk_ctx *c) {
    if (!c) return PLK_OK;
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->stop = true;
        c->cv_work.notify_all();
    }
    for (auto &t : c->workers) t.join();
    if (c->metrics) std::fclose(c->metrics);
    if (c->host) {
        std::free(c->arena_base);
        delete c;
        return PLK_OK;
    }
    cudaSetDevice(c->device);
    if (c->own_streams)
        for (auto s : c->streams) cudaStreamDestroy(s);
    if (c->own_arena) cudaFree(c->arena_base);
    delete c;
    return PLK_OK;
}

extern "C" plk_status plk_create_with_evaluator(plk_ctx **out, size_t arena_bytes, int n_workers,
                                                plk_host_eval_fn fn, void *user) {
    if (!out || !fn) return fail(PLK_E_INVALID, "NULL argument");
    if (arena_bytes < (1u << 20)) return fail(PLK_E_INVALID, "arena_bytes too small");
    if (n_workers < 1 || n_workers > 64) return fail(PLK_E_INVALID, "n_workers must be in [1, 64]");
    auto c = std::make_unique<plk_ctx>();
    c->host = true;
    c->host_fn = fn;
    c->host_user = user;
    c->device = -1;
    c->t0 = std::chrono::steady_clock::now();
    const size_t bytes = arena_bytes / ALIGN * ALIGN;
    c->arena_base = static_cast<char *>(std::aligned_alloc(ALIGN, bytes));
    if (!c->arena_base) return fail(PLK_E_NOMEM, "host arena of %zu bytes", bytes);
    c->own_arena = true;
    c->arena.init(c->arena_base, bytes);
    for (int i = 0; i < n_workers; ++i) c->workers.emplace_back(stream_worker, c.get(), i);
    *out = c.release();
    return PLK_OK;
}

extern "C" plk_status plk_cancel(plk_ctx *c, plk_job job) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->jobs.find(job);
    if (it == c->jobs.end()) return fail(PLK_E_INVALID, "unknown job %lld", (long long)job);
    Job *j = it->second.get();
    if (j->done) return PLK_OK;   // finished already: its results stay available
    j->cancelled = true;
    j->next_k = j->K;             // no further batches
    if (j->inflight == 0) {       // nothing running: it ends now
        if (j->started) {
            finish_job(c, j);
        } else {
            c->datasets[j->ds]->active_jobs--;
            j->done = true;
            j->t_done = c->now();
            write_metrics(c, j);
        }
        c->order.erase(std::find(c->order.begin(), c->order.end(), j));
        notify_done(c);
    }
    c->cv_work.notify_all();
    return PLK_OK;
}

extern "C" plk_status plk_inject_fault(plk_ctx *c, int32_t kind, int32_t count) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    if (count < 0) return fail(PLK_E_INVALID, "count < 0");
    std::lock_guard<std::mutex> lk(c->mu);
    switch (kind) {
        case PLK_FAULT_ARENA_ALLOC: c->fault_arena = count; break;
        case PLK_FAULT_BATCH: c->fault_item = count; break;
        case PLK_FAULT_DROP_COMPLETION: c->fault_drop = count; break;
        default: return fail(PLK_E_INVALID, "unknown fault kind %d", kind);
    }
    c->cv_work.notify_all();
    return PLK_OK;
}

extern "C" plk_status plk_pipe_counters(uint64_t *out, int32_t reset) {
    if (!out) return fail(PLK_E_INVALID, "out is NULL");
    const cudaError_t e = pipe_counters(reinterpret_cast<unsigned long long *>(out), reset);
    if (e == cudaErrorNotSupported) return fail(PLK_E_INVALID, "library built without PLK_PIPE_COUNTERS");
    if (e != cudaSuccess) return cuda_fail(e, "pipe counters");
    return PLK_OK;
}

extern "C" plk_status plk_set_mixed_tolerance(double tol) {
    if (!(tol > 0.0 && tol <= 1.0)) return fail(PLK_E_INVALID, "mixed tolerance %g outside (0, 1]", tol);
    g_mixed_tol.store(tol);
    return PLK_OK;
}

extern "C" double plk_get_mixed_tolerance(void) { return g_mixed_tol.load(); }

extern "C" plk_status plk_set_schedule_policy(plk_ctx *c, int32_t policy) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    if (policy != PLK_SCHED_FIFO && policy != PLK_SCHED_LARGEST_FIRST) return fail(PLK_E_INVALID, "unknown policy %d", policy);
    std::lock_guard<std::mutex> lk(c->mu);
    c->policy = policy;
    return PLK_OK;
}

extern "C" plk_status plk_set_metrics_log(plk_ctx *c, const char *path) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    if (c->metrics) std::fclose(c->metrics);
    c->metrics = nullptr;
    if (!path) return PLK_OK;
    c->metrics = std::fopen(path, "a");
    if (!c->metrics) return fail(PLK_E_INVALID, "cannot open %s for appending", path);
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
// Times the scheduler itself on a synthetic dataset of n sites: for each
// candidate batch size b, one job of 2 b x (number of streams) points (two
// batches per stream) from submit to results on the host, and keeps the b with
// the most points per second for n's half-octave bucket.
extern "C" plk_status plk_autotune(plk_ctx *c, int64_t n, int32_t p, int32_t M, int32_t precision,
                                   const int32_t *candidates, int32_t n_candidates, int32_t *best_batch,
                                   double *best_rate) {
    if (!c) return fail(PLK_E_INVALID, "ctx is NULL");
    if (c->host) return fail(PLK_E_INVALID, "autotune needs a GPU context");
    if (!sizes_ok(n, p, M)) return fail(PLK_E_INVALID, "invalid sizes n=%lld p=%d M=%d", (long long)n, p, M);
    if (precision != PLK_FP64 && precision != PLK_MIXED) return fail(PLK_E_INVALID, "unknown precision");
    std::vector<int> cand;
    if (candidates && n_candidates > 0) {
        for (int i = 0; i < n_candidates; ++i)
            if (candidates[i] >= 1 && candidates[i] <= 65535) cand.push_back(candidates[i]);
    } else {
        cand = {32, 64, 148, 296, 592};
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    if (cand.empty()) return fail(PLK_E_INVALID, "no valid candidate batch size");
    const int ns = (int)c->streams.size();
    // synthetic dataset: sites uniform on a square of side sqrt(n / 10), X = [1, N(0,1)...],
    // y > 0; parameter points spread over the box phi_X in [0.5, 8], kappa in [0.1, 8]
    // (log-uniform), nu^2 in [0, 0.5], ratio in [1, 4] (log-uniform), angle in [0, pi)
    std::mt19937_64 rng(0x9e3779b97f4a7c15ull ^ (uint64_t)n);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    std::normal_distribution<double> N01(0.0, 1.0);
    const double side = std::sqrt((double)n / 10.0);
    std::vector<double> coords(2 * n), y(n), X(n * p), lam(M);
    for (int64_t i = 0; i < n; ++i) {
        coords[2 * i] = side * U(rng);
        coords[2 * i + 1] = side * U(rng);
        X[i * p] = 1.0;
        double eta = 1.0;
        for (int k = 1; k < p; ++k) {
            X[i * p + k] = N01(rng);
            eta += 0.5 * X[i * p + k];
        }
        y[i] = std::exp(eta + 0.3 * std::sin(coords[2 * i]) + 0.3 * N01(rng));
    }
    for (int m = 0; m < M; ++m) lam[m] = M > 1 ? -0.5 + 2.0 * m / (M - 1) : 0.0;
    const int64_t kmax = 2 * (int64_t)cand.back() * ns;
    std::vector<double> P(5 * kmax);
    for (int64_t k = 0; k < kmax; ++k) {
        P[5 * k + 0] = 0.5 * std::pow(16.0, U(rng));
        P[5 * k + 1] = 0.1 * std::pow(80.0, U(rng));
        P[5 * k + 2] = 0.5 * U(rng);
        P[5 * k + 3] = std::pow(4.0, U(rng));
        P[5 * k + 4] = M_PI * U(rng);
    }
    plk_dataset ds = 0;
    plk_status st = plk_create_dataset(c, coords.data(), y.data(), X.data(), n, p, &ds);
    if (st != PLK_OK) return st;
    auto run = [&](int b, int64_t K, double *secs) -> plk_status {
        plk_options o{};
        o.precision = precision;
        o.batch = b;
        plk_job job = 0;
        const auto t0 = std::chrono::steady_clock::now();
        plk_status r = plk_submit_profile(c, ds, P.data(), K, lam.data(), M, &o, &job);
        if (r == PLK_OK) r = plk_poll(c, job, -1, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr);
        *secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return r;
    };
    double secs = 0.0;
    st = run(cand.front(), std::min<int64_t>(kmax, cand.front()), &secs);   // warm-up (module load, streams)
    int best = 0;
    double rate = 0.0;
    for (int b : cand) {
        if (st != PLK_OK) break;
        size_t free_bytes;
        {
            std::lock_guard<std::mutex> lk(c->mu);
            free_bytes = c->arena.size() - c->arena.used();
        }
        const int64_t K = 2 * (int64_t)b * ns;
        if (item_bytes(n, p, M, b, precision) * ns + job_io_bytes(K, M, p, n) > free_bytes) break;
        st = run(b, K, &secs);
        if (st == PLK_OK && secs > 0.0 && K / secs > rate) {
            rate = K / secs;
            best = b;
        }
    }
    std::string err = st != PLK_OK ? std::string(plk_last_error()) : std::string();
    plk_release_dataset(c, ds);
    if (st != PLK_OK) return fail(st, "autotune: %s", err.c_str());
    if (best == 0) return fail(PLK_E_NOMEM, "autotune: no candidate batch fits in the arena");
    {
        std::lock_guard<std::mutex> lk(c->mu);
        c->tuned[{n_bucket(n), precision}] = {best, rate};
    }
    if (best_batch) *best_batch = best;
    if (best_rate) *best_rate = rate;
    return PLK_OK;
}

extern "C" plk_status plk_scheduled_batch(plk_ctx *c, int64_t n, int32_t precision, int64_t K, int32_t *batch,
                                          int32_t *tuned) {
    if (!c || !batch) return fail(PLK_E_INVALID, "NULL argument");
    if (n < 1) return fail(PLK_E_INVALID, "n < 1");
    std::lock_guard<std::mutex> lk(c->mu);
    int t = 0;
    *batch = scheduled_batch(c, n, precision, K, &t);
    if (tuned) *tuned = t;
    return PLK_OK;
}

// ---------------------------------------------------------------------------
// failure detection self-test
// ---------------------------------------------------------------------------
static __device__ int g_selftest_err;

extern "C" plk_status plk_selftest_bounded_wait(int32_t max_iter, void *stream) {
    if (max_iter < 1 || max_iter > 1000000) return fail(PLK_E_INVALID, "max_iter must be in [1, 1e6]");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int *err = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&err), g_selftest_err);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_wait_selftest((uint32_t)max_iter, err, s);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    if (h) return fail(PLK_E_TIMEOUT, "a bounded device wait gave up after %d tries (self-test)", max_iter);
    return PLK_OK;
}

extern "C" plk_status plk_selftest_df_exp(const float *xh, const float *xl, float *yh, float *yl, int64_t count,
                                         void *stream) {
    if (count < 0 || count > ((int64_t)1 << 31)) return fail(PLK_E_INVALID, "count must be in [0, 2^31]");
    if (count > 0 && (!xh || !xl || !yh || !yl)) return fail(PLK_E_INVALID, "NULL pointer");
    const cudaError_t e = launch_df_exp_selftest(count, xh, xl, yh, yl, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "double-float exp self-test");
    return PLK_OK;
}
