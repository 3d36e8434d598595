"""ctypes binding of libplk.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; this module only passes
pointers, sizes and streams.  If the library is missing or cannot be loaded the
functions raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("PLK_LIBRARY") or os.path.join(HERE, "libplk.so")   # PLK_LIBRARY: another build
HEADER = os.path.join(os.path.dirname(HERE), "include", "plk.h")

PLK_OK, PLK_E_INVALID, PLK_E_NOMEM, PLK_E_NOT_READY, PLK_E_TIMEOUT, PLK_E_CUDA, PLK_E_CANCELLED = range(7)
POINT_OK, POINT_NOT_PD, POINT_BAD_PARAM, POINT_RSS_NONPOS, POINT_RETRIED, POINT_FP64 = 0, 1, 2, 3, 16, 32
FP64, MIXED = 0, 1


class PlkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"plk status {status}: {msg}")
        self.status = status


class EvalArgs(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int32), ("M", C.c_int32),
                ("coords", C.c_void_p), ("y", C.c_void_p), ("X", C.c_void_p), ("lambdas", C.c_void_p),
                ("K", C.c_int64), ("params", C.c_void_p),
                ("logL", C.c_void_p), ("sigma2", C.c_void_p), ("beta", C.c_void_p),
                ("logdet", C.c_void_p), ("status", C.c_void_p), ("err_bound", C.c_void_p),
                ("ssq_yx", C.c_void_p)]


class StatsArgs(C.Structure):
    _fields_ = [("n", C.c_int64), ("p", C.c_int32), ("M", C.c_int32), ("K", C.c_int64),
                ("y", C.c_void_p), ("lambdas", C.c_void_p), ("ssq_yx", C.c_void_p),
                ("logdet", C.c_void_p), ("status", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("reml", C.c_int32), ("batch", C.c_int32), ("flags", C.c_int32)]


class FitOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("reml", C.c_int32), ("kappa_fixed", C.c_int32), ("kappa", C.c_double),
                ("delta", C.c_double), ("delta_lambda", C.c_double), ("max_iter", C.c_int32), ("tol", C.c_double)]


class CloudOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("reml", C.c_int32), ("kappa_fixed", C.c_int32), ("n_sphere", C.c_int32),
                ("n_levels", C.c_int32), ("level_probs", C.c_void_p), ("n_lambda", C.c_int32),
                ("delta", C.c_double), ("delta_lambda", C.c_double), ("seed", C.c_uint64),
                ("sphere_rounds", C.c_int32)]


_PD = C.POINTER(C.c_double)
HOST_EVAL_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int64, C.c_int32, _PD, _PD, _PD, _PD, C.c_int64, _PD, C.c_int32,
                           _PD, _PD, _PD, _PD, C.POINTER(C.c_int32))
FAULT_ARENA_ALLOC, FAULT_BATCH, FAULT_DROP_COMPLETION = 1, 2, 3
SCHED_FIFO, SCHED_LARGEST_FIRST = 0, 1

EVAL_FN = C.CFUNCTYPE(C.c_int32, C.c_void_p, C.POINTER(C.c_double), C.c_int64, C.POINTER(C.c_double), C.c_int32,
                      C.POINTER(C.c_double))

_lib = None


def declared_symbols():
    """Names of the functions include/plk.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(plk_[a-z0-9_]+)\s*\(", text)))


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2305_04318_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    sig = {
        "plk_eval_workspace_bytes": (sz, [i64, i32, i32, i32, i32]),
        "plk_eval_device": (C.c_int, [C.POINTER(EvalArgs), C.POINTER(Options), vp, sz, vp]),
        "plk_eval_device_static": (C.c_int, [C.POINTER(EvalArgs), i32, vp]),
        "plk_build_covariance_device": (C.c_int, [vp, i64, vp, i64, i32, vp, vp, sz, vp]),
        "plk_create": (C.c_int, [C.POINTER(vp), C.c_int, vp, sz, C.POINTER(vp), C.c_int]),
        "plk_create_dataset": (C.c_int, [vp, vp, vp, vp, i64, i32, C.POINTER(i64)]),
        "plk_submit_profile": (C.c_int, [vp, i64, vp, i64, vp, i32, C.POINTER(Options), C.POINTER(i64)]),
        "plk_poll": (C.c_int, [vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp]),
        "plk_release_dataset": (C.c_int, [vp, i64]),
        "plk_memory_stats": (C.c_int, [vp, C.POINTER(sz), C.POINTER(sz)]),
        "plk_destroy": (C.c_int, [vp]),
        "plk_autotune": (C.c_int, [vp, i64, i32, i32, i32, vp, i32, C.POINTER(i32), C.POINTER(dbl)]),
        "plk_scheduled_batch": (C.c_int, [vp, i64, i32, i64, C.POINTER(i32), C.POINTER(i32)]),
        "plk_last_error": (C.c_char_p, []),
        "plk_profile_max_device": (C.c_int, [vp, i64, i64, vp, vp]),
        "plk_profile_ci_device": (C.c_int, [vp, vp, i64, dbl, vp, vp]),
        "plk_profile_ci": (C.c_int, [vp, vp, i64, dbl, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl),
                                     C.POINTER(i32)]),
        "plk_chi2_1_quantile": (dbl, [dbl]),
        "plk_profile_beta_device": (C.c_int, [C.POINTER(StatsArgs), i32, vp, i64, vp, vp]),
        "plk_profile_beta_reml_device": (C.c_int, [C.POINTER(StatsArgs), i32, vp, i64, vp, vp]),
        "plk_profile_sigma_device": (C.c_int, [C.POINTER(StatsArgs), vp, i64, vp, vp]),
        "plk_profile_lambda_device": (C.c_int, [vp, i64, i32, vp, vp]),
        "plk_profile_hull_device": (C.c_int, [vp, i64, vp, i64, vp, i64, vp, vp, vp]),
        "plk_internal_params_device": (C.c_int, [vp, i64, i32, vp, vp]),
        "plk_kernel_timing": (C.c_int, [C.POINTER(dbl), C.POINTER(i64), i32, i32, C.POINTER(i32)]),
        "plk_natural_params": (C.c_int, [vp, i64, i32, vp]),
        "plk_chi2_quantile": (dbl, [i32, dbl]),
        "plk_hessian_stencil": (C.c_int, [vp, i32, dbl, vp, C.POINTER(i32)]),
        "plk_hessian_from_stencil": (C.c_int, [i32, dbl, vp, dbl, vp, vp, vp, vp]),
        "plk_fix_hessian": (C.c_int, [i32, vp, vp, vp]),
        "plk_sphere_points": (C.c_int, [i32, i32, C.c_uint64, i32, vp, C.POINTER(dbl)]),
        "plk_fit_mle": (C.c_int, [vp, i64, vp, dbl, C.POINTER(FitOptions), vp, C.POINTER(dbl), C.POINTER(dbl),
                                  C.POINTER(i32)]),
        "plk_fit_mle_cb": (C.c_int, [EVAL_FN, vp, vp, dbl, C.POINTER(FitOptions), vp, C.POINTER(dbl),
                                     C.POINTER(dbl), C.POINTER(i32)]),
        "plk_quadratic_cloud": (C.c_int, [vp, i64, vp, dbl, C.POINTER(CloudOptions), vp, i64, C.POINTER(i64), vp,
                                          vp, vp]),
        "plk_quadratic_cloud_cb": (C.c_int, [EVAL_FN, vp, vp, dbl, C.POINTER(CloudOptions), vp, i64,
                                             C.POINTER(i64), vp, vp, vp]),
        "plk_kernel_class_name": (C.c_char_p, [i32]),
        "plk_selftest_bounded_wait": (C.c_int, [i32, vp]),
        "plk_cancel": (C.c_int, [vp, i64]),
        "plk_set_metrics_log": (C.c_int, [vp, C.c_char_p]),
        "plk_set_schedule_policy": (C.c_int, [vp, i32]),
        "plk_set_mixed_tolerance": (C.c_int, [C.c_double]),
        "plk_pipe_counters": (C.c_int, [vp, i32]),
        "plk_get_mixed_tolerance": (C.c_double, []),
        "plk_inject_fault": (C.c_int, [vp, i32, i32]),
        "plk_create_with_evaluator": (C.c_int, [C.POINTER(vp), sz, C.c_int, HOST_EVAL_FN, vp]),
        "plk_selftest_df_exp": (C.c_int, [vp, vp, vp, vp, i64, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st):
    if st != PLK_OK:
        raise PlkError(st, lib().plk_last_error().decode())


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _stream_handle(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def workspace_bytes(n, p, M, batch, precision=FP64):
    return int(lib().plk_eval_workspace_bytes(n, p, M, batch, precision))


def default_batch(n, K, limit_bytes=8e9):
    """Points per batch so that the tile workspace stays near limit_bytes."""
    nb = -(-int(n) // 128)
    per = (nb + 1) * (nb + 2) // 2 * 128 * 128 * 8
    return int(max(1, min(296, limit_bytes // per, max(K, 1))))


FLAG_KERNEL_TIMING = 1
FLAG_NO_RETRY = 2
FLAG_NO_FP64_TIER = 4
FLAG_GRAPH = 8
FLAG_FULL_FIRST_PASS = 16
FLAG_NO_FUSED = 32
FLAG_PIPELINED_RETRY = 64


PIPE_COUNTER_NAMES = ("loop_cycles", "items", "mma_wait_accumulators", "mma_wait_B", "mma_wait_A",
                      "epilogue_wait_mma", "epilogue_wait_C", "epilogue_wait_store_read", "epilogue_update")
PIPE_MODES = ("triangle", "column", "rhs_row")


def pipe_counters(reset=True):
    """Wait-cycle counters of the 5-slice trailing update (a library built with
    -DPLK_PIPE_COUNTERS; plk_pipe_counters): {mode: {name: cycles}}."""
    buf = (C.c_uint64 * (3 * len(PIPE_COUNTER_NAMES)))()
    _check(lib().plk_pipe_counters(C.cast(buf, C.c_void_p), int(bool(reset))))
    n = len(PIPE_COUNTER_NAMES)
    return {m: {k: int(buf[i * n + j]) for j, k in enumerate(PIPE_COUNTER_NAMES)} for i, m in enumerate(PIPE_MODES)}


def set_mixed_tolerance(tol):
    """Tolerance of the mixed-precision retry rule on |Delta l_p| (process-wide;
    default 1e-3): plk_set_mixed_tolerance."""
    _check(lib().plk_set_mixed_tolerance(float(tol)))


def get_mixed_tolerance():
    return float(lib().plk_get_mixed_tolerance())


def kernel_timing(reset=True):
    """{class name: (total ms, launches)} of launches made with FLAG_KERNEL_TIMING."""
    n = 32
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    nd = C.c_int32()
    _check(lib().plk_kernel_timing(ms, cnt, n, int(bool(reset)), C.byref(nd)))
    return {lib().plk_kernel_class_name(c).decode(): (ms[c], cnt[c]) for c in range(nd.value)}


def eval_device(coords, y, X, lambdas, params, precision=FP64, reml=False, batch=0,
                workspace=None, stream=None, outputs=None, flags=0, with_ssq=False):
    """Evaluate l_p at all rows of `params` (torch CUDA float64 tensors).

    Returns a dict of CUDA tensors logL[K,M], sigma2[K,M], beta[K,M,p],
    logdet[K,2], status[K] (int32), err_bound[K], and ssq_yx[K,M+p,M+p] (the
    Table-1 cross-products) when with_ssq.  The workspace (uint8 CUDA tensor)
    is allocated with torch when not given.  Asynchronous on `stream`.
    """
    import torch
    dev = coords.device
    n, p = X.shape
    M = lambdas.shape[0]
    K = params.shape[0]
    for t in (coords, y, X, lambdas, params):
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    if batch <= 0:
        batch = default_batch(n, K)
    if outputs is None:
        outputs = dict(logL=torch.empty((K, M), dtype=torch.float64, device=dev),
                       sigma2=torch.empty((K, M), dtype=torch.float64, device=dev),
                       beta=torch.empty((K, M, p), dtype=torch.float64, device=dev),
                       logdet=torch.empty((K, 2), dtype=torch.float64, device=dev),
                       status=torch.empty((K,), dtype=torch.int32, device=dev),
                       err_bound=torch.empty((K,), dtype=torch.float64, device=dev))
        if with_ssq:
            outputs["ssq_yx"] = torch.empty((K, M + p, M + p), dtype=torch.float64, device=dev)
    wsb = workspace_bytes(n, p, M, batch, precision)
    if wsb == 0:
        raise PlkError(PLK_E_INVALID, f"invalid sizes n={n} p={p} M={M}")
    if workspace is None:
        workspace = torch.empty((wsb,), dtype=torch.uint8, device=dev)
    a = EvalArgs(n, p, M, _ptr(coords), _ptr(y), _ptr(X), _ptr(lambdas), K, _ptr(params),
                 _ptr(outputs.get("logL")), _ptr(outputs.get("sigma2")), _ptr(outputs.get("beta")),
                 _ptr(outputs.get("logdet")), _ptr(outputs.get("status")), _ptr(outputs.get("err_bound")),
                 _ptr(outputs.get("ssq_yx")))
    o = Options(precision, int(bool(reml)), batch, int(flags))
    _check(lib().plk_eval_device(C.byref(a), C.byref(o), _ptr(workspace), workspace.numel(),
                                 _stream_handle(stream)))
    return outputs


BUILD_FP64, BUILD_DF_FAST, BUILD_DF = 0, 1, 2


def build_covariance_device(coords, params, mode=BUILD_FP64, workspace=None, stream=None, out=None):
    """Dense V(omega_k) = R + nu^2 I for every row of `params` (CUDA float64),
    as the evaluation builds it: mode BUILD_FP64 (FP64 path), BUILD_DF_FAST
    (mixed path, first pass), BUILD_DF (mixed path, 7-slice tier).  Returns a
    [K, n, n] CUDA float64 tensor."""
    import torch
    n = coords.shape[0]
    K = params.shape[0]
    for t in (coords, params):
        assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
    if out is None:
        out = torch.empty((K, n, n), dtype=torch.float64, device=coords.device)
    if workspace is None:
        workspace = torch.empty((workspace_bytes(n, 1, 1, K, FP64),), dtype=torch.uint8, device=coords.device)
    _check(lib().plk_build_covariance_device(_ptr(coords), n, _ptr(params), K, int(mode), _ptr(out),
                                             _ptr(workspace), workspace.numel(), _stream_handle(stream)))
    return out


STATIC_SCRATCH_BYTES = 64 << 20


def selftest_bounded_wait(max_iter=1000, stream=None):
    """Run the bounded-wait self-test (plk_selftest_bounded_wait); returns the
    status (PLK_E_TIMEOUT expected) without raising."""
    return int(lib().plk_selftest_bounded_wait(int(max_iter), _stream_handle(stream)))


def selftest_df_exp(xh, xl, stream=None):
    """(yh, yl) = the library's double-float exp of xh + xl (CUDA float32 tensors)."""
    import torch
    yh, yl = torch.empty_like(xh), torch.empty_like(xh)
    _check(lib().plk_selftest_df_exp(_ptr(xh), _ptr(xl), _ptr(yh), _ptr(yl), xh.numel(), _stream_handle(stream)))
    return yh, yl


def eval_device_static(coords, y, X, lambdas, params, reml=False, stream=None, outputs=None):
    """FP64 evaluation through plk_eval_device_static: the library uses its own
    fixed device scratch array, so this call allocates no device memory beyond
    the output tensors (pass `outputs` to allocate none at all)."""
    import torch
    dev = coords.device
    n, p = X.shape
    M = lambdas.shape[0]
    K = params.shape[0]
    if outputs is None:
        outputs = dict(logL=torch.empty((K, M), dtype=torch.float64, device=dev),
                       sigma2=torch.empty((K, M), dtype=torch.float64, device=dev),
                       beta=torch.empty((K, M, p), dtype=torch.float64, device=dev),
                       logdet=torch.empty((K, 2), dtype=torch.float64, device=dev),
                       status=torch.empty((K,), dtype=torch.int32, device=dev))
    a = EvalArgs(n, p, M, _ptr(coords), _ptr(y), _ptr(X), _ptr(lambdas), K, _ptr(params),
                 _ptr(outputs.get("logL")), _ptr(outputs.get("sigma2")), _ptr(outputs.get("beta")),
                 _ptr(outputs.get("logdet")), _ptr(outputs.get("status")), None,
                 _ptr(outputs.get("ssq_yx")))
    _check(lib().plk_eval_device_static(C.byref(a), int(bool(reml)), _stream_handle(stream)))
    return outputs


def profile_max_device(vals, prof=None, stream=None):
    """prof[g] = NaN-skipping max of vals[g, ...] (CUDA float64)."""
    import torch
    G = vals.shape[0]
    SM = int(np.prod(vals.shape[1:])) if vals.dim() > 1 else 1
    if prof is None:
        prof = torch.empty((G,), dtype=torch.float64, device=vals.device)
    _check(lib().plk_profile_max_device(_ptr(vals), G, SM, _ptr(prof), _stream_handle(stream)))
    return prof


def profile_ci_device(grid, prof, level=0.95, out=None, stream=None):
    """CUDA tensor [lo, hi, argmax, censored] of the likelihood CI."""
    import torch
    if out is None:
        out = torch.empty((4,), dtype=torch.float64, device=grid.device)
    _check(lib().plk_profile_ci_device(_ptr(grid), _ptr(prof), grid.shape[0], float(level), _ptr(out),
                                       _stream_handle(stream)))
    return out


def profile_ci(grid, prof, level=0.95):
    """Likelihood CI from host arrays (plk_profile_ci): dict(lo, hi, argmax, censored)."""
    g = np.ascontiguousarray(grid, dtype=np.float64)
    v = np.ascontiguousarray(prof, dtype=np.float64)
    lo, hi, am, cens = C.c_double(), C.c_double(), C.c_double(), C.c_int32()
    _check(lib().plk_profile_ci(_np_ptr(g), _np_ptr(v), g.shape[0], float(level), C.byref(lo), C.byref(hi),
                                C.byref(am), C.byref(cens)))
    return dict(lo=lo.value, hi=hi.value, argmax=am.value, censored=cens.value)


def chi2_1_quantile(level):
    return float(lib().plk_chi2_1_quantile(float(level)))


def _stats_args(y, lambdas, ssq_yx, logdet, status):
    K, q = ssq_yx.shape[0], ssq_yx.shape[1]
    M = lambdas.shape[0]
    return StatsArgs(y.shape[0], q - M, M, K, _ptr(y), _ptr(lambdas), _ptr(ssq_yx), _ptr(logdet),
                     _ptr(status))


def profile_beta_device(y, lambdas, ssq_yx, logdet, status, j, grid, prof=None, stream=None, reml=False):
    """Profile of beta_j at the CUDA float64 `grid` from the evaluation's
    statistics (ssq_yx [K,M+p,M+p], logdet [K,2], status [K] or None); reml:
    the Appendix's REML criterion."""
    import torch
    if prof is None:
        prof = torch.empty((grid.shape[0],), dtype=torch.float64, device=grid.device)
    a = _stats_args(y, lambdas, ssq_yx, logdet, status)
    fn = lib().plk_profile_beta_reml_device if reml else lib().plk_profile_beta_device
    _check(fn(C.byref(a), int(j), _ptr(grid), grid.shape[0], _ptr(prof), _stream_handle(stream)))
    return prof


def profile_sigma_device(y, lambdas, ssq_yx, logdet, status, grid, prof=None, stream=None):
    """Profile of sigma at the CUDA float64 `grid` (standard deviations)."""
    import torch
    if prof is None:
        prof = torch.empty((grid.shape[0],), dtype=torch.float64, device=grid.device)
    a = _stats_args(y, lambdas, ssq_yx, logdet, status)
    _check(lib().plk_profile_sigma_device(C.byref(a), _ptr(grid), grid.shape[0], _ptr(prof),
                                          _stream_handle(stream)))
    return prof


def profile_lambda_device(logL, prof=None, stream=None):
    """prof[m] = NaN-skipping max over the omega points of logL[:, m]."""
    import torch
    K, M = logL.shape
    if prof is None:
        prof = torch.empty((M,), dtype=torch.float64, device=logL.device)
    _check(lib().plk_profile_lambda_device(_ptr(logL), K, M, _ptr(prof), _stream_handle(stream)))
    return prof


def profile_hull_device(x, v, xq, x_stride=1, out=None, on_hull=None, stream=None):
    """Upper-hull profile of the cloud (x[k * x_stride], v[k]) at the points xq.

    Returns (out [Q] float64, on_hull [K] int32), CUDA tensors."""
    import torch
    K = v.shape[0]
    if out is None:
        out = torch.empty((xq.shape[0],), dtype=torch.float64, device=v.device)
    if on_hull is None:
        on_hull = torch.empty((K,), dtype=torch.int32, device=v.device)
    _check(lib().plk_profile_hull_device(_ptr(x), int(x_stride), _ptr(v), K, _ptr(xq), xq.shape[0],
                                         _ptr(out), _ptr(on_hull), _stream_handle(stream)))
    return out, on_hull


def internal_params_device(params, kappa_hat_large=False, out=None, stream=None):
    """omega' = (gamma_1, kappa~, nu, gamma_2, gamma_3) of each parameter row."""
    import torch
    if out is None:
        out = torch.empty_like(params)
    _check(lib().plk_internal_params_device(_ptr(params), params.shape[0], int(bool(kappa_hat_large)),
                                            _ptr(out), _stream_handle(stream)))
    return out


def _host_eval_callback(fn):
    """Wrap fn(coords[n,2], y[n], X[n,p], params[count,5], lambdas[M]) ->
    dict(logL, sigma2, beta, logdet, status) as a plk_host_eval_fn."""
    def cb(user, n, p, coords, y, X, params, count, lambdas, M, logL, sigma2, beta, logdet, status):
        try:
            arr = np.ctypeslib.as_array
            r = fn(arr(coords, shape=(n, 2)).copy(), arr(y, shape=(n,)).copy(), arr(X, shape=(n, p)).copy(),
                   arr(params, shape=(count, 5)).copy(), arr(lambdas, shape=(M,)).copy())
            arr(logL, shape=(count, M))[:] = r["logL"]
            arr(sigma2, shape=(count, M))[:] = r["sigma2"]
            arr(beta, shape=(count, M, p))[:] = r["beta"]
            arr(logdet, shape=(count, 2))[:] = r["logdet"]
            arr(status, shape=(count,))[:] = r["status"]
            return 0
        except Exception:
            return 1
    return HOST_EVAL_FN(cb)


class Context:
    """Device-resident datasets and asynchronous profile jobs (plk_create ... plk_destroy).

    `arena` may be a torch uint8 CUDA tensor (PyTorch owns the memory); if None
    the library allocates `arena_bytes` itself.  With `evaluator` (a host
    function, see _host_eval_callback) the context runs its batches on
    `n_streams` host worker threads through it instead of on a GPU
    (plk_create_with_evaluator: for testing the scheduler without a GPU).
    """

    def __init__(self, arena_bytes, device=0, arena=None, n_streams=4, streams=None, evaluator=None):
        self._arena = arena
        h = C.c_void_p()
        if evaluator is not None:
            self._cb = _host_eval_callback(evaluator)
            _check(lib().plk_create_with_evaluator(C.byref(h), int(arena_bytes), int(n_streams), self._cb, None))
            self.h = h
            return
        sarr = None
        if streams is not None:
            sarr = (C.c_void_p * len(streams))(*[s.cuda_stream for s in streams])
            n_streams = len(streams)
            self._streams = streams
        _check(lib().plk_create(C.byref(h), device, _ptr(arena) if arena is not None else None,
                                int(arena_bytes), sarr, n_streams))
        self.h = h

    def create_dataset(self, coords, y, X):
        coords = np.ascontiguousarray(coords, dtype=np.float64)
        y = np.ascontiguousarray(y, dtype=np.float64)
        X = np.ascontiguousarray(X, dtype=np.float64)
        out = C.c_int64()
        _check(lib().plk_create_dataset(self.h, _np_ptr(coords), _np_ptr(y), _np_ptr(X), X.shape[0],
                                        X.shape[1], C.byref(out)))
        return out.value

    def submit(self, ds, params, lambdas, precision=FP64, reml=False, batch=0, flags=0):
        params = np.ascontiguousarray(params, dtype=np.float64).reshape(-1, 5)
        lambdas = np.ascontiguousarray(lambdas, dtype=np.float64)
        out = C.c_int64()
        o = Options(precision, int(bool(reml)), batch, int(flags))
        _check(lib().plk_submit_profile(self.h, ds, _np_ptr(params), params.shape[0], _np_ptr(lambdas),
                                        lambdas.shape[0], C.byref(o), C.byref(out)))
        return dict(id=out.value, K=params.shape[0], M=lambdas.shape[0])

    def poll(self, job, p, timeout_ms=-1):
        """Results as numpy arrays, or None if not ready within timeout_ms."""
        K, M = job["K"], job["M"]
        r = dict(logL=np.empty((K, M)), sigma2=np.empty((K, M)), beta=np.empty((K, M, p)),
                 logdet=np.empty((K, 2)), status=np.empty(K, dtype=np.int32))
        ts, t0, t1 = C.c_double(), C.c_double(), C.c_double()
        st = lib().plk_poll(self.h, job["id"], int(timeout_ms), _np_ptr(r["logL"]), _np_ptr(r["sigma2"]),
                            _np_ptr(r["beta"]), _np_ptr(r["logdet"]), _np_ptr(r["status"]),
                            C.byref(ts), C.byref(t0), C.byref(t1))
        if st == PLK_E_NOT_READY:
            return None
        _check(st)
        r.update(t_submit=ts.value, t_start=t0.value, t_done=t1.value)
        return r

    def release_dataset(self, ds):
        _check(lib().plk_release_dataset(self.h, ds))

    def cancel(self, job):
        _check(lib().plk_cancel(self.h, job["id"]))

    def set_schedule_policy(self, policy):
        """SCHED_FIFO (default) or SCHED_LARGEST_FIRST (plk_set_schedule_policy)."""
        _check(lib().plk_set_schedule_policy(self.h, int(policy)))

    def set_metrics_log(self, path):
        _check(lib().plk_set_metrics_log(self.h, None if path is None else os.fsencode(path)))

    def inject_fault(self, kind, count):
        """Host-side fault hook (plk_inject_fault): FAULT_ARENA_ALLOC, FAULT_BATCH
        or FAULT_DROP_COMPLETION for the next `count` events."""
        _check(lib().plk_inject_fault(self.h, int(kind), int(count)))

    def autotune(self, n, p, M, precision=FP64, candidates=None):
        """Tune the points per scheduled batch for datasets of about n sites
        (plk_autotune).  Returns (batch, points per second)."""
        arr, k = None, 0
        if candidates is not None:
            k = len(candidates)
            arr = (C.c_int32 * k)(*[int(x) for x in candidates])
        b, r = C.c_int32(), C.c_double()
        _check(lib().plk_autotune(self.h, int(n), int(p), int(M), int(precision), arr, k, C.byref(b), C.byref(r)))
        return b.value, r.value

    def scheduled_batch(self, n, precision=FP64, K=1 << 30):
        """(batch, tuned) the scheduler uses for a job on n sites with opts.batch = 0."""
        b, t = C.c_int32(), C.c_int32()
        _check(lib().plk_scheduled_batch(self.h, int(n), int(precision), int(K), C.byref(b), C.byref(t)))
        return b.value, bool(t.value)

    def memory_stats(self):
        a, b = C.c_size_t(), C.c_size_t()
        _check(lib().plk_memory_stats(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if getattr(self, "h", None):
            _check(lib().plk_destroy(self.h))
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# Steps 1 and 2 (Sections 3.1-3.2): host logic in the library
# ---------------------------------------------------------------------------

def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def natural_params(internal, kappa_hat_large=False):
    v = _f64(internal).reshape(-1, 5)
    out = np.empty_like(v)
    _check(lib().plk_natural_params(_np_ptr(v), v.shape[0], int(bool(kappa_hat_large)), _np_ptr(out)))
    return out


def chi2_quantile(dof, p):
    return float(lib().plk_chi2_quantile(int(dof), float(p)))


def hessian_stencil(center_internal, kappa_fixed=False, delta=0.05):
    c = _f64(center_internal)
    out = np.empty((51, 5))
    S = C.c_int32()
    _check(lib().plk_hessian_stencil(_np_ptr(c), int(bool(kappa_fixed)), float(delta), _np_ptr(out), C.byref(S)))
    return out[:S.value].copy()


def hessian_from_stencil(logL3, kappa_fixed=False, delta=0.05, tmax=1.0):
    f = _f64(logL3).reshape(-1, 3)
    d = 4 if kappa_fixed else 5
    H, g = np.empty((d, d)), np.empty(d)
    L, T = np.empty(f.shape[0]), np.empty(f.shape[0])
    _check(lib().plk_hessian_from_stencil(int(bool(kappa_fixed)), float(delta), _np_ptr(f), float(tmax), _np_ptr(H),
                                          _np_ptr(g), _np_ptr(L), _np_ptr(T)))
    return H, g, L, T


def fix_hessian(H):
    H = _f64(H)
    d = H.shape[0]
    E, D = np.empty((d, d)), np.empty(d)
    _check(lib().plk_fix_hessian(d, _np_ptr(H), _np_ptr(E), _np_ptr(D)))
    return E, D


def sphere_points(d, n, seed=1, rounds=200):
    x = np.empty((n, d))
    m = C.c_double()
    _check(lib().plk_sphere_points(int(d), int(n), int(seed), int(rounds), _np_ptr(x), C.byref(m)))
    return x, m.value


def _eval_callback(fn):
    """Wrap a Python evaluator fn(params[K,5], lambdas[M]) -> logL[K,M]."""
    def cb(user, params, K, lambdas, M, out):
        try:
            P = np.ctypeslib.as_array(params, shape=(K, 5)).copy()
            lam = np.ctypeslib.as_array(lambdas, shape=(M,)).copy()
            r = np.asarray(fn(P, lam), dtype=np.float64).reshape(K, M)
            np.ctypeslib.as_array(out, shape=(K, M))[:] = r
            return 0
        except Exception:
            return PLK_E_INVALID
    return EVAL_FN(cb)


def _fit_opts(precision, kappa_fixed, kappa, delta, delta_lambda, max_iter, tol, reml=False):
    return FitOptions(int(precision), int(bool(reml)), int(bool(kappa_fixed)), float(kappa or 0.0), float(delta),
                      float(delta_lambda), int(max_iter), float(tol))


def _fit_result(w, lam, L, it):
    return dict(omega=w, lam=lam.value, logL=L.value, iterations=it.value)


def fit_mle(ctx, ds, omega0, lambda0, precision=FP64, kappa_fixed=False, kappa=None, delta=0.05, delta_lambda=0.05,
            max_iter=60, tol=1e-7, reml=False):
    """Step 1 on the context's GPU evaluation (plk_fit_mle); reml: the REML profile likelihood."""
    w0 = _f64(omega0)
    w, lam, L, it = np.empty(5), C.c_double(), C.c_double(), C.c_int32()
    o = _fit_opts(precision, kappa_fixed, kappa, delta, delta_lambda, max_iter, tol, reml)
    _check(lib().plk_fit_mle(ctx.h, ds, _np_ptr(w0), float(lambda0), C.byref(o), _np_ptr(w), C.byref(lam),
                             C.byref(L), C.byref(it)))
    return _fit_result(w, lam, L, it)


def fit_mle_cb(evaluate, omega0, lambda0, kappa_fixed=False, kappa=None, delta=0.05, delta_lambda=0.05,
               max_iter=60, tol=1e-7):
    """Step 1 with a Python evaluator evaluate(params[K,5], lambdas[M]) -> logL[K,M]."""
    w0 = _f64(omega0)
    w, lam, L, it = np.empty(5), C.c_double(), C.c_double(), C.c_int32()
    o = _fit_opts(FP64, kappa_fixed, kappa, delta, delta_lambda, max_iter, tol)
    cb = _eval_callback(evaluate)
    _check(lib().plk_fit_mle_cb(cb, None, _np_ptr(w0), float(lambda0), C.byref(o), _np_ptr(w), C.byref(lam),
                                C.byref(L), C.byref(it)))
    return _fit_result(w, lam, L, it)


def _cloud_call(fn, first, omega_hat, lambda_hat, precision, kappa_fixed, n_sphere, level_probs, n_lambda, delta,
                delta_lambda, seed, sphere_rounds, reml=False):
    w = _f64(omega_hat)
    probs = None if level_probs is None else _f64(level_probs)
    o = CloudOptions(int(precision), int(bool(reml)), int(bool(kappa_fixed)), int(n_sphere),
                     0 if probs is None else len(probs),
                     None if probs is None else _np_ptr(probs), int(n_lambda), float(delta), float(delta_lambda),
                     int(seed), int(sphere_rounds))
    K = C.c_int64()
    _check(fn(*first, _np_ptr(w), float(lambda_hat), C.byref(o), None, 0, C.byref(K), None, None, None))
    d = 4 if kappa_fixed else 5
    P, lam, H, D = np.empty((K.value, 5)), np.empty(max(n_lambda, 1)), np.empty((d, d)), np.empty(d)
    _check(fn(*first, _np_ptr(w), float(lambda_hat), C.byref(o), _np_ptr(P), K.value, C.byref(K), _np_ptr(lam),
              _np_ptr(H), _np_ptr(D)))
    return dict(params=P, lambdas=lam[:n_lambda], hessian=H, eigenvalues=D)


def quadratic_cloud(ctx, ds, omega_hat, lambda_hat, precision=FP64, kappa_fixed=False, n_sphere=0, level_probs=None,
                    n_lambda=30, delta=0.05, delta_lambda=0.05, seed=1, sphere_rounds=0, reml=False):
    """Step 2 on the context's GPU evaluation (plk_quadratic_cloud); reml: the REML profile likelihood."""
    return _cloud_call(lib().plk_quadratic_cloud, (ctx.h, ds), omega_hat, lambda_hat, precision, kappa_fixed,
                       n_sphere, level_probs, n_lambda, delta, delta_lambda, seed, sphere_rounds, reml)


def quadratic_cloud_cb(evaluate, omega_hat, lambda_hat, kappa_fixed=False, n_sphere=0, level_probs=None,
                       n_lambda=30, delta=0.05, delta_lambda=0.05, seed=1, sphere_rounds=0):
    """Step 2 with a Python evaluator evaluate(params[K,5], lambdas[M]) -> logL[K,M]."""
    cb = _eval_callback(evaluate)
    return _cloud_call(lib().plk_quadratic_cloud_cb, (cb, None), omega_hat, lambda_hat, FP64, kappa_fixed,
                       n_sphere, level_probs, n_lambda, delta, delta_lambda, seed, sphere_rounds)
