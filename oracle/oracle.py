"""ctypes binding of the C oracle (plk_oracle.c) plus thin numpy marshalling.

Test infrastructure only: used by tests/, __graft_entry__.smoke() and the
benchmark's CPU-baseline leg.  Every function here forwards to the C oracle;
none of the method's arithmetic lives in Python.
"""
import ctypes as C

import numpy as np

from . import build as _build

__all__ = [
    "bessel_k", "bessel_k_scaled", "matern", "aniso_distance", "build_v",
    "boxcox", "profile_point", "profile_batch", "chi2_1_quantile",
    "profile_max", "profile_ci", "profile_beta", "profile_sigma", "profile_lambda",
    "profile_hull", "internal_params", "sum_log", "OR_OK", "OR_NOT_PD", "OR_INVALID", "OR_RSS_NONPOS",
]

OR_OK, OR_NOT_PD, OR_INVALID, OR_RSS_NONPOS = 0, 1, 2, 3

_lib = None
_D = C.c_double
_PD = C.POINTER(C.c_double)
_PI32 = C.POINTER(C.c_int32)
_I64 = C.c_int64
_I32 = C.c_int32


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.oracle_bessel_k.restype = _D
        L.oracle_bessel_k.argtypes = [_D, _D]
        L.oracle_bessel_k_scaled.restype = _D
        L.oracle_bessel_k_scaled.argtypes = [_D, _D]
        L.oracle_matern.restype = _D
        L.oracle_matern.argtypes = [_D, _D]
        L.oracle_aniso_distance.restype = _D
        L.oracle_aniso_distance.argtypes = [_D, _D, _D, _D, _D]
        L.oracle_build_v.restype = None
        L.oracle_build_v.argtypes = [_I64, _PD, _PD, _PD]
        L.oracle_boxcox.restype = _D
        L.oracle_boxcox.argtypes = [_D, _D]
        L.oracle_profile_point.restype = C.c_int
        L.oracle_profile_point.argtypes = [_I64, _I32, _PD, _PD, _PD, _PD, _I32, _PD, C.c_int,
                                           _PD, _PD, _PD, _PD, _PD, _PD]
        L.oracle_profile_batch.restype = C.c_int
        L.oracle_profile_batch.argtypes = [_I64, _I32, _PD, _PD, _PD, _I64, _PD, _I32, _PD,
                                           C.c_int, C.c_int, _PD, _PD, _PD, _PD, _PD, _PI32]
        L.oracle_chi2_1_quantile.restype = _D
        L.oracle_chi2_1_quantile.argtypes = [_D]
        L.oracle_profile_max.restype = None
        L.oracle_profile_max.argtypes = [_I64, _I64, _PD, _PD]
        L.oracle_profile_ci.restype = C.c_int
        L.oracle_profile_ci.argtypes = [_PD, _PD, _I64, _D, _PD, _PD, _PD, _PI32]
        L.oracle_profile_beta.restype = C.c_int
        L.oracle_profile_beta.argtypes = [_I64, _I32, _I32, _I64, _PD, _PD, _PI32, _PD, _D, _I32,
                                          _I64, _PD, _PD]
        L.oracle_profile_beta_reml.restype = C.c_int
        L.oracle_profile_beta_reml.argtypes = [_I64, _I32, _I32, _I64, _PD, _PD, _PI32, _PD, _D, _I32,
                                               _I64, _PD, _PD, _I32]
        L.oracle_profile_sigma.restype = C.c_int
        L.oracle_profile_sigma.argtypes = [_I64, _I32, _I32, _I64, _PD, _PD, _PI32, _PD, _D,
                                           _I64, _PD, _PD]
        L.oracle_profile_hull.restype = _I64
        L.oracle_profile_hull.argtypes = [_I64, _PD, _PD, _I64, _PD, _PD, _PI32]
        L.oracle_internal_params.restype = None
        L.oracle_internal_params.argtypes = [_PD, C.c_int, _PD]
        L.oracle_sum_log.restype = _D
        L.oracle_sum_log.argtypes = [_I64, _PD]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_PD)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _elementwise(fn, *args):
    arrs = np.broadcast_arrays(*[np.asarray(a, float) for a in args])
    flat = [a.ravel() for a in arrs]
    out = np.array([fn(*vals) for vals in zip(*flat)], dtype=float)
    return out.reshape(arrs[0].shape)


def bessel_k(nu, x):
    """K_nu(x), elementwise over broadcast arrays."""
    return _elementwise(lib().oracle_bessel_k, nu, x)


def bessel_k_scaled(nu, x):
    """e^x K_nu(x), elementwise."""
    return _elementwise(lib().oracle_bessel_k_scaled, nu, x)


def matern(d, kappa):
    """Matern correlation rho(d; kappa) of eq. matern (normaliser 2^{1-kappa}/Gamma)."""
    return _elementwise(lib().oracle_matern, d, kappa)


def aniso_distance(h1, h2, phi_x, phi_r, phi_a):
    return lib().oracle_aniso_distance(float(h1), float(h2), float(phi_x), float(phi_r), float(phi_a))


def build_v(coords, omega):
    coords = _f64(coords)
    n = coords.shape[0]
    V = np.empty((n, n))
    lib().oracle_build_v(n, _p(coords), _p(_f64(omega)), _p(V))
    return V


def boxcox(y, lam):
    f = lib().oracle_boxcox
    y = np.asarray(y, float)
    return np.array([f(v, float(lam)) for v in y.ravel()]).reshape(y.shape)


def profile_point(coords, y, X, omega, lambdas, reml=False):
    """All Table-1 statistics and l_p for one omega point.  Returns a dict."""
    coords, y, X, omega, lambdas = map(_f64, (coords, y, X, omega, lambdas))
    n, p = X.shape
    M = lambdas.shape[0]
    q = M + p
    out = dict(logL=np.empty(M), sigma2=np.empty(M), beta=np.empty((M, p)),
               rss=np.empty(M), ssq=np.empty((q, q)), logdet=np.empty(2))
    st = lib().oracle_profile_point(n, p, _p(coords), _p(y), _p(X), _p(omega), M, _p(lambdas),
                                    int(bool(reml)), _p(out["logL"]), _p(out["sigma2"]),
                                    _p(out["beta"]), _p(out["rss"]), _p(out["ssq"]),
                                    _p(out["logdet"]))
    out["status"] = st
    return out


def profile_batch(coords, y, X, params, lambdas, reml=False, nthreads=0, with_ssq=False):
    """l_p at K omega points (rows of params), OpenMP over the points.

    Returns dict(logL[K,M], sigma2[K,M], beta[K,M,p], logdet[K,2], status[K], threads),
    plus ssq[K,M+p,M+p] (Table 1 ssqYX) when with_ssq.
    """
    coords, y, X, params, lambdas = map(_f64, (coords, y, X, params, lambdas))
    n, p = X.shape
    K = params.shape[0]
    M = lambdas.shape[0]
    out = dict(logL=np.empty((K, M)), sigma2=np.empty((K, M)), beta=np.empty((K, M, p)),
               logdet=np.empty((K, 2)), status=np.empty(K, dtype=np.int32))
    if with_ssq:
        out["ssq"] = np.empty((K, M + p, M + p))
    used = lib().oracle_profile_batch(n, p, _p(coords), _p(y), _p(X), K, _p(params), M,
                                      _p(lambdas), int(bool(reml)), int(nthreads),
                                      _p(out["logL"]), _p(out["sigma2"]), _p(out["beta"]),
                                      _p(out["logdet"]), _p(out["ssq"]) if with_ssq else None,
                                      out["status"].ctypes.data_as(_PI32))
    out["threads"] = used
    return out


def chi2_1_quantile(level):
    return lib().oracle_chi2_1_quantile(float(level))


def profile_max(vals_g_sm):
    v = _f64(vals_g_sm)
    G = v.shape[0]
    prof = np.empty(G)
    lib().oracle_profile_max(G, int(np.prod(v.shape[1:])), _p(v), _p(prof))
    return prof


def profile_ci(grid, prof, level=0.95):
    grid, prof = _f64(grid), _f64(prof)
    lo, hi, am = _D(), _D(), _D()
    cens = _I32()
    st = lib().oracle_profile_ci(_p(grid), _p(prof), grid.shape[0], float(level),
                                 C.byref(lo), C.byref(hi), C.byref(am), C.byref(cens))
    return dict(status=st, lo=lo.value, hi=hi.value, argmax=am.value, censored=cens.value)


def sum_log(y):
    y = _f64(y)
    return lib().oracle_sum_log(y.shape[0], _p(y))


def _status_ptr(status):
    if status is None:
        return None, None
    s = np.ascontiguousarray(status, dtype=np.int32)
    return s, s.ctypes.data_as(_PI32)


def profile_beta(n, ssq, logdet, lambdas, sumlogy, j, grid, status=None, reml=False):
    """Profile of beta_j on `grid` from Table-1 statistics (Section 3.4; with
    reml, the Appendix's REML form).

    ssq: [K, M+p, M+p]; logdet: [K, 2]; lambdas: [M]; status: [K] or None."""
    ssq, logdet, lambdas, grid = map(_f64, (ssq, logdet, lambdas, grid))
    K, q = ssq.shape[0], ssq.shape[1]
    M = lambdas.shape[0]
    s, sp = _status_ptr(status)
    prof = np.empty(grid.shape[0])
    st = lib().oracle_profile_beta_reml(int(n), q - M, M, K, _p(ssq), _p(logdet), sp, _p(lambdas),
                                        float(sumlogy), int(j), grid.shape[0], _p(grid), _p(prof),
                                        int(bool(reml)))
    if st != OR_OK:
        raise ValueError("oracle_profile_beta: invalid arguments")
    return prof


def profile_sigma(n, ssq, logdet, lambdas, sumlogy, sgrid, status=None):
    """Profile of sigma on `sgrid` from Table-1 statistics (Section 3.5)."""
    ssq, logdet, lambdas, sgrid = map(_f64, (ssq, logdet, lambdas, sgrid))
    K, q = ssq.shape[0], ssq.shape[1]
    M = lambdas.shape[0]
    s, sp = _status_ptr(status)
    prof = np.empty(sgrid.shape[0])
    st = lib().oracle_profile_sigma(int(n), q - M, M, K, _p(ssq), _p(logdet), sp, _p(lambdas),
                                    float(sumlogy), sgrid.shape[0], _p(sgrid), _p(prof))
    if st != OR_OK:
        raise ValueError("oracle_profile_sigma: invalid arguments")
    return prof


def profile_lambda(logL):
    """Profile of lambda (Section 3.6): max over the omega points for each lambda."""
    return profile_max(np.ascontiguousarray(np.asarray(logL, float).T))


def profile_hull(x, v, xq):
    """Upper-convex-hull 1-D profile (Section 3.6).  Returns (out[Q], on_hull[K], n_vertices)."""
    x, v, xq = map(_f64, (x, v, xq))
    K = x.shape[0]
    out = np.empty(xq.shape[0])
    on = np.empty(K, dtype=np.int32)
    nh = lib().oracle_profile_hull(K, _p(x), _p(v), xq.shape[0], _p(xq), _p(out),
                                   on.ctypes.data_as(_PI32))
    return out, on, nh


def internal_params(params, kappa_hat_large=False):
    """omega' = (gamma_1, kappa~, nu, gamma_2, gamma_3) for each row of params (Section 3.2)."""
    params = np.atleast_2d(_f64(params))
    out = np.empty_like(params)
    for k in range(params.shape[0]):
        row = np.ascontiguousarray(params[k])
        o = np.empty(5)
        lib().oracle_internal_params(_p(row), int(bool(kappa_hat_large)), _p(o))
        out[k] = o
    return out
