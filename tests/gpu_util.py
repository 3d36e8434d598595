"""Helpers shared by the GPU tests: move inputs to the device, run the CUDA
path through the C ABI, run the oracle on the same inputs, compare."""
import numpy as np
import torch

from paper_2305_04318_b300 import native as nv

# FP64 mode: |Delta l_p| <= 1e-8 |l_p| (the tolerance the method's FP64 mode
# promises), with matching per-point status.
RTOL_LOGL = 1e-8


def to_dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def gpu_eval(ds, params, lambdas, **kw):
    out = nv.eval_device(to_dev(ds.coords), to_dev(ds.y), to_dev(ds.X), to_dev(lambdas), to_dev(params), **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def oracle_eval(ds, params, lambdas, reml=False):
    import oracle
    return oracle.profile_batch(ds.coords, ds.y, ds.X, params, lambdas, reml=reml)


def compare(g, o, rtol=RTOL_LOGL, what=""):
    np.testing.assert_array_equal(g["status"], o["status"], err_msg=f"{what} status")
    ok = o["status"] == 0
    gl, ol = g["logL"][ok], o["logL"][ok]
    fin = np.isfinite(ol)
    np.testing.assert_array_equal(np.isfinite(gl), fin, err_msg=f"{what} finiteness")
    err = np.abs(gl[fin] - ol[fin]) / np.abs(ol[fin])
    assert err.size == 0 or err.max() <= rtol, f"{what} max rel logL err {err.max():.3e}"
    np.testing.assert_allclose(g["logdet"][ok], o["logdet"][ok], rtol=rtol, atol=1e-9, err_msg=f"{what} logdet")
    np.testing.assert_allclose(g["sigma2"][ok], o["sigma2"][ok], rtol=100 * rtol, err_msg=f"{what} sigma2")
    scale = np.abs(o["beta"][ok]).max() if ok.any() else 1.0
    np.testing.assert_allclose(g["beta"][ok], o["beta"][ok], rtol=100 * rtol, atol=100 * rtol * scale,
                               err_msg=f"{what} beta")
    bad = ~ok
    assert np.all(np.isnan(g["logL"][bad & (o["status"] != 3)]))
    return float(err.max()) if err.size else 0.0


# Near-singularity, judged on the oracle's matrix.  The 7-slice tier of the
# mixed path (the last one that can call a point not positive definite) keeps
# the trailing matrix in double-float: every stored entry of a Schur
# complement is rounded to ~2^-48 of its size (<= 1 + nu^2) at each of the
# nb/2 two-panel updates, ~2^-44 (1 + nu^2) accumulated, so its factorisation
# may fail where V is within n 2^-44 (1 + nu^2) of singular.  Since every
# Cholesky pivot of an SPD matrix is >= its smallest eigenvalue, a smallest
# pivot below that level proves V that close to singular; a factorisation that
# fails in FP64 proves it for FP64 itself.
def singular_threshold(n, nug, safety=4.0, unit=2.0 ** -44):
    """unit: 2^-44 for the mixed path's 7-slice tier, 2^-52 for FP64."""
    return safety * n * unit * (1.0 + nug)


def min_pivot(coords, omega):
    """Smallest Cholesky pivot L_jj^2 of the oracle's V(omega), or -inf when
    the FP64 factorisation fails."""
    import oracle
    V = oracle.build_v(coords, omega)
    try:
        L = np.linalg.cholesky(V)
    except np.linalg.LinAlgError:
        return -np.inf
    return float(np.min(np.diag(L)) ** 2)


def check_disagreements(coords, params, idx, max_count, unit=2.0 ** -44):
    """Every point in idx (GPU and reference statuses differ) must be near
    singular at the level `unit`; at most max_count of them.  Returns
    [(index, min pivot, threshold)]."""
    n = coords.shape[0]
    rows = []
    for k in idx:
        piv = min_pivot(coords, params[k])
        rows.append((int(k), piv, singular_threshold(n, params[k][2], unit=unit)))
    print("status disagreements (index, oracle min pivot, threshold):", rows)
    assert len(idx) <= max_count, f"{len(idx)} status disagreements (cap {max_count}): {rows}"
    bad = [r for r in rows if not r[1] <= r[2]]
    assert not bad, f"status disagreement on points that are not near singular: {bad}"
    return rows


def compare_fp64_singular(g, o, coords, params, rtol=RTOL_LOGL, max_count=None, what=""):
    """compare() for FP64 results where some V are singular to working
    precision: a point whose status differs from the oracle's must have a V
    within FP64 rounding of singular (smallest oracle pivot below
    4 n 2^-52 (1 + nu^2), or an FP64 factorisation that fails).  Such a
    point's log-likelihood, where both sides return one, is decided by a pivot
    of rounding size (log|V| holds the log of that pivot, and the exact value
    is -inf), so it is left out of the comparison too; the other points are
    compared as usual."""
    diff = np.flatnonzero(g["status"] != o["status"])
    if len(diff):
        check_disagreements(coords, params, diff, len(params) if max_count is None else max_count,
                            unit=2.0 ** -52)
    n = coords.shape[0]
    keep = g["status"] == o["status"]
    for k in np.flatnonzero(keep & (o["status"] == 0)):
        if min_pivot(coords, params[k]) <= singular_threshold(n, params[k][2], unit=2.0 ** -52):
            keep[k] = False
    return compare({k: v[keep] for k, v in g.items()},
                   {k: v[keep] for k, v in o.items() if k != "threads"}, rtol=rtol, what=what)
