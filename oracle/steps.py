"""Oracle of Steps 1-2 of the method (Sections 3.1-3.2), in plain numpy.

Test infrastructure only (imported by tests/ alone).  Each function is the
textbook definition the paper's step refers to, written for checking by eye,
and shares no code with the library:

  natural_from_internal  inverse of the internal parameters of Section 3.2
  lambda_profile         maximum over lambda of the parabola through l_p at
                         lambda-hat - dl, lambda-hat, lambda-hat + dl (the
                         Hessian is taken with lambda at its maximiser given
                         omega', Section 3.2 "Hessian matrix")
  hessian_fd             central-difference gradient and Hessian
  fix_eigen              eigen-decomposition of -H and the fix-up of negative
                         and near-zero eigenvalues (Section 3.2)
  ellipsoid              points of the contour ellipsoid
                         (w - w_hat)^T (-H~) (w - w_hat) = c
  profiled_loglik        l_p at natural rows, maximised over lambda by the
                         parabola, from the C oracle's l_p
The readings taken where the paper is garbled or silent (the ellipsoid map,
"close to 0", the finite-difference step, the lambda handling) are the ones
stated in the design notes; the library takes the same readings.
"""
import numpy as np

from . import oracle as _o


def natural_from_internal(v, kappa_large=False):
    """Rows (gamma_1, kappa~, nu, gamma_2, gamma_3) -> (phi_X, kappa, nu^2, phi_R, phi_A)."""
    v = np.atleast_2d(np.asarray(v, float))
    g1, kt, nu, g2, g3 = v.T
    ratio = 1.0 + g2 ** 2 + g3 ** 2                 # phi_X / phi_Y
    phi_x = np.sqrt(np.exp(g1) * ratio)             # phi_X^2 = (phi_X phi_Y)(phi_X / phi_Y)
    kappa = 1.0 / kt ** 2 if kappa_large else np.exp(kt)
    angle = np.where(g2 ** 2 + g3 ** 2 > 0, 0.5 * np.arctan2(g3, g2), 0.0)
    angle = np.where(angle < 0, angle + np.pi, angle)
    return np.column_stack([phi_x, kappa, nu ** 2, ratio, angle])


def internal_from_natural(w, kappa_large=False):
    return _o.internal_params(np.atleast_2d(np.asarray(w, float)), kappa_large)


def lambda_profile(fm, f0, fp, tmax=1.0):
    """max over |t| <= tmax of the parabola through (-1, fm), (0, f0), (1, fp),
    or the largest of the three values when it is not concave; (value, t)."""
    vals = np.array([fm, f0, fp], float)
    if not np.all(np.isfinite(vals)):
        return np.nan, 0.0
    b = (fp - fm) / 2.0
    c = (fp + fm - 2.0 * f0) / 2.0
    t, v = 0.0, f0
    if c < 0:
        t = float(np.clip(-b / (2.0 * c), -tmax, tmax))
        v = f0 + b * t + c * t * t
    if fm > v:
        t, v = -1.0, fm
    if fp > v:
        t, v = 1.0, fp
    return v, t


def hessian_fd(F, center, free, delta):
    """Central differences of F (a function of a 5-vector) in the coordinates
    `free`: g_i = (F(+i) - F(-i)) / 2 delta, H_ii = (F(+i) - 2 F(0) + F(-i)) /
    delta^2, H_ij = (F(++) - F(+-) - F(-+) + F(--)) / 4 delta^2."""
    c = np.asarray(center, float)
    d = len(free)

    def at(*moves):
        x = c.copy()
        for k, s in moves:
            x[free[k]] += s * delta
        return F(x)

    f0 = F(c)
    H = np.zeros((d, d))
    g = np.zeros(d)
    for i in range(d):
        fp, fm = at((i, 1)), at((i, -1))
        g[i] = (fp - fm) / (2 * delta)
        H[i, i] = (fp - 2 * f0 + fm) / delta ** 2
    for i in range(d):
        for j in range(i + 1, d):
            H[i, j] = H[j, i] = (at((i, 1), (j, 1)) - at((i, 1), (j, -1)) - at((i, -1), (j, 1))
                                 + at((i, -1), (j, -1))) / (4 * delta ** 2)
    return H, g


def fix_eigen(H):
    """-H = E diag(D) E^T; |negative| eigenvalues; if max D > 100 those below 0.1
    become 0.1; numerically zero (below 1e-8 max(1, max D)) or non-finite ones
    become 0.1."""
    D, E = np.linalg.eigh(-np.asarray(H, float))
    D = np.abs(D)
    mx = np.max(D[np.isfinite(D)]) if np.any(np.isfinite(D)) else 0.0
    D = np.where(~np.isfinite(D) | (D <= 1e-8 * max(1.0, mx)), 0.1, D)
    if mx > 100:
        D = np.where(D < 0.1, 0.1, D)
    return E, D


def ellipsoid(center, free, E, D, c, x):
    """Points w = center + sqrt(c) S x, S = E D^{-1/2} E^T the symmetric inverse
    square root of E D E^T (x on the unit sphere, n x d), in the coordinates
    `free`: (w - center)^T E D E^T (w - center) = c."""
    S = E @ np.diag(1.0 / np.sqrt(D)) @ E.T
    W = np.tile(np.asarray(center, float), (x.shape[0], 1))
    W[:, free] += np.sqrt(c) * x @ S.T
    return W


def profiled_loglik(coords, y, X, natural_rows, lam_hat, dl, tmax=1.0):
    """max over lambda in [lam_hat - tmax dl, lam_hat + tmax dl] of the parabola
    through the C oracle's l_p at lam_hat - dl, lam_hat, lam_hat + dl."""
    P = np.atleast_2d(np.asarray(natural_rows, float))
    r = _o.profile_batch(coords, y, X, P, np.array([lam_hat - dl, lam_hat, lam_hat + dl]))
    L = r["logL"]
    return np.array([lambda_profile(*L[k], tmax=tmax)[0] for k in range(P.shape[0])])
