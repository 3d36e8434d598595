"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds none of the profile-likelihood arithmetic: no Box-Cox
transform, no Matern/Bessel evaluation, no factorisation.  It draws sites,
covariates, responses, parameter grids and lambda grids from numpy's
``default_rng(seed)`` so that the CUDA path and the CPU oracle see identical
inputs.

Responses are simulated from a spatially correlated Gaussian field made of
random Fourier features whose frequencies are drawn from the Matern spectral
density.  For the correlation of eq. matern (Section 2) in the rotated and
scaled coordinates z = diag(1/phi_X, 1/phi_Y) Rot(phi_A) h, the spectral density
of rho(|z|) is a bivariate Student-t with 2*kappa degrees of freedom and scale
2, so a frequency is w_z = 2 g / sqrt(chi2_{2 kappa} / (2 kappa)) with g ~ N(0, I),
mapped back to site coordinates by w = Rot^T diag(1/phi_X, 1/phi_Y) w_z.  The
field U(s) = sqrt(2/J) sum_j cos(w_j . s + b_j) has unit variance and, as J
grows, the Matern correlation.  The likelihood is evaluated for whatever y is
given, so the simulation only has to look like the paper's data, not be exact.

Workloads (the paper's real datasets, Swiss rainfall n=100 and soil mercury
n=829, are not available; these synthetic inputs stand in for them):
  iso100     n=100 on [0,1]^2, X=[1,x1], kappa=1, K=100 (20 ranges x 5 nuggets), lambda={0}
  aniso1000  n=1000 on [0,10]^2, X=[1,x1,x2], K=4096 Halton points, 9 lambdas
  mixed4000  n=4000 on [0,20]^2, p=3, K=1024 (960 Halton + 64 ill-conditioned), 9 lambdas
  uneven     256 datasets, n log-uniform in [200,3000], p in {2,3,5}, 512 points each
  serving    32 datasets, n log-uniform in [500,8000], p=3; profile jobs of 64 x 4^4 points
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAMBDA_GRID_9 = np.linspace(-0.5, 1.5, 9)

# Box of correlation parameters for the Halton / uniform omega draws:
# log phi_X in [log .5, log 8], log kappa in [log .1, log 8], nu^2 in [0, .5],
# log phi_R in [0, log 4], phi_A in [0, pi).
OMEGA_BOX = dict(log_phix=(math.log(0.5), math.log(8.0)), log_kappa=(math.log(0.1), math.log(8.0)),
                 nug=(0.0, 0.5), log_ratio=(0.0, math.log(4.0)), angle=(0.0, math.pi))


@dataclass
class Dataset:
    coords: np.ndarray          # n x 2
    y: np.ndarray               # n, all > 0
    X: np.ndarray               # n x p
    name: str = ""
    truth: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.coords.shape[0]

    @property
    def p(self):
        return self.X.shape[1]


@dataclass
class Workload:
    name: str
    datasets: list
    params: list                # per dataset: K_d x 5 array [phi_X, kappa, nu^2, phi_R, phi_A]
    lambdas: np.ndarray         # M
    meta: dict = field(default_factory=dict)


def radical_inverse(i: np.ndarray, base: int) -> np.ndarray:
    """Van der Corput radical inverse of integers i in the given base."""
    i = np.asarray(i, dtype=np.int64).copy()
    f = np.ones_like(i, dtype=np.float64)
    r = np.zeros_like(i, dtype=np.float64)
    while np.any(i > 0):
        f = f / base
        r = r + f * (i % base)
        i = i // base
    return r


def halton(K: int, bases=(2, 3, 5, 7, 11), start: int = 1) -> np.ndarray:
    idx = np.arange(start, start + K)
    return np.column_stack([radical_inverse(idx, b) for b in bases])


def omega_from_unit(u: np.ndarray) -> np.ndarray:
    """Map points of [0,1)^5 to the omega box (columns phi_X, kappa, nu^2, phi_R, phi_A)."""
    b = OMEGA_BOX
    lo = np.array([b["log_phix"][0], b["log_kappa"][0], b["nug"][0], b["log_ratio"][0], b["angle"][0]])
    hi = np.array([b["log_phix"][1], b["log_kappa"][1], b["nug"][1], b["log_ratio"][1], b["angle"][1]])
    v = lo + u * (hi - lo)
    return np.column_stack([np.exp(v[:, 0]), np.exp(v[:, 1]), v[:, 2], np.exp(v[:, 3]), v[:, 4]])


def gaussian_field(rng, coords, kappa, phi_x, phi_r=1.0, phi_a=0.0, J=1024):
    """Unit-variance field with (approximately) anisotropic Matern correlation."""
    g = rng.standard_normal((J, 2))
    chi = rng.chisquare(2.0 * kappa, size=J)
    wz = 2.0 * g / np.sqrt(chi / (2.0 * kappa))[:, None]
    phi_y = phi_x / phi_r
    c, s = math.cos(phi_a), math.sin(phi_a)
    # w = Rot^T diag(1/phi_X, 1/phi_Y) w_z, Rot = [[c, -s], [s, c]]
    a = wz[:, 0] / phi_x
    b = wz[:, 1] / phi_y
    w = np.column_stack([c * a + s * b, -s * a + c * b])
    phase = rng.uniform(0.0, 2.0 * math.pi, size=J)
    return math.sqrt(2.0 / J) * np.cos(coords @ w.T + phase).sum(axis=1)


def _inverse_boxcox_positive(z, lam):
    """y with b(y; lam) = z, or None if 1 + lam z <= 0 somewhere."""
    if lam == 0.0:
        return np.exp(z)
    base = 1.0 + lam * z
    if np.any(base <= 0.0):
        return None
    return base ** (1.0 / lam)


def simulate_dataset(seed, n, side, p, beta, sigma, kappa, phi_x, nug, phi_r=1.0, phi_a=0.0,
                     lam=0.0, name=""):
    """Sites U[0,side]^2, X = [1, N(0,1) columns], y = inverse Box-Cox of
    X beta + sigma U + sigma nu eps.  Redraws with seed + 1000 k if the inverse
    transform would leave the positive reals."""
    for k in range(100):
        rng = np.random.default_rng(seed + 1000 * k)
        coords = rng.uniform(0.0, side, size=(n, 2))
        X = np.column_stack([np.ones(n)] + [rng.standard_normal(n) for _ in range(p - 1)])
        U = gaussian_field(rng, coords, kappa, phi_x, phi_r, phi_a)
        eps = rng.standard_normal(n)
        z = X @ np.asarray(beta, float) + sigma * U + sigma * math.sqrt(nug) * eps
        y = _inverse_boxcox_positive(z, lam)
        if y is not None and np.all(np.isfinite(y)) and np.all(y > 0):
            return Dataset(coords, y, X, name=name,
                           truth=dict(beta=list(beta), sigma=sigma, kappa=kappa, phi_x=phi_x,
                                      nug=nug, phi_r=phi_r, phi_a=phi_a, lam=lam, seed=seed + 1000 * k))
    raise RuntimeError("could not draw a positive response")


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------

def iso100(seed=1) -> Workload:
    ds = simulate_dataset(seed, 100, 1.0, 2, beta=(1.0, 0.5), sigma=1.0, kappa=1.0, phi_x=0.2,
                          nug=0.1, lam=0.0, name="iso100")
    phx = np.linspace(0.05, 1.0, 20)
    nug = np.linspace(0.0, 0.5, 5)
    P, N = np.meshgrid(phx, nug, indexing="ij")
    params = np.column_stack([P.ravel(), np.ones(P.size), N.ravel(), np.ones(P.size), np.zeros(P.size)])
    return Workload("iso100", [ds], [params], np.array([0.0]))


def aniso_dataset(seed, n, side, p, name=""):
    beta = (4.0,) + (0.5,) * (p - 1)
    return simulate_dataset(seed, n, side, p, beta=beta, sigma=1.0, kappa=1.5, phi_x=2.0, nug=0.1,
                            phi_r=2.0, phi_a=math.pi / 6, lam=0.5, name=name)


def aniso1000(seed=2, K=4096) -> Workload:
    ds = aniso_dataset(seed, 1000, 10.0, 3, name="aniso1000")
    return Workload("aniso1000", [ds], [omega_from_unit(halton(K))], LAMBDA_GRID_9.copy())


def ill_conditioned_points() -> np.ndarray:
    """64 deliberately ill-conditioned omega: kappa=8, phi_X in [8,40] (8 log-spaced),
    nu^2 in {0, 1e-6, 1e-3, 1e-2}, phi_R in {1, 2} (angle pi/6)."""
    rows = []
    for phx in np.geomspace(8.0, 40.0, 8):
        for nug in (0.0, 1e-6, 1e-3, 1e-2):
            for ratio in (1.0, 2.0):
                rows.append([phx, 8.0, nug, ratio, math.pi / 6])
    return np.array(rows)


def mixed4000(seed=3, K_halton=960, n=4000) -> Workload:
    ds = aniso_dataset(seed, n, 20.0 * math.sqrt(n / 4000.0), 3, name="mixed4000")
    params = np.vstack([omega_from_unit(halton(K_halton)), ill_conditioned_points()])
    return Workload("mixed4000", [ds], [params], LAMBDA_GRID_9.copy(), meta=dict(n_ill=64))


def uneven(seed=4, D=256, per=512, n_lo=200, n_hi=3000) -> Workload:
    rng = np.random.default_rng(seed)
    ns = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=D))).astype(int)
    ps = [(2, 3, 5)[d % 3] for d in range(D)]
    dsets, params = [], []
    for d in range(D):
        side = math.sqrt(ns[d] / 10.0)
        dsets.append(aniso_dataset(seed * 100000 + d, int(ns[d]), side, ps[d], name=f"uneven{d}"))
        params.append(omega_from_unit(rng.uniform(0.0, 1.0, size=(per, 5))))
    return Workload("uneven", dsets, params, LAMBDA_GRID_9.copy())


PROFILE_PARAM_NAMES = ("phi_x", "kappa", "nugget", "ratio", "angle")


def serving_pool(seed=5, D=32, n_lo=500, n_hi=8000):
    rng = np.random.default_rng(seed)
    ns = np.round(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=D))).astype(int)
    return [aniso_dataset(seed * 100000 + d, int(ns[d]), math.sqrt(ns[d] / 10.0), 3, name=f"pool{d}")
            for d in range(D)]


def profile_job_grid(which: int, G=64, sub=4):
    """Omega grid of one profile job for parameter `which` (0..4, in the order
    phi_X, kappa, nu^2, phi_R, phi_A): G values of that parameter across its box
    x sub^4 values of the other four.  Rows are grid-major: row g*sub^4 + s.
    Returns (grid_values[G], params[G*sub^4, 5])."""
    def axis(j, m):
        t = (np.arange(m) + 0.5) / m
        return omega_from_unit(np.tile(t[:, None], (1, 5)))[:, j]
    gvals = axis(which, G)
    others = [j for j in range(5) if j != which]
    subs = np.meshgrid(*[axis(j, sub) for j in others], indexing="ij")
    S = subs[0].size
    params = np.empty((G * S, 5))
    for g in range(G):
        blk = params[g * S:(g + 1) * S]
        blk[:, which] = gvals[g]
        for k, j in enumerate(others):
            blk[:, j] = subs[k].ravel()
    return gvals, params


WORKLOADS = dict(iso100=iso100, aniso1000=aniso1000, mixed4000=mixed4000, uneven=uneven)
