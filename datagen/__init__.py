"""Seeded synthetic designs for the l0-l2 sparse-regression workloads.

This module only draws inputs: it holds none of the branch-and-bound arithmetic
(no psi, prox, dual bound, ADMM or upper-bound step).  Both the FP64 oracle
tests and the CUDA path tests take their inputs from here.

Recipe (Section 5.1 "Datasets", with a Toeplitz covariance in place of the
constant-correlation one):
  * rows of X are iid N(0, Sigma) with Sigma_ij = rho^|i-j|, drawn exactly as an
    AR(1) recursion along the feature index:
        x_0 = e_0,  x_j = rho * x_{j-1} + sqrt(1 - rho^2) * e_j ;
  * the draws are staged in float32, every column is scaled to unit l2 norm
    (norms taken from the float64 draws) and the scaled matrix is rounded to
    FP32; that FP32-representable X (held in float64 arrays) is the problem data;
  * beta_true has k entries equal to 1.0 at indices floor(j * p / k);
  * y = X beta_true + eps, eps ~ N(0, sigma^2 I), sigma^2 = Var(X beta_true)/SNR
    (sample variance of the noiseless response);
  * seeds: numpy PCG64 with seed = 1000 * config_id + instance.
"""
from __future__ import annotations

import dataclasses
import numpy as np
from scipy.signal import lfilter


@dataclasses.dataclass
class Instance:
    X: np.ndarray          # (n, p) float64, FP32-representable, Fortran (column-major) order
    y: np.ndarray          # (n,) float64
    beta_true: np.ndarray  # (p,) float64
    support_true: np.ndarray  # (k,) int64
    sigma2: float
    seed: int
    rho: float
    snr: float

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def p(self) -> int:
        return self.X.shape[1]


def toeplitz_design(n: int, p: int, rho: float, rng: np.random.Generator,
                    block: int = 2048) -> np.ndarray:
    """Rows iid N(0, Sigma), Sigma_ij = rho^|i-j|, unit-norm columns, FP32-rounded.

    Rows are drawn in blocks (staged in float32); the result is a column-major
    float64 array whose entries are exactly representable in float32.
    """
    stage = np.empty((n, p), dtype=np.float32, order="F")
    s = np.sqrt(1.0 - rho * rho)
    sq = np.zeros(p)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        e = rng.standard_normal((r1 - r0, p))
        if s > 0:
            e[:, 0] /= s
            xb = lfilter([s], [1.0, -rho], e, axis=1)
        else:  # rho = +-1 degenerate: every column equals the first
            xb = np.repeat(e[:, :1], p, axis=1)
        sq += np.einsum("ij,ij->j", xb, xb)
        stage[r0:r1, :] = xb
    # unit-norm scaling (norms from the float64 draws), then the one rounding
    # to float32 that defines the problem data
    scale = 1.0 / np.sqrt(sq)
    res = np.empty((n, p), dtype=np.float64, order="F")
    for j0 in range(0, p, 4096):
        j1 = min(p, j0 + 4096)
        res[:, j0:j1] = (stage[:, j0:j1].astype(np.float64) * scale[None, j0:j1]).astype(np.float32)
    return res


def true_support(p: int, k: int) -> np.ndarray:
    return np.array([(j * p) // k for j in range(k)], dtype=np.int64)


def make_instance(n: int, p: int, rho: float, k: int, snr: float, seed: int) -> Instance:
    rng = np.random.Generator(np.random.PCG64(seed))
    X = toeplitz_design(n, p, rho, rng)
    S = true_support(p, k)
    beta = np.zeros(p)
    beta[S] = 1.0
    mu = X[:, S].sum(axis=1)
    var = float(np.var(mu))
    sigma2 = var / snr if snr > 0 else 0.0
    y = mu + np.sqrt(sigma2) * rng.standard_normal(n)
    return Instance(X=X, y=y, beta_true=beta, support_true=S, sigma2=sigma2,
                    seed=seed, rho=rho, snr=snr)


def ridge_on_support(X: np.ndarray, y: np.ndarray, S, lam2: float) -> np.ndarray:
    """argmin 0.5||y - X_S b||^2 + lam2 ||b||^2 (input recipe for the big-M value)."""
    S = np.asarray(S, dtype=np.int64)
    XS = X[:, S]
    A = XS.T @ XS + 2.0 * lam2 * np.eye(len(S))
    return np.linalg.solve(A, XS.T @ y)


def big_m(X: np.ndarray, y: np.ndarray, S, lam2: float, factor: float = 1.5) -> float:
    """M = factor * ||ridge solution restricted to the true support||_inf (Section 5.1)."""
    return float(factor * np.max(np.abs(ridge_on_support(X, y, S, lam2))))


def lambda0_scale(X: np.ndarray, y: np.ndarray, lam2: float) -> float:
    """Scale for lambda0 grids: max_j (X_j^T y)^2 / (2 (||X_j||^2 + 2 lam2)).

    This is the objective drop of the best single-coordinate fit from beta = 0
    (an input recipe used to place lambda0 values where supports change).
    """
    c = X.T @ y
    d = np.einsum("ij,ij->j", X, X) + 2.0 * lam2
    return float(np.max(c * c / (2.0 * d)))


def random_fixings(p: int, K: int, rng: np.random.Generator, max_fixed: int,
                   p_one: float = 0.3) -> np.ndarray:
    """K rows of node fixings (-1 free, 0 fixed to zero, 1 fixed to one)."""
    fix = np.full((K, p), -1, dtype=np.int8)
    for k in range(K):
        d = int(rng.integers(0, max_fixed + 1))
        idx = rng.choice(p, size=min(d, p), replace=False)
        vals = (rng.random(len(idx)) < p_one).astype(np.int8)
        fix[k, idx] = vals
    return fix


# Named workload shapes: the five workloads and small variants of the same recipe.
CONFIGS = {
    "c1": dict(n=200, p=50, rho=0.1, k=5, snr=5.0, lam2=0.01, cfg_id=1),
    "c1_p16": dict(n=200, p=16, rho=0.1, k=3, snr=5.0, lam2=0.01, cfg_id=1),
    "c2": dict(n=1000, p=5000, rho=0.3, k=10, snr=5.0, lam2=1e-3, cfg_id=2),
    "c2_small": dict(n=100, p=500, rho=0.3, k=10, snr=5.0, lam2=1e-3, cfg_id=2),
    "c3": dict(n=5000, p=50000, rho=0.5, k=20, snr=3.0, lam2=1e-3, cfg_id=3),
    "c4": dict(n=2000, p=20000, rho=0.7, k=15, snr=2.0, lam2=0.01, cfg_id=4),
    "c4_small": dict(n=200, p=2000, rho=0.7, k=15, snr=2.0, lam2=0.01, cfg_id=4),
}


def config_instance(name: str, instance: int = 0) -> Instance:
    c = CONFIGS[name]
    seed = 1000 * c["cfg_id"] + instance
    return make_instance(c["n"], c["p"], c["rho"], c["k"], c["snr"], seed)
