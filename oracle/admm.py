"""ADMM for one node relaxation, FP64, direct D (test infrastructure only).

Follows Section 3.1: the splitting b = beta of Eq. ADMM1, the augmented
Lagrangian Eq. ADMM2 and the update order of Eq. admm-update:
    b    = D (c + rho beta - v),  D = (X^T X + rho I)^{-1},  c = X^T y   (Eq. b_update)
    beta = prox(b + v / rho)                                              (Eq. minbetalower)
    v    = v + rho (b - beta)                                             (Eq. v_i-update)
The dual candidate is r = y - X b (text after Proposition 1).  D is formed
directly (no Woodbury) so that the oracle does not share the CUDA path's
rewrite of the b-update.

Over-relaxation (not in the paper; an option of the engine, from Boyd, Parikh,
Chu, Peleato and Eckstein, "Distributed Optimization and Statistical Learning
via the Alternating Direction Method of Multipliers", 2011, Section 3.4.3): with
alpha != 1 the beta- and v-updates use bh = alpha b + (1 - alpha) beta_prev in
place of b.  alpha = 1 is the paper's iteration.

Node stop rule (Section 5.1 "BnB Settings"): relative primal-dual gap
(P(beta) - D(r)) / max(1, |P(beta)|) <= tol, P from Eq. relaxnode2 at the
feasible beta and D from Eq. dual (the best D seen so far is kept: every r
gives a valid bound).
"""
from __future__ import annotations

import dataclasses
import numpy as np

from . import relax


@dataclasses.dataclass
class AdmmResult:
    beta: np.ndarray
    b: np.ndarray
    v: np.ndarray
    r: np.ndarray
    primal: float
    dual: float
    iters: int

    @property
    def gap(self) -> float:
        return (self.primal - self.dual) / max(1.0, abs(self.primal))


class AdmmData:
    """Per-tree shared data: X, y, c = X^T y and D (Section 3.2, shared reference)."""

    def __init__(self, X, y, rho):
        self.X = np.asarray(X, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.rho = float(rho)
        p = self.X.shape[1]
        self.c = self.X.T @ self.y
        self.D = np.linalg.inv(self.X.T @ self.X + self.rho * np.eye(p))


def admm_iteration(data: AdmmData, beta, v, fix, lam0, lam2, M, alpha=1.0):
    """One pass of Eq. admm-update (over-relaxed when alpha != 1); returns (b, beta_new, v_new)."""
    rho = data.rho
    b = data.D @ (data.c + rho * beta - v)
    bh = b if alpha == 1.0 else alpha * b + (1.0 - alpha) * beta
    bt = bh + v / rho
    beta_new = relax.prox(bt, fix, lam0, lam2, M, rho)
    v_new = v + rho * (bh - beta_new)
    return b, beta_new, v_new


def solve_node(data: AdmmData, fix, lam0, lam2, M, beta0=None, v0=None,
               tol=1e-10, max_iter=20000, check_every=10, alpha=1.0) -> AdmmResult:
    X, y = data.X, data.y
    p = X.shape[1]
    fix = np.asarray(fix)
    beta = np.zeros(p) if beta0 is None else np.array(beta0, dtype=np.float64)
    v = np.zeros(p) if v0 is None else np.array(v0, dtype=np.float64)
    b = beta.copy()
    primal = np.inf
    best_dual = -np.inf
    best_r = y.copy()
    it = 0
    while it < max_iter:
        b, beta, v = admm_iteration(data, beta, v, fix, lam0, lam2, M, alpha)
        it += 1
        if it % check_every == 0 or it == max_iter:
            r = y - X @ b
            dual = relax.dual_value(X, y, r, fix, lam0, lam2, M)
            if dual > best_dual:
                best_dual, best_r = dual, r
            primal = relax.primal_value(X, y, beta, fix, lam0, lam2, M)
            if (primal - best_dual) / max(1.0, abs(primal)) <= tol:
                break
    return AdmmResult(beta=beta, b=b, v=v, r=best_r, primal=primal, dual=best_dual, iters=it)
