"""Brute-force optimum of Eq. perspective for p <= 16 (test infrastructure only).

With z fixed, Eq. perspective is lambda0 |S| plus the box ridge of Eq.
upperboundbeta on S = {i : z_i = 1}; so its optimum is
    min over S subset of [p] of  lambda0 |S| + min_{|beta_S| <= M} U_S(beta_S).
Every support is enumerated.  The unconstrained ridge of each support is a
linear solve with X_S^T X_S + 2 lambda2 I; supports whose ridge solution leaves
the box are re-solved exactly by ``ub.box_ridge``.  The result carries the
best and second-best objective, whose difference is the certified margin of
the optimal support.
"""
from __future__ import annotations

import dataclasses
import itertools
import numpy as np

from . import ub


@dataclasses.dataclass
class BruteResult:
    support: tuple
    beta: np.ndarray
    objective: float
    second: float

    @property
    def margin(self) -> float:
        return self.second - self.objective


def solve(X, y, lam0, lam2, M, max_p=16) -> BruteResult:
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    if p > max_p:
        raise ValueError(f"brute force limited to p <= {max_p}")
    G = X.T @ X
    c = X.T @ y
    yy = float(y @ y)
    vals = [((), 0.5 * yy)]
    for s in range(1, p + 1):
        combos = np.array(list(itertools.combinations(range(p), s)), dtype=np.int64).reshape(-1, s)
        A = G[combos[:, :, None], combos[:, None, :]] + 2.0 * lam2 * np.eye(s)[None]
        rhs = c[combos]
        sol = np.linalg.solve(A, rhs[..., None])[..., 0]
        bad = np.max(np.abs(sol), axis=1) > M
        for i in np.nonzero(bad)[0]:
            sol[i] = ub.box_ridge(X, y, combos[i], lam2, M)
        # 1/2||y - X_S b||^2 + lam2||b||^2 = 1/2 y^T y - c_S^T b + 1/2 b^T (G_SS + 2 lam2 I) b
        quad = np.einsum("ki,kij,kj->k", sol, A, sol)
        val = 0.5 * yy - np.einsum("ki,ki->k", rhs, sol) + 0.5 * quad + lam0 * s
        vals.extend((tuple(int(t) for t in combos[i]), float(val[i])) for i in range(len(combos)))
    vals.sort(key=lambda t: t[1])
    bestS, best = vals[0]
    second = vals[1][1] if len(vals) > 1 else np.inf
    beta = np.zeros(p)
    if bestS:
        S = np.array(bestS, dtype=np.int64)
        beta[S] = ub.box_ridge(X, y, S, lam2, M)
    return BruteResult(support=bestS, beta=beta, objective=best, second=second)
