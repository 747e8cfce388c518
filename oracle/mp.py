"""Matching-pursuit root heuristic, FP64 (test infrastructure only).

Appendix A.2 ("Matching Pursuit Algorithm") and Section 3.5: greedy forward and
backward single-coordinate moves on Eq. original, from beta = 0.
  forward  for j not in S, with r = y - X_S beta_S, c_j = X_j^T r, D_j = ||X_j||^2 + 2 lambda2:
           beta_j = clip(c_j / D_j, [-M, M]),
           Delta_j = -beta_j c_j + 1/2 D_j beta_j^2 + lambda0   (objective change, others frozen);
           add the j of smallest Delta_j if Delta_j < 0.
  backward for j in S: Delta_j = beta_j c_j + (1/2 ||X_j||^2 - lambda2) beta_j^2 - lambda0
           (objective change of setting beta_j = 0, residual r fixed otherwise);
           remove the j of smallest Delta_j if Delta_j < 0.
Reading (the alternation is not spelled out): forward moves while one improves,
then one backward move if it improves, repeated; ties go to the lowest index; at
most `max_moves` moves.  The resulting support is polished by the exact box ridge
(oracle.ub) to give the initial incumbent.
"""
from __future__ import annotations

import numpy as np

from . import ub


def forward_deltas(X, r, lam0, lam2, M, col_sq):
    c = X.T @ r
    D = col_sq + 2.0 * lam2
    b = np.clip(c / D, -M, M)
    return -b * c + 0.5 * D * b * b + lam0, b, c


def backward_deltas(X, r, beta, lam0, lam2, col_sq):
    c = X.T @ r
    return beta * c + (0.5 * col_sq - lam2) * beta * beta - lam0, c


def matching_pursuit(X, y, lam0, lam2, M, max_moves=None):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    max_moves = max_moves or 4 * p
    col_sq = np.einsum("ij,ij->j", X, X)
    beta = np.zeros(p)
    r = y.copy()
    in_s = np.zeros(p, dtype=bool)
    moves = 0
    while moves < max_moves:
        d, b, _ = forward_deltas(X, r, lam0, lam2, M, col_sq)
        d = np.where(in_s, np.inf, d)
        j = int(np.argmin(d))
        if d[j] < 0.0:
            in_s[j] = True
            beta[j] = b[j]
            r = r - X[:, j] * b[j]
            moves += 1
            continue
        if not in_s.any():
            break
        db, _ = backward_deltas(X, r, beta, lam0, lam2, col_sq)
        db = np.where(in_s, db, np.inf)
        j = int(np.argmin(db))
        if db[j] < 0.0:
            r = r + X[:, j] * beta[j]
            beta[j] = 0.0
            in_s[j] = False
            moves += 1
            continue
        break
    return np.nonzero(in_s)[0], beta


def root_incumbent(X, y, lam0, lam2, M):
    S, _ = matching_pursuit(X, y, lam0, lam2, M)
    return ub.support_objective(X, y, S, lam0, lam2, M), S
