"""Upper bound on a support S, FP64 (test infrastructure only).

Eq. upperboundbeta (Section 3.3): with z fixed to the rounded support S,
    U_S(beta) = 1/2 ||y - X_S beta||^2 + lambda2 ||beta||^2,  |beta_i| <= M.

``box_ridge``  the exact minimiser by a feasible primal active-set method for
               a strictly convex bound-constrained QP (Nocedal and Wright,
               Algorithm 16.3); ``kkt_residual`` checks its optimality.
``fista_backtracking``  the paper's own method, written from Eqs.
               fpg_extrapolate, fpg_grad, fpg_step, fpg_armijo: momentum
               t/(t+3), projected step, Armijo backtracking.  Reading:
               initial step 1/L with L = ||X_S||_2^2 + 2 lambda2, step
               halved on Armijo failure, stop on relative decrease < tol.
``support_objective``  Eq. original at the minimiser, counting lambda0 once per
               nonzero coefficient (a feasible value of Eq. perspective).
"""
from __future__ import annotations

import numpy as np


def _gram(X, y, S, lam2):
    XS = X[:, S]
    Q = XS.T @ XS + 2.0 * lam2 * np.eye(len(S))
    q = XS.T @ y
    return Q, q


def box_ridge(X, y, S, lam2, M, max_iter=None):
    """Exact argmin of U_S over |beta| <= M.  Returns beta_S (len |S|)."""
    S = np.asarray(S, dtype=np.int64)
    s = len(S)
    if s == 0:
        return np.zeros(0)
    Q, q = _gram(np.asarray(X, dtype=np.float64), np.asarray(y, dtype=np.float64), S, lam2)
    beta = np.zeros(s)
    W = np.zeros(s, dtype=np.int64)  # working set: 0 free, +1 at +M, -1 at -M
    max_iter = max_iter or (10 * s + 50)
    for _ in range(max_iter):
        F = W == 0
        target = beta.copy()
        if np.any(F):
            rhs = q[F] - Q[np.ix_(F, ~F)] @ beta[~F]
            target[F] = np.linalg.solve(Q[np.ix_(F, F)], rhs)
        d = target - beta
        if np.max(np.abs(d), initial=0.0) <= 1e-15 * max(1.0, M):
            g = Q @ beta - q
            lam = np.where(W == 1, -g, np.where(W == -1, g, 0.0))
            j = int(np.argmin(lam))
            if W[j] == 0 or lam[j] >= -1e-13 * max(1.0, np.max(np.abs(q))):
                break
            W[j] = 0
            continue
        alpha = 1.0
        block = -1
        for i in np.nonzero(F & (d != 0.0))[0]:
            lim = (M - beta[i]) / d[i] if d[i] > 0 else (-M - beta[i]) / d[i]
            if lim < alpha:
                alpha, block = lim, i
        beta = beta + alpha * d
        if block >= 0:
            W[block] = 1 if d[block] > 0 else -1
            beta[block] = M * W[block]
    return np.clip(beta, -M, M)


def kkt_residual(X, y, S, lam2, M, beta_S):
    """Largest violation of the KKT conditions of Eq. upperboundbeta at beta_S."""
    S = np.asarray(S, dtype=np.int64)
    if len(S) == 0:
        return 0.0
    Q, q = _gram(np.asarray(X, dtype=np.float64), np.asarray(y, dtype=np.float64), S, lam2)
    g = Q @ beta_S - q
    viol = np.where(np.abs(beta_S) < M, np.abs(g),
                    np.where(beta_S >= M, np.maximum(g, 0.0), np.maximum(-g, 0.0)))
    viol = np.maximum(viol, np.maximum(np.abs(beta_S) - M, 0.0))
    return float(np.max(viol))


def u_value(X, y, S, lam2, beta_S):
    r = y - X[:, S] @ beta_S
    return 0.5 * float(r @ r) + lam2 * float(beta_S @ beta_S)


def fista_backtracking(X, y, S, lam2, M, tol=1e-14, max_iter=20000, shrink=0.5):
    """Eqs. fpg_extrapolate .. fpg_armijo on one support; returns beta_S."""
    S = np.asarray(S, dtype=np.int64)
    XS = np.asarray(X, dtype=np.float64)[:, S]
    y = np.asarray(y, dtype=np.float64)
    s = len(S)
    if s == 0:
        return np.zeros(0)
    L = float(np.linalg.norm(XS, 2) ** 2) + 2.0 * lam2
    alpha = 1.0 / L

    def U(b):
        r = y - XS @ b
        return 0.5 * float(r @ r) + lam2 * float(b @ b)

    cur = np.zeros(s)
    prev = cur.copy()
    fcur = U(cur)
    for t in range(max_iter):
        ext = cur + (t / (t + 3.0)) * (cur - prev)              # Eq. fpg_extrapolate
        g = XS.T @ (XS @ ext - y) + 2.0 * lam2 * ext            # Eq. fpg_grad
        fext = U(ext)
        while True:
            new = np.clip(ext - alpha * g, -M, M)               # Eq. fpg_step
            d = new - ext
            if U(new) <= fext + float(g @ d) + float(d @ d) / (2.0 * alpha) + 1e-15 * abs(fext):
                break                                           # Eq. fpg_armijo
            alpha *= shrink
        fnew = U(new)
        prev, cur = cur, new
        if abs(fcur - fnew) <= tol * max(1.0, abs(fnew)) and np.max(np.abs(cur - prev)) <= 1e-13:
            break
        fcur = fnew
    return cur


def support_objective(X, y, S, lam0, lam2, M):
    """(objective, full beta) of the box ridge on S, counting lambda0 per nonzero."""
    X = np.asarray(X, dtype=np.float64)
    p = X.shape[1]
    S = np.asarray(S, dtype=np.int64)
    beta = np.zeros(p)
    if len(S):
        beta[S] = box_ridge(X, y, S, lam2, M)
    r = y - X @ beta
    obj = 0.5 * float(r @ r) + lam0 * float(np.count_nonzero(beta)) + lam2 * float(beta @ beta)
    return obj, beta
