"""Second, independent solver for the node relaxation (test infrastructure only).

Accelerated proximal gradient (Beck and Teboulle's FISTA, with the standard
t_k sequence and function-value restart) on Eq. relaxnode2:
    min_beta 1/2 ||y - X beta||^2 + sum_i psi_i(beta_i)   s.t. ||beta||_inf <= M.
The smooth part has gradient X^T (X beta - y) and Lipschitz constant
L = ||X||_2^2; the proximal step with step 1/L is the coordinate-wise
argmin of L/2 (beta - u)^2 + psi_i(beta), which is Eq. minbetalower with
rho = L.  Used only to cross-check the ADMM oracle: the two must reach the
same relaxation value.
"""
from __future__ import annotations

import numpy as np

from . import relax


def solve_node(X, y, fix, lam0, lam2, M, tol=1e-12, max_iter=100000):
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = X.shape[1]
    L = float(np.linalg.norm(X, 2) ** 2) * (1.0 + 1e-12) + 1e-300
    beta = np.zeros(p)
    yk = beta.copy()
    t = 1.0
    fval = relax.primal_value(X, y, beta, fix, lam0, lam2, M)
    for _ in range(max_iter):
        g = X.T @ (X @ yk - y)
        new = relax.prox(yk - g / L, fix, lam0, lam2, M, L)
        fnew = relax.primal_value(X, y, new, fix, lam0, lam2, M)
        if fnew > fval:  # restart the momentum
            if t == 1.0:
                break
            t = 1.0
            yk = beta.copy()
            continue
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        yk = new + ((t - 1.0) / t_new) * (new - beta)
        done = (fval - fnew) <= tol * max(1.0, abs(fnew)) and np.max(np.abs(new - beta)) <= 1e-11
        beta, fval, t = new, fnew, t_new
        if done:
            break
    return beta, fval
