"""Closed forms of the node relaxation, FP64 (test infrastructure only).

Fixing codes used throughout: FREE = -1, F0 = 0 (z_i = 0), F1 = 1 (z_i = 1).

Passages followed:
  * Eq. relaxnode / Eq. relaxnode2 and Eq. psi (Section 3.1): the relaxation
    reduced to beta, with the four-case psi_i.
  * Eq. Tdef: the box-constrained soft-threshold T(t; a, m).
  * Eq. minbetalower with its derivation in Appendix A.1: the beta-update.
    Reading: the regime test sqrt(lambda0/lambda2) > M is applied first for
    free coordinates (Appendix A.1 case 4 holds for all free i in that
    regime); in the other regime the full two-branch rule is used, including
    the ridge branch for |beta~| >= 2 sqrt(l0 l2)/rho + sqrt(l0/l2).
  * Appendix A.1 ("Derivation of problem relaxnode2"): z_i, s_i recovery.
  * Proposition 1, Eqs. hdef, dual, nudef: the dual bound valid for every r.
"""
from __future__ import annotations

import numpy as np

FREE, F0, F1 = -1, 0, 1


def _free_regime_linear(lam0: float, lam2: float, M: float) -> bool:
    """True when sqrt(lambda0/lambda2) > M (psi linear on the whole box)."""
    return np.sqrt(lam0 / lam2) > M


def T(t, a, m):
    """Eq. Tdef: 0 if |t| <= a; (|t| - a) sign(t) if a < |t| <= a + m; m sign(t) otherwise."""
    t = np.asarray(t, dtype=np.float64)
    at = np.abs(t)
    return np.where(at <= a, 0.0, np.where(at <= a + m, (at - a) * np.sign(t), m * np.sign(t)))


def psi(beta, fix, lam0, lam2, M):
    """Eq. psi, per coordinate; +inf outside the feasible set (|beta| <= M, beta_F0 = 0)."""
    beta = np.asarray(beta, dtype=np.float64)
    fix = np.asarray(fix)
    ab = np.abs(beta)
    s0 = np.sqrt(lam0 / lam2)
    ridge = lam0 + lam2 * beta * beta
    if _free_regime_linear(lam0, lam2, M):
        free_val = (lam0 / M + lam2 * M) * ab
    else:
        free_val = np.where(ab <= s0, 2.0 * np.sqrt(lam0 * lam2) * ab, ridge)
    out = np.where(fix == F1, ridge, free_val)
    out = np.where(fix == F0, np.where(beta == 0.0, 0.0, np.inf), out)
    out = np.where(ab > M, np.inf, out)
    return out


def prox(bt, fix, lam0, lam2, M, rho):
    """Eq. minbetalower: argmin_b rho/2 (b - bt)^2 + psi_i(b) s.t. |b| <= M, per coordinate."""
    bt = np.asarray(bt, dtype=np.float64)
    fix = np.asarray(fix)
    ridge = np.clip(rho / (rho + 2.0 * lam2) * bt, -M, M)
    if _free_regime_linear(lam0, lam2, M):
        free = T(bt, (lam0 / M + lam2 * M) / rho, M)
    else:
        a = 2.0 * np.sqrt(lam0 * lam2) / rho
        tau = a + np.sqrt(lam0 / lam2)
        free = np.where(np.abs(bt) >= tau, ridge, T(bt, a, M))
    out = np.where(fix == F1, ridge, free)
    out = np.where(fix == F0, 0.0, out)
    return out


def z_of_beta(beta, fix, lam0, lam2, M):
    """Appendix A.1: optimal z_i for fixed beta (F0 -> 0, F1 -> 1, free -> three sub-cases)."""
    beta = np.asarray(beta, dtype=np.float64)
    fix = np.asarray(fix)
    ab = np.abs(beta)
    if lam0 == 0.0:
        zf = np.where(ab > 0.0, 1.0, 0.0)
    else:
        zf = np.minimum(1.0, np.maximum(ab / M, np.sqrt(lam2 / lam0) * ab))
    z = np.where(fix == F1, 1.0, zf)
    z = np.where(fix == F0, 0.0, z)
    return z


def h(x, lam0, lam2, M):
    """Eq. hdef."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x <= 2.0 * M * lam2, x * x / (4.0 * lam2) - lam0, M * x - lam0 - lam2 * M * M)


def nu(x, fix, lam0, lam2, M):
    """Eq. nudef, evaluated at x = |X_i^T r| >= 0."""
    x = np.asarray(x, dtype=np.float64)
    fix = np.asarray(fix)
    hx = h(x, lam0, lam2, M)
    if _free_regime_linear(lam0, lam2, M):
        free = np.maximum(M * x - lam0 - lam2 * M * M, 0.0)
    else:
        free = np.maximum(hx, 0.0)
    out = np.where(fix == F1, hx, free)
    out = np.where(fix == F0, 0.0, out)
    return out


def primal_value(X, y, beta, fix, lam0, lam2, M):
    """Objective of Eq. relaxnode2 at beta (inf if beta is infeasible)."""
    r = y - X @ beta
    return 0.5 * float(r @ r) + float(np.sum(psi(beta, fix, lam0, lam2, M)))


def dual_value(X, y, r, fix, lam0, lam2, M):
    """Eq. dual at r: -1/2||r||^2 + y^T r - sum_i nu_i(|X_i^T r|) (a lower bound for every r)."""
    r = np.asarray(r, dtype=np.float64)
    g = X.T @ r
    return -0.5 * float(r @ r) + float(y @ r) - float(np.sum(nu(np.abs(g), fix, lam0, lam2, M)))


def mip_objective(X, y, beta, lam0, lam2):
    """Eq. original: 1/2||y - X beta||^2 + lambda0 ||beta||_0 + lambda2 ||beta||^2."""
    r = y - X @ beta
    return 0.5 * float(r @ r) + lam0 * float(np.count_nonzero(beta)) + lam2 * float(beta @ beta)
