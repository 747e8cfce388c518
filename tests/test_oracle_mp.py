"""Pins for the matching-pursuit heuristic: the closed-form objective changes of
Appendix A.2 equal direct differences of Eq. original, and the heuristic only
ever improves the objective and returns a feasible support."""
import numpy as np
import pytest

import datagen
from oracle import mp, relax, ub


def _inst(seed=0):
    inst = datagen.make_instance(80, 30, 0.3, 4, 5.0, seed)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.05 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    return inst, lam0, lam2, M


@pytest.mark.parametrize("mfac", [1.5, 0.2])
def test_forward_delta_is_objective_change(mfac):
    inst, lam0, lam2, M = _inst(1)
    M *= mfac
    rng = np.random.default_rng(2)
    X, y = inst.X, inst.y
    beta = np.zeros(inst.p)
    S = rng.choice(inst.p, 4, replace=False)
    beta[S] = rng.uniform(-M, M, 4)
    r = y - X @ beta
    col_sq = np.einsum("ij,ij->j", X, X)
    d, b, _ = mp.forward_deltas(X, r, lam0, lam2, M, col_sq)
    base = relax.mip_objective(X, y, beta, lam0, lam2)
    for j in range(inst.p):
        if j in S or b[j] == 0.0:
            continue
        assert abs(b[j]) <= M          # the single-coordinate step stays in the box
        nb = beta.copy()
        nb[j] = b[j]
        assert d[j] == pytest.approx(relax.mip_objective(X, y, nb, lam0, lam2) - base, abs=1e-10)
        # and b_j is the best single-coordinate value on the box (grid check)
        grid = np.linspace(-M, M, 2001)
        vals = [0.5 * np.sum((r - X[:, j] * g) ** 2) + lam2 * g * g for g in grid]
        assert 0.5 * np.sum((r - X[:, j] * b[j]) ** 2) + lam2 * b[j] ** 2 <= min(vals) + 1e-12


def test_backward_delta_is_objective_change():
    inst, lam0, lam2, M = _inst(3)
    rng = np.random.default_rng(4)
    X, y = inst.X, inst.y
    beta = np.zeros(inst.p)
    S = rng.choice(inst.p, 5, replace=False)
    beta[S] = rng.uniform(-M, M, 5)
    r = y - X @ beta
    col_sq = np.einsum("ij,ij->j", X, X)
    d, _ = mp.backward_deltas(X, r, beta, lam0, lam2, col_sq)
    base = relax.mip_objective(X, y, beta, lam0, lam2)
    for j in S:
        nb = beta.copy()
        nb[j] = 0.0
        assert d[j] == pytest.approx(relax.mip_objective(X, y, nb, lam0, lam2) - base, abs=1e-10)


def test_heuristic_improves_and_is_feasible():
    inst, lam0, lam2, M = _inst(5)
    S, beta = mp.matching_pursuit(inst.X, inst.y, lam0, lam2, M)
    assert np.all(np.abs(beta) <= M)
    obj0 = relax.mip_objective(inst.X, inst.y, np.zeros(inst.p), lam0, lam2)
    obj = relax.mip_objective(inst.X, inst.y, beta, lam0, lam2)
    assert obj < obj0
    (pol, bpol), S2 = mp.root_incumbent(inst.X, inst.y, lam0, lam2, M)
    assert pol <= obj + 1e-12
    assert ub.kkt_residual(inst.X, inst.y, S2, lam2, M, bpol[S2]) < 1e-9


def test_matching_pursuit_orthonormal_design():
    """X^T X = I: single-coordinate moves do not interact, so the greedy search must end
    on exactly the coordinates whose own gain beats lambda0 (the separable MIP optimum,
    beta_j = clip(c_j / (1 + 2 lambda2), +-M) kept when its gain exceeds lambda0)."""
    rng = np.random.default_rng(21)
    n, p = 40, 12
    Q, _ = np.linalg.qr(rng.normal(size=(n, p)))
    y = Q @ rng.normal(0, 1, p) + 0.1 * rng.normal(size=n)
    lam0, lam2, M = 0.15, 0.05, 0.9
    c = Q.T @ y
    bj = np.clip(c / (1 + 2 * lam2), -M, M)
    keep = c * bj - (0.5 + lam2) * bj * bj > lam0
    assert 0 < keep.sum() < p and np.any(np.abs(c / (1 + 2 * lam2)) > M)
    S, beta = mp.matching_pursuit(Q, y, lam0, lam2, M)
    assert set(S.tolist()) == set(np.nonzero(keep)[0].tolist())
    np.testing.assert_allclose(beta[keep], bj[keep], atol=1e-12)


# the second case is one where the search must take a backward move to stop (found by
# scanning seeds: with forward moves only it ends on a larger support)
@pytest.mark.parametrize("case", [(80, 30, 0.3, 4, 5.0, 5, 0.05), (60, 25, 0.7, 5, 3.0, 934, 0.1)])
def test_matching_pursuit_ends_at_a_single_move_optimum(case):
    """Where the greedy search stops (Appendix A.2), no single move improves Eq. original:
    setting one coordinate outside S to any value on a grid of [-M, M], or one coordinate
    in S to zero, never lowers the objective (checked by direct evaluation)."""
    n, p, rho, k, snr, seed, frac = case
    inst = datagen.make_instance(n, p, rho, k, snr, seed)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    X, y = inst.X, inst.y
    S, beta = mp.matching_pursuit(X, y, lam0, lam2, M)
    assert len(S) > 0
    base = relax.mip_objective(X, y, beta, lam0, lam2)
    grid = np.linspace(-M, M, 801)
    for j in range(inst.p):
        trial = beta.copy()
        if j in S:
            trial[j] = 0.0
            assert relax.mip_objective(X, y, trial, lam0, lam2) >= base - 1e-12
        else:
            for g in grid:
                trial[j] = g
                assert relax.mip_objective(X, y, trial, lam0, lam2) >= base - 1e-12
