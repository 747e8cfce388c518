"""Pins for the oracle's solvers: duality, two independent relaxation solvers,
the exact box ridge against a library routine, brute force against the
branch-and-bound, the orthonormal special case and the BnB invariants."""
import numpy as np
import pytest
from scipy.optimize import lsq_linear

import datagen
from oracle import relax, admm, pgd, ub, brute, bnb


def _small(seed=0, n=60, p=12, rho=0.3, k=3, snr=5.0):
    return datagen.make_instance(n, p, rho, k, snr, seed)


def _params(inst, lam2=0.01, frac=0.05, mfac=1.5):
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2, mfac)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    return lam0, lam2, M


# ---------------------------------------------------------------- duality


@pytest.mark.parametrize("mfac", [1.5, 0.3])   # both regimes of Eq. psi
def test_weak_duality_random_r(mfac):
    inst = _small(1)
    lam0, lam2, M = _params(inst, mfac=mfac)
    rng = np.random.default_rng(0)
    X, y = inst.X, inst.y
    for _ in range(200):
        fix = datagen.random_fixings(inst.p, 1, rng, 5)[0]
        r = y * rng.uniform(-1, 2) + rng.normal(0, 1, inst.n)
        beta = rng.uniform(-M, M, inst.p)
        beta[fix == relax.F0] = 0.0
        d = relax.dual_value(X, y, r, fix, lam0, lam2, M)
        pval = relax.primal_value(X, y, beta, fix, lam0, lam2, M)
        assert d <= pval + 1e-12


# rho != 1 separates v from v / rho; y -> -y flips every coefficient (psi is even), so
# the negative side of each closed form is exercised too
@pytest.mark.parametrize("mfac,rho,ysign", [(1.5, 1.0, 1), (0.3, 1.0, 1), (1.5, 0.35, 1),
                                            (0.3, 0.35, 1), (1.5, 1.0, -1), (0.3, 0.35, -1)])
def test_admm_matches_second_solver_and_strong_duality(mfac, rho, ysign):
    inst = _small(2)
    lam0, lam2, M = _params(inst, mfac=mfac)
    y = ysign * inst.y
    rng = np.random.default_rng(4)
    data = admm.AdmmData(inst.X, y, rho)
    for _ in range(4):
        fix = datagen.random_fixings(inst.p, 1, rng, 4)[0]
        a = admm.solve_node(data, fix, lam0, lam2, M, tol=1e-12, max_iter=200000)
        b, fb = pgd.solve_node(inst.X, y, fix, lam0, lam2, M)
        # strong duality at the ADMM optimum (Proposition 1.2, 1.3)
        assert a.primal - a.dual <= 1e-9 * max(1.0, abs(a.primal))
        # two independent algorithms reach the same relaxation value
        assert a.primal == pytest.approx(fb, rel=1e-9, abs=1e-10)
        # and the dual bound never exceeds the relaxation optimum
        assert a.dual <= fb + 1e-10


@pytest.mark.parametrize("mfac,ysign", [(1.5, 1), (0.3, -1)])
def test_over_relaxed_admm_reaches_the_same_optimum(mfac, ysign):
    """Over-relaxation (alpha = 1.6) changes the iterates, not the fixed point: strong
    duality at convergence and agreement with the independent second solver; and one
    over-relaxed step differs from the plain one (the option is not a no-op)."""
    inst = _small(2)
    lam0, lam2, M = _params(inst, mfac=mfac)
    y = ysign * inst.y
    rng = np.random.default_rng(14)
    data = admm.AdmmData(inst.X, y, 0.35)
    for _ in range(3):
        fix = datagen.random_fixings(inst.p, 1, rng, 4)[0]
        a = admm.solve_node(data, fix, lam0, lam2, M, tol=1e-12, max_iter=200000, alpha=1.6)
        _, fb = pgd.solve_node(inst.X, y, fix, lam0, lam2, M)
        assert a.primal - a.dual <= 1e-9 * max(1.0, abs(a.primal))
        assert a.primal == pytest.approx(fb, rel=1e-9, abs=1e-10)
    beta0 = rng.uniform(-M, M, inst.p) * (fix != relax.F0)
    v0 = rng.normal(size=inst.p)
    _, b1, v1 = admm.admm_iteration(data, beta0, v0, fix, lam0, lam2, M)
    _, b2, v2 = admm.admm_iteration(data, beta0, v0, fix, lam0, lam2, M, alpha=1.6)
    assert np.max(np.abs(v1 - v2)) > 1e-6


def test_woodbury_reading():
    """b-update inverse: (1/rho)(I - X^T (X X^T + rho I)^{-1} X) is the inverse of
    X^T X + rho I; the printed coefficient 1/rho^2 on the second term is not."""
    rng = np.random.default_rng(5)
    n, p, rho = 7, 19, 2.5
    X = rng.normal(size=(n, p))
    A = X.T @ X + rho * np.eye(p)
    inner = np.linalg.inv(X @ X.T + rho * np.eye(n))
    good = (np.eye(p) - X.T @ inner @ X) / rho
    printed = np.eye(p) / rho - X.T @ inner @ X / rho**2
    assert np.max(np.abs(good @ A - np.eye(p))) < 1e-12
    assert np.max(np.abs(printed @ A - np.eye(p))) > 1e-2


def test_admm_iteration_identity_u_equals_xb():
    """With the exact b-update, X b = (X X^T + rho I)^{-1} X w (push-through identity)."""
    inst = _small(3)
    rho = 0.7
    data = admm.AdmmData(inst.X, inst.y, rho)
    rng = np.random.default_rng(6)
    w = rng.normal(size=inst.p)
    b = data.D @ w
    U = np.linalg.solve(inst.X @ inst.X.T + rho * np.eye(inst.n), inst.X @ w)
    assert np.max(np.abs(inst.X @ b - U)) < 1e-10


# ---------------------------------------------------------------- upper bound


@pytest.mark.parametrize("M", [10.0, 0.4, 0.15])   # box loose, binding, strongly binding
def test_box_ridge_matches_library(M):
    inst = _small(7, n=80, p=14, k=5)
    X, y, lam2 = inst.X, inst.y, 0.02
    rng = np.random.default_rng(8)
    for t in range(20):
        y = inst.y if t % 2 == 0 else -inst.y     # upper and lower bounds binding
        S = np.sort(rng.choice(inst.p, size=int(rng.integers(1, 9)), replace=False))
        b = ub.box_ridge(X, y, S, lam2, M)
        A = np.vstack([X[:, S], np.sqrt(2 * lam2) * np.eye(len(S))])
        rhs = np.concatenate([y, np.zeros(len(S))])
        ref = lsq_linear(A, rhs, bounds=(-M, M), tol=1e-15, lsmr_tol=1e-15, max_iter=10000).x
        assert ub.kkt_residual(X, y, S, lam2, M, b) < 1e-10
        assert ub.u_value(X, y, S, lam2, b) <= ub.u_value(X, y, S, lam2, ref) + 1e-12
        np.testing.assert_allclose(b, ref, atol=1e-7)
        f = ub.fista_backtracking(X, y, S, lam2, M)
        assert ub.u_value(X, y, S, lam2, f) == pytest.approx(ub.u_value(X, y, S, lam2, b), rel=1e-10)


# ---------------------------------------------------------------- optimum


@pytest.mark.parametrize("lam0", [0.05, 3.0, 30.0])   # the best support has 2, 1 and 0 features
@pytest.mark.parametrize("M", [100.0, 0.5])           # box loose; box binding
def test_brute_force_two_features_by_hand(lam0, M):
    """p = 2: enumerate the four supports by explicit formulas (the normal equations,
    or a library bound-constrained least squares when the box binds); best and
    second best."""
    rng = np.random.default_rng(9)
    X = rng.normal(size=(10, 2))
    y = X @ np.array([1.1, -0.6]) + 0.4 * rng.normal(size=10)
    lam2 = 0.05

    def ridge_val(cols):
        if not cols:
            return 0.5 * y @ y
        A = X[:, cols]
        b = np.linalg.solve(A.T @ A + 2 * lam2 * np.eye(len(cols)), A.T @ y)
        if np.max(np.abs(b)) > M:
            Aug = np.vstack([A, np.sqrt(2 * lam2) * np.eye(len(cols))])
            b = lsq_linear(Aug, np.concatenate([y, np.zeros(len(cols))]), bounds=(-M, M),
                           tol=1e-15, lsmr_tol=1e-15, max_iter=10000).x
        r = y - A @ b
        return 0.5 * r @ r + lam2 * b @ b + lam0 * len(cols)

    vals = {(): ridge_val([]), (0,): ridge_val([0]), (1,): ridge_val([1]), (0, 1): ridge_val([0, 1])}
    order = sorted(vals, key=vals.get)
    res = brute.solve(X, y, lam0, lam2, M)
    assert res.support == order[0]
    assert res.objective == pytest.approx(vals[order[0]], rel=1e-11)
    assert res.second == pytest.approx(vals[order[1]], rel=1e-11)


@pytest.mark.parametrize("frac", [0.5, 0.05, 0.005])
def test_bnb_matches_brute_force_p16(frac):
    inst = datagen.config_instance("c1_p16", 0)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res = bnb.solve(inst.X, inst.y, lam0, lam2, M, gap=1e-9)
    assert tuple(np.nonzero(res.beta)[0]) == br.support
    assert res.ub == pytest.approx(br.objective, rel=1e-9)
    # invariants: LB <= opt <= UB along the whole run
    for _, U, L in res.history:
        assert L <= br.objective * (1 + 1e-9) + 1e-12
        assert U >= br.objective * (1 - 1e-12)


def _check_bound_inheritance(node_log):
    """Every solved child carries its parent's bound max(LB_parent, D(r)) (Algorithm 1).
    The parent is the one solved node that equals the child with one index freed."""
    seen = {fix.tobytes(): (lbp, d) for fix, lbp, d in node_log}
    assert len(seen) == len(node_log)
    for fix, lbp, _ in node_log[1:]:
        parents = []
        for j in np.nonzero(fix != relax.FREE)[0]:
            cand = fix.copy()
            cand[j] = relax.FREE
            if cand.tobytes() in seen:
                parents.append(seen[cand.tobytes()])
        assert len(parents) == 1
        plbp, pd = parents[0]
        assert lbp == max(plbp, pd)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("frac", [0.2, 0.02, 0.002])
def test_bnb_leaf_incumbents_match_brute_force(seed, frac):
    """Incumbents taken at leaves only: the optimum is then reached by the search
    itself (both children of every branch, best-first selection, pruning, the
    global bound), not by a lucky rounding.  Exact node solves and loose batched
    ones (Prop. 1.1: every r gives a valid bound) must both find it."""
    inst = datagen.make_instance(50, 10, 0.5, 3, 3.0, 700 + seed)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    assert br.margin > 1e-9 * br.objective
    for kw in (dict(K=1), dict(K=3, node_tol=1e-2, max_admm_iter=10)):
        res = bnb.solve(inst.X, inst.y, lam0, lam2, M, gap=1e-9, round_incumbent=False, **kw)
        assert res.status == "optimal"
        assert tuple(np.nonzero(res.beta)[0]) == br.support
        assert res.ub == pytest.approx(br.objective, rel=1e-10)
        for _, U, L in res.history:
            assert L <= br.objective * (1 + 1e-12)
            assert U >= br.objective * (1 - 1e-12)
        if kw["K"] == 1:
            # best-first (Section 2.2.1): children inherit at least their parent's bound,
            # so the bounds of the nodes taken one at a time never decrease
            keys = np.array([lbp for _, lbp, _ in res.node_log])
            assert np.all(keys[1:] >= keys[:-1])
            _check_bound_inheritance(res.node_log)


@pytest.mark.parametrize("K", [1, 4])
def test_bnb_batched_selection_same_optimum(K):
    inst = datagen.config_instance("c1_p16", 1)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.02 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res = bnb.solve(inst.X, inst.y, lam0, lam2, M, gap=1e-9, K=K)
    assert tuple(np.nonzero(res.beta)[0]) == br.support


def test_bnb_exact_with_loose_node_solves():
    """Prop. 1.1: the dual bound holds for every r, so stopping ADMM early weakens
    bounds but never loses the optimum.  Every node whose fixings keep the optimal
    support feasible must report a bound below the optimum."""
    inst = datagen.config_instance("c1_p16", 2)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.02 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res = bnb.solve(inst.X, inst.y, lam0, lam2, M, gap=1e-9, node_tol=1e-2, max_admm_iter=20)
    assert tuple(np.nonzero(res.beta)[0]) == br.support
    for _, U, L in res.history:
        assert L <= br.objective * (1 + 1e-12)
    opt = np.zeros(inst.p, dtype=bool)
    opt[list(br.support)] = True
    checked = 0
    for fix, lbp, d in res.node_log:
        if np.all(~opt[fix == relax.F0]) and np.all(opt[fix == relax.F1]):
            assert d <= br.objective * (1 + 1e-12)
            checked += 1
    assert checked >= 1


@pytest.mark.parametrize("mfac", [1.5, 0.3])   # both regimes of Eq. psi
def test_primal_at_feasible_points_bounds_the_node_value_from_above(mfac):
    """The premise of the early-branch node stop: the relaxation objective at any point
    feasible for the node (|beta_i| <= M, beta = 0 on F0) -- in particular every ADMM iterate
    after its prox step -- is at least the node's relaxation value (from the independent
    second solver), so a primal value below the prune threshold proves the node cannot be
    pruned.  A point outside the box is infeasible and has no such bound (psi = inf)."""
    inst = _small(4)
    lam0, lam2, M = _params(inst, frac=0.03, mfac=mfac)
    X, y = inst.X, inst.y
    rng = np.random.default_rng(7)
    data = admm.AdmmData(X, y, 0.5)
    for trial in range(6):
        fix = np.full(inst.p, relax.FREE, dtype=np.int8)
        idx = rng.choice(inst.p, size=4, replace=False)
        fix[idx[:2]] = relax.F0
        fix[idx[2:3]] = relax.F1
        _, opt = pgd.solve_node(X, y, fix, lam0, lam2, M)
        for _ in range(20):
            b = rng.uniform(-M, M, inst.p) * (rng.random(inst.p) < 0.5)
            b[fix == relax.F0] = 0.0
            assert relax.primal_value(X, y, b, fix, lam0, lam2, M) >= opt - 1e-12 * max(1.0, abs(opt))
        beta = np.zeros(inst.p)
        v = np.zeros(inst.p)
        for _ in range(15):
            _, beta, v = admm.admm_iteration(data, beta, v, fix, lam0, lam2, M)
            assert np.all(np.abs(beta) <= M * (1 + 1e-15)) and np.all(beta[fix == relax.F0] == 0)
            assert relax.primal_value(X, y, beta, fix, lam0, lam2, M) >= opt - 1e-12 * max(1.0, abs(opt))
    out = np.zeros(inst.p)
    out[0] = 2 * M
    assert relax.primal_value(X, y, out, np.full(inst.p, relax.FREE, np.int8), lam0, lam2, M) == np.inf


def test_branch_index_hand_cases():
    """The branching rule on hand-made inputs: the most fractional free z_i
    (min(z, 1 - z) largest), the lowest index on ties, fixed indices never chosen, and
    with every free z integral the free index of largest |X_i^T r|; -1 at a leaf."""
    FR, Z, O = relax.FREE, relax.F0, relax.F1
    g = np.array([0.1, -3.0, 2.0, 0.5, -0.2])
    fix = np.array([FR, FR, FR, FR, FR], dtype=np.int8)
    assert bnb.branch_index(np.array([0.2, 0.9, 0.45, 0.1, 0.0]), fix, g) == 2
    assert bnb.branch_index(np.array([0.25, 0.75, 0.0, 0.25, 1.0]), fix, g) == 0  # three-way tie
    fix2 = np.array([Z, FR, O, FR, FR], dtype=np.int8)
    assert bnb.branch_index(np.array([0.0, 0.8, 0.5, 0.4, 0.1]), fix2, g) == 3
    g2 = np.array([0.1, 0.2, 2.0, -0.5, -0.9])
    assert bnb.branch_index(np.array([0.0, 1.0, 1.0, 0.0, 0.0]), fix2, g2) == 4  # |g| = 0.9
    assert bnb.branch_index(np.array([0.0, 0.0, 1.0, 1.0, 0.0]),
                            np.array([Z, Z, O, FR, FR], dtype=np.int8), g) == 3
    assert bnb.branch_index(np.zeros(5), np.array([Z, O, O, Z, Z], dtype=np.int8), g) == -1


def test_orthonormal_design_closed_form():
    """X^T X = I: the problem separates per coordinate (a textbook case)."""
    rng = np.random.default_rng(10)
    n, p = 40, 10
    Q, _ = np.linalg.qr(rng.normal(size=(n, p)))
    X = Q
    y = X @ rng.normal(0, 1, p) * 0.8 + 0.1 * rng.normal(size=n)
    lam0, lam2, M = 0.08, 0.05, 1.2
    c = X.T @ y
    # MIP optimum: beta_j = clip(c_j / (1 + 2 lam2), +-M) if its gain beats lam0
    bj = np.clip(c / (1 + 2 * lam2), -M, M)
    gain = c * bj - (0.5 + lam2) * bj * bj
    keep = gain > lam0
    opt = 0.5 * y @ y - np.sum(np.where(keep, gain - lam0, 0.0))
    res = bnb.solve(X, y, lam0, lam2, M, gap=1e-10)
    assert res.ub == pytest.approx(opt, rel=1e-10)
    assert set(np.nonzero(res.beta)[0]) == set(np.nonzero(keep)[0])
    # root relaxation: separable, min 1/2 (b - c_j)^2 + psi(b) solved coordinate-wise
    # by the prox at rho = 1; checked against the independent second solver
    fix = np.full(p, relax.FREE, dtype=np.int8)
    bstar = relax.prox(c, fix, lam0, lam2, M, 1.0)
    root = 0.5 * y @ y - 0.5 * c @ c + np.sum(0.5 * (bstar - c) ** 2 + relax.psi(bstar, fix, lam0, lam2, M))
    _, fb = pgd.solve_node(X, y, fix, lam0, lam2, M)
    assert root == pytest.approx(fb, rel=1e-10)


def test_lambda0_zero_relaxation_is_box_ridge():
    inst = _small(11)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2, 0.8)
    fix = np.full(inst.p, relax.FREE, dtype=np.int8)
    a = admm.solve_node(admm.AdmmData(inst.X, inst.y, 1.0), fix, 0.0, lam2, M, tol=1e-12, max_iter=100000)
    obj, _ = ub.support_objective(inst.X, inst.y, np.arange(inst.p), 0.0, lam2, M)
    assert a.dual == pytest.approx(obj, rel=1e-9)


def test_leaf_relaxation_equals_support_value():
    inst = _small(12)
    lam0, lam2, M = _params(inst)
    rng = np.random.default_rng(13)
    fix = (rng.random(inst.p) < 0.4).astype(np.int8)  # every coordinate fixed
    a = admm.solve_node(admm.AdmmData(inst.X, inst.y, 1.0), fix, lam0, lam2, M, tol=1e-12, max_iter=100000)
    S = np.nonzero(fix == relax.F1)[0]
    b = ub.box_ridge(inst.X, inst.y, S, lam2, M)
    leaf = ub.u_value(inst.X, inst.y, S, lam2, b) + lam0 * len(S)
    assert a.dual == pytest.approx(leaf, rel=1e-9)


def test_child_relaxations_dominate_parent():
    inst = _small(14)
    lam0, lam2, M = _params(inst, frac=0.02)
    fix = np.full(inst.p, relax.FREE, dtype=np.int8)
    _, parent = pgd.solve_node(inst.X, inst.y, fix, lam0, lam2, M)
    for j in (0, 3, 7):
        for v in (relax.F0, relax.F1):
            child = fix.copy()
            child[j] = v
            _, cv = pgd.solve_node(inst.X, inst.y, child, lam0, lam2, M)
            assert cv >= parent - 1e-10


def test_datagen_toeplitz_recipe():
    rng = np.random.default_rng(0)
    X = datagen.toeplitz_design(4000, 6, 0.6, rng)
    assert X.flags.f_contiguous
    np.testing.assert_array_equal(X, X.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(np.linalg.norm(X, axis=0), 1.0, atol=1e-6)
    C = np.corrcoef(X, rowvar=False)
    for lag in range(1, 4):
        assert np.mean(np.diag(C, lag)) == pytest.approx(0.6 ** lag, abs=0.04)
    assert list(datagen.true_support(50, 5)) == [0, 10, 20, 30, 40]


def test_datagen_noise_and_seeds():
    """y = X beta_true + eps with sigma^2 = Var(X beta_true) / SNR (sample variance of the
    noiseless response, Section 5.1), beta_true ones on the evenly spaced support, and the
    seed rule 1000 * config + instance."""
    inst = datagen.make_instance(4000, 20, 0.3, 4, 5.0, 77)
    mu = inst.X @ inst.beta_true
    assert list(np.nonzero(inst.beta_true)[0]) == [0, 5, 10, 15]
    assert np.all(inst.beta_true[inst.support_true] == 1.0)
    assert inst.sigma2 == pytest.approx(np.var(mu) / 5.0, rel=1e-12)
    assert np.var(inst.y - mu) / inst.sigma2 == pytest.approx(1.0, abs=0.1)
    assert abs(np.mean(inst.y - mu)) < 4 * np.sqrt(inst.sigma2 / 4000)
    again = datagen.make_instance(4000, 20, 0.3, 4, 5.0, 77)
    np.testing.assert_array_equal(inst.X, again.X)
    np.testing.assert_array_equal(inst.y, again.y)
    assert datagen.config_instance("c1", 3).seed == 1003
    assert datagen.config_instance("c2_small", 0).seed == 2000
