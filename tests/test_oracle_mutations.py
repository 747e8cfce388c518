"""The oracle's pins are sensitive: each planted mistake fails the pin meant to catch it.

A mutant is one oracle function recompiled from its own source with a single
textual edit (a dropped term, a flipped sign, a wrong constant or index, a
skipped case), substituted into the oracle for the duration of one test with
monkeypatch, on the CPU.  The pin named beside it must then fail.  The
unmutated pins pass in their own modules, so a mutant that slipped through
would mean a part of the oracle that no pin fixes.

The edits model the mistakes a reader of the paper could plausibly make:
the batched prox listing without the ridge branch (Section 3.1), the prox
case order in the regime sqrt(lambda0/lambda2) > M (Appendix A.1 case 4),
the conjugate nu without its clipping at zero (Eq. nudef), the dual of
Proposition 1 with a sign or a term wrong, the ADMM updates of Eq. admm-update
with the scaled dual misplaced, the upper-bound solver of Eq. upperboundbeta
without its ridge term or projection, the matching-pursuit deltas of
Appendix A.2 with a wrong coefficient, and the branch-and-bound's global
bound taken over the wrong extreme (Section 2.2.1).
"""
import importlib
import inspect
import sys
import textwrap

import pytest

from oracle import admm, bnb, brute, mp, pgd, relax, ub

CF = "test_oracle_closed_forms"
SV = "test_oracle_solvers"
MP = "test_oracle_mp"

# (id, owner, function, old text, new text, occurrences, pin module, pin, pin args)
MUTANTS = [
    ("T-sign-dropped", relax, "T", "(at - a) * np.sign(t)", "(at - a)", 1,
     CF, "test_T_definition_values", ()),
    ("T-box-cap-dropped", relax, "T", "m * np.sign(t)))", "(at - a) * np.sign(t)))", 1,
     CF, "test_T_definition_values", ()),
    ("psi-ridge-without-lambda0", relax, "psi", "ridge = lam0 + lam2 * beta * beta",
     "ridge = lam2 * beta * beta", 1, CF, "test_psi_is_min_over_z_s", (0.05, 0.01, 3.0)),
    ("psi-perspective-slope-halved", relax, "psi", "2.0 * np.sqrt(lam0 * lam2) * ab",
     "np.sqrt(lam0 * lam2) * ab", 1, CF, "test_psi_is_min_over_z_s", (0.05, 0.01, 3.0)),
    ("psi-linear-slope-without-lambda2-M", relax, "psi", "(lam0 / M + lam2 * M) * ab",
     "(lam0 / M) * ab", 1, CF, "test_psi_is_min_over_z_s", (0.05, 0.01, 1.5)),
    ("prox-ridge-branch-dropped", relax, "prox",
     "free = np.where(np.abs(bt) >= tau, ridge, T(bt, a, M))", "free = T(bt, a, M)", 1,
     CF, "test_prox_is_numeric_argmin", (0.05, 0.01, 3.0, 1.0)),
    ("prox-regime-test-skipped", relax, "prox", "if _free_regime_linear(lam0, lam2, M):",
     "if False:", 1, CF, "test_prox_is_numeric_argmin", (0.05, 0.01, 1.5, 1.0)),
    ("prox-ridge-shrink-lambda2", relax, "prox", "rho / (rho + 2.0 * lam2) * bt",
     "rho / (rho + lam2) * bt", 1, CF, "test_prox_is_numeric_argmin", (0.3, 0.5, 1.0, 1.0)),
    ("prox-threshold-times-rho", relax, "prox", "a = 2.0 * np.sqrt(lam0 * lam2) / rho",
     "a = 2.0 * np.sqrt(lam0 * lam2) * rho", 1, CF, "test_prox_is_numeric_argmin",
     (0.05, 0.01, 3.0, 4.0)),
    ("z-box-bound-dropped", relax, "z_of_beta", "np.maximum(ab / M, np.sqrt(lam2 / lam0) * ab)",
     "np.sqrt(lam2 / lam0) * ab", 1, CF, "test_z_recovery_is_argmin", (0.05, 0.01, 1.5)),
    ("z-square-root-dropped", relax, "z_of_beta", "np.sqrt(lam2 / lam0) * ab", "(lam2 / lam0) * ab", 1,
     CF, "test_z_recovery_is_argmin", (0.05, 0.01, 3.0)),
    ("h-quadratic-piece-halved", relax, "h", "x * x / (4.0 * lam2)", "x * x / (2.0 * lam2)", 1,
     CF, "test_h_continuous_at_kink", ()),
    ("h-linear-piece-sign", relax, "h", "M * x - lam0 - lam2 * M * M", "M * x - lam0 + lam2 * M * M", 1,
     CF, "test_h_continuous_at_kink", ()),
    ("nu-clip-at-zero-dropped", relax, "nu", "free = np.maximum(hx, 0.0)", "free = hx", 1,
     CF, "test_nu_is_conjugate_of_psi", (0.05, 0.01, 3.0)),
    ("nu-F1-treated-as-free", relax, "nu", "out = np.where(fix == F1, hx, free)", "out = free", 1,
     CF, "test_nu_is_conjugate_of_psi", (0.05, 0.01, 3.0)),
    ("nu-linear-regime-constant-dropped", relax, "nu",
     "free = np.maximum(M * x - lam0 - lam2 * M * M, 0.0)", "free = np.maximum(M * x - lam0, 0.0)", 1,
     CF, "test_nu_is_conjugate_of_psi", (0.05, 0.01, 1.5)),
    ("dual-sign-of-yr", relax, "dual_value", "+ float(y @ r)", "- float(y @ r)", 1,
     SV, "test_admm_matches_second_solver_and_strong_duality", (1.5, 1.0, 1)),
    ("dual-sign-of-quadratic", relax, "dual_value", "-0.5 * float(r @ r)", "0.5 * float(r @ r)", 1,
     SV, "test_weak_duality_random_r", (1.5,)),
    ("dual-abs-dropped", relax, "dual_value", "nu(np.abs(g),", "nu(g,", 1,
     SV, "test_admm_matches_second_solver_and_strong_duality", (0.3, 0.35, -1)),
    ("primal-psi-dropped", relax, "primal_value",
     " + float(np.sum(psi(beta, fix, lam0, lam2, M)))", "", 1,
     SV, "test_admm_matches_second_solver_and_strong_duality", (1.5, 1.0, 1)),
    ("admm-dual-update-sign", admm, "admm_iteration", "v + rho * (bh - beta_new)",
     "v - rho * (bh - beta_new)", 1, SV, "test_admm_matches_second_solver_and_strong_duality",
     (1.5, 1.0, 1)),
    ("admm-b-update-without-v", admm, "admm_iteration", "data.c + rho * beta - v",
     "data.c + rho * beta", 1, SV, "test_admm_matches_second_solver_and_strong_duality",
     (1.5, 1.0, 1)),
    ("admm-scaled-dual-unscaled", admm, "admm_iteration", "bt = bh + v / rho", "bt = bh + v", 1,
     SV, "test_admm_matches_second_solver_and_strong_duality", (1.5, 0.35, 1)),
    ("admm-D-without-rho", admm.AdmmData, "__init__", "self.X.T @ self.X + self.rho * np.eye(p)",
     "self.X.T @ self.X + np.eye(p)", 1, SV, "test_admm_matches_second_solver_and_strong_duality",
     (1.5, 0.35, 1)),
    ("admm-over-relaxation-weights-swapped", admm, "admm_iteration",
     "alpha * b + (1.0 - alpha) * beta", "alpha * beta + (1.0 - alpha) * b", 1,
     SV, "test_over_relaxed_admm_reaches_the_same_optimum", (1.5, 1)),
    ("pgd-prox-at-unit-step", pgd, "solve_node", "relax.prox(yk - g / L, fix, lam0, lam2, M, L)",
     "relax.prox(yk - g / L, fix, lam0, lam2, M, 1.0)", 1,
     SV, "test_admm_matches_second_solver_and_strong_duality", (1.5, 1.0, 1)),
    ("ub-gram-ridge-halved", ub, "_gram", "2.0 * lam2 * np.eye(len(S))", "lam2 * np.eye(len(S))", 1,
     SV, "test_box_ridge_matches_library", (10.0,)),
    ("ub-active-set-lower-bound-sign", ub, "box_ridge", "beta[block] = M * W[block]",
     "beta[block] = M", 1, SV, "test_box_ridge_matches_library", (0.15,)),
    ("ub-fista-gradient-without-ridge", ub, "fista_backtracking", " + 2.0 * lam2 * ext", "", 1,
     SV, "test_box_ridge_matches_library", (10.0,)),
    ("ub-fista-projection-dropped", ub, "fista_backtracking", "np.clip(ext - alpha * g, -M, M)",
     "(ext - alpha * g)", 1, SV, "test_box_ridge_matches_library", (0.4,)),
    ("brute-lambda0-dropped", brute, "solve", "+ 0.5 * quad + lam0 * s", "+ 0.5 * quad", 1,
     SV, "test_brute_force_two_features_by_hand", (3.0, 100.0)),
    ("brute-linear-term-sign", brute, "solve", '0.5 * yy - np.einsum("ki,ki->k", rhs, sol)',
     '0.5 * yy + np.einsum("ki,ki->k", rhs, sol)', 1, SV, "test_brute_force_two_features_by_hand", (3.0, 100.0)),
    ("brute-ridge-halved", brute, "solve", "+ 2.0 * lam2 * np.eye(s)[None]", "+ lam2 * np.eye(s)[None]", 1,
     SV, "test_brute_force_two_features_by_hand", (3.0, 100.0)),
    ("bnb-F0-child-only", bnb, "solve", "for val in (relax.F0, relax.F1):",
     "for val in (relax.F0,):", 1, SV, "test_bnb_leaf_incumbents_match_brute_force", (0, 0.02)),
    ("bnb-F1-child-only", bnb, "solve", "for val in (relax.F0, relax.F1):",
     "for val in (relax.F1,):", 1, SV, "test_bnb_leaf_incumbents_match_brute_force", (0, 0.02)),
    ("bnb-bound-from-primal", bnb, "solve", "lb_u = max(lb_parent, res.dual)",
     "lb_u = max(lb_parent, res.primal)", 1, SV, "test_bnb_leaf_incumbents_match_brute_force", (1, 0.2)),
    ("bnb-global-bound-max", bnb, "solve", "LB = min(min((e[0] for e in heap), default=UB), UB)",
     "LB = min(max((e[0] for e in heap), default=UB), UB)", 1, SV, "test_bnb_leaf_incumbents_match_brute_force",
     (2, 0.02)),
    ("bnb-worst-first", bnb, "solve", "heapq.heappush(heap, (lb_u,", "heapq.heappush(heap, (-lb_u,", 1,
     SV, "test_bnb_leaf_incumbents_match_brute_force", (0, 0.2)),
    ("bnb-child-bound-dropped", bnb, "solve", "heapq.heappush(heap, (lb_u,", "heapq.heappush(heap, (-np.inf,", 1,
     SV, "test_bnb_leaf_incumbents_match_brute_force", (0, 0.2)),
    ("bnb-prune-inverted", bnb, "solve", "if lb_u >= UB * (1.0 - gap):", "if lb_u <= UB * (1.0 - gap):", 2,
     SV, "test_bnb_matches_brute_force_p16", (0.05,)),
    ("brute-box-resolve-skipped", brute, "solve", "bad = np.max(np.abs(sol), axis=1) > M",
     "bad = np.zeros(len(sol), dtype=bool)", 1, SV, "test_brute_force_two_features_by_hand", (0.05, 0.5)),
    ("psi-box-not-enforced", relax, "psi", "out = np.where(ab > M, np.inf, out)", "out = out", 1,
     CF, "test_psi_is_min_over_z_s", (0.05, 0.01, 3.0)),
    ("prox-F0-not-zeroed", relax, "prox", "out = np.where(fix == F0, 0.0, out)", "out = out", 1,
     CF, "test_prox_is_numeric_argmin", (0.05, 0.01, 3.0, 1.0)),
    ("nu-F0-not-zeroed", relax, "nu", "out = np.where(fix == F0, 0.0, out)", "out = out", 1,
     CF, "test_nu_is_conjugate_of_psi", (0.05, 0.01, 3.0)),
    ("z-F1-not-one", relax, "z_of_beta", "z = np.where(fix == F1, 1.0, zf)", "z = zf", 1,
     CF, "test_z_recovery_is_argmin", (0.05, 0.01, 3.0)),
    ("branch-least-fractional", bnb, "branch_index", "j = int(np.argmax(frac))", "j = int(np.argmin(frac))", 1,
     SV, "test_branch_index_hand_cases", ()),
    ("branch-fixed-indices-eligible", bnb, "branch_index", "free = np.nonzero(fix == relax.FREE)[0]",
     "free = np.arange(len(fix))", 1, SV, "test_branch_index_hand_cases", ()),
    ("branch-integral-fallback-lowest", bnb, "branch_index", "return int(free[int(np.argmax(np.abs(g[free])))])",
     "return int(free[0])", 1, SV, "test_branch_index_hand_cases", ()),
    ("branch-fallback-signed-g", bnb, "branch_index", "np.argmax(np.abs(g[free]))", "np.argmax(g[free])", 1,
     SV, "test_branch_index_hand_cases", ()),
    ("mp-selected-not-masked", mp, "matching_pursuit", "d = np.where(in_s, np.inf, d)", "d = d", 1,
     MP, "test_matching_pursuit_orthonormal_design", ()),
    ("mp-forward-argmax", mp, "matching_pursuit", "j = int(np.argmin(d))", "j = int(np.argmax(d))", 1,
     MP, "test_matching_pursuit_orthonormal_design", ()),
    ("mp-residual-not-updated", mp, "matching_pursuit", "r = r - X[:, j] * b[j]", "r = r", 1,
     MP, "test_matching_pursuit_ends_at_a_single_move_optimum", ((80, 30, 0.3, 4, 5.0, 5, 0.05),)),
    ("mp-backward-never-taken", mp, "matching_pursuit", "if db[j] < 0.0:", "if False:", 1,
     MP, "test_matching_pursuit_ends_at_a_single_move_optimum", ((60, 25, 0.7, 5, 3.0, 934, 0.1),)),
    ("mp-forward-curvature-doubled", mp, "forward_deltas", "+ 0.5 * D * b * b + lam0", "+ D * b * b + lam0", 1,
     MP, "test_forward_delta_is_objective_change", (1.5,)),
    ("mp-forward-step-unclipped", mp, "forward_deltas", "np.clip(c / D, -M, M)", "(c / D)", 1,
     MP, "test_forward_delta_is_objective_change", (0.2,)),
    ("mp-backward-ridge-sign", mp, "backward_deltas", "(0.5 * col_sq - lam2) * beta * beta",
     "(0.5 * col_sq + lam2) * beta * beta", 1, MP, "test_backward_delta_is_objective_change", ()),
]


def _plant(monkeypatch, owner, name, old, new, count):
    """Recompile owner.name from its source with `old` replaced by `new` (a planted mistake)."""
    fn = getattr(owner, name)
    src = textwrap.dedent(inspect.getsource(fn))
    assert src.count(old) == count, f"{name}: expected {count} occurrence(s) of {old!r}"
    module = sys.modules[fn.__module__]
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), module.__file__, "exec"), ns)
    monkeypatch.setattr(owner, name, ns[name])


@pytest.mark.filterwarnings("ignore::RuntimeWarning")     # a diverging mutant overflows
@pytest.mark.parametrize("mutant", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_its_pin(monkeypatch, mutant):
    _, owner, name, old, new, count, pin_mod, pin_name, args = mutant
    pin = getattr(importlib.import_module(pin_mod), pin_name)
    _plant(monkeypatch, owner, name, old, new, count)
    with pytest.raises(AssertionError):
        pin(*args)


def test_unmutated_recompile_passes(monkeypatch):
    """The recompilation itself changes nothing: an identity edit keeps every pin green."""
    _plant(monkeypatch, relax, "prox", "return out", "return out", 1)
    getattr(importlib.import_module(CF), "test_prox_is_numeric_argmin")(0.05, 0.01, 3.0, 1.0)
    _plant(monkeypatch, admm, "admm_iteration", "return b, beta_new, v_new", "return b, beta_new, v_new", 1)
    getattr(importlib.import_module(SV), "test_admm_matches_second_solver_and_strong_duality")(1.5, 0.35, 1)
