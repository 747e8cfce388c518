"""Plain FP64 CPU oracle for the l0-l2 branch-and-bound (arxiv 2602.04551).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the test suite, the package smoke check and the
CPU-baseline leg of the benchmark use it.  It shares no code with the CUDA
path; the two meet only through the seeded generators in ``datagen``.

Every function is written from the paper's definitions in float64 with plain
numpy, in the order the paper states them, with no blocking or fusion:

  relax   psi (Eq. psi), the box soft-threshold T (Eq. Tdef), the beta prox
          (Eq. minbetalower; Appendix A.1), z/s recovery (Appendix A.1),
          h and nu (Eqs. hdef, nudef), the relaxation primal (Eq. relaxnode2)
          and the dual bound of Proposition 1 (Eq. dual).
  admm    ADMM on Eq. ADMM1 with the direct D = (X^T X + rho I)^{-1}
          (Eqs. admm-update, b_update, v_i-update; warm start Section 3.1.3).
  pgd     an independent second relaxation solver: accelerated proximal
          gradient on Eq. relaxnode2 (used only to cross-check ADMM).
  ub      the box-constrained ridge on a support (Eq. upperboundbeta) solved
          exactly by an active-set method, and the literal accelerated
          projected gradient with backtracking (Eqs. fpg_extrapolate ..
          fpg_armijo).
  brute   enumeration of every support (p <= 16): the definition of the
          optimum of Eq. perspective.
  bnb     best-first branch-and-bound (Section 2.2.1, Algorithm 1).
  mp      the matching-pursuit root heuristic (Appendix A.2).

Pins (tests marked "not gpu"): brute force, closed forms against 1-D numeric
optimisation, weak and strong duality, agreement of two independent
relaxation solvers, the orthonormal-design special case, library
box-constrained least squares, and a branch-and-bound that takes incumbents at
leaves only.  A mutation test plants one mistake at a time in these functions
and checks that a pin fails.
"""
from . import relax, admm, pgd, ub, brute, bnb, mp  # noqa: F401
