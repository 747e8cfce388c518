"""Best-first branch-and-bound for Eq. perspective, FP64 (test infrastructure only).

Follows Section 2.2.1 and Algorithm 1 (Section 2.4):
  * a node is (F0, F1, LB of its parent); the root is (empty, empty, -inf);
  * Algorithm 1 batch: select the min(K, |N|) open nodes of smallest LB;
  * each node's relaxation is solved by ADMM (oracle.admm) warm-started from
    its parent (Section 3.1.3) and bounded by the dual of Proposition 1 at
    r = y - X b;  LB_u = max(LB_parent, D(r)) (both are valid bounds);
  * upper bound (Section 3.3): round z (Appendix A.1 recovery) to the support
    S = F1 + {free i : z_i >= 1/2}, solve Eq. upperboundbeta exactly;  with
    round_incumbent=False the incumbent comes from leaves only (the textbook
    rule, Section 2.2.1), so the answer rests on the search alone;
  * prune when LB_u >= UB (1 - gap) (reading of Section 2.2.1 that makes the
    final (UB - LB)/UB <= gap);
  * branch on the free index with the most fractional z_i, ties to the lowest
    index (reading: "Select j" in Algorithm 1 is unspecified); if every free
    z_i is integral, branch on the free index of largest |X_i^T r|;  a node
    with no free index is a leaf whose value is its support's box ridge plus
    lambda0 |F1|, so it is closed after its upper bound is taken;
  * global LB = min LB over the open nodes, and never above UB (the
    incumbent is itself a feasible point, so once every open node's bound
    exceeds it the optimum is the incumbent); stop when N is empty or
    (UB - LB)/UB <= gap.
"""
from __future__ import annotations

import dataclasses
import heapq
import itertools
import numpy as np

from . import relax, admm, ub


@dataclasses.dataclass
class BnbResult:
    beta: np.ndarray
    ub: float
    lb: float
    nodes: int
    status: str
    max_depth: int
    history: list      # (nodes, UB, LB) after each batch
    node_log: list     # (fix, LB_parent, dual bound D(r)) per solved node


def branch_index(z, fix, g):
    free = np.nonzero(fix == relax.FREE)[0]
    if len(free) == 0:
        return -1
    frac = np.minimum(z[free], 1.0 - z[free])
    j = int(np.argmax(frac))  # argmax returns the lowest index on ties
    if frac[j] > 0.0:
        return int(free[j])
    return int(free[int(np.argmax(np.abs(g[free])))])


def solve(X, y, lam0, lam2, M, gap=1e-6, K=1, rho=1.0, node_tol=1e-10,
          max_admm_iter=20000, max_nodes=100000, warm_start=True,
          round_incumbent=True) -> BnbResult:
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, p = X.shape
    data = admm.AdmmData(X, y, rho)
    counter = itertools.count()
    root = (-np.inf, next(counter), np.full(p, relax.FREE, dtype=np.int8), None, None, 0)
    heap = [root]
    UB = np.inf
    best = np.zeros(p)
    LB = -np.inf
    nodes = 0
    max_depth = 0
    history = []
    node_log = []
    status = "optimal"
    while heap and not (UB < np.inf and (UB - LB) / UB <= gap):
        if nodes >= max_nodes:
            status = "node_limit"
            break
        batch = [heapq.heappop(heap) for _ in range(min(K, len(heap)))]
        solved = []
        for (lb_parent, _, fix, wb, wv, depth) in batch:
            res = admm.solve_node(data, fix, lam0, lam2, M, beta0=wb, v0=wv,
                                  tol=node_tol, max_iter=max_admm_iter)
            nodes += 1
            max_depth = max(max_depth, depth)
            solved.append((lb_parent, fix, depth, res))
        for lb_parent, fix, depth, res in solved:
            lb_u = max(lb_parent, res.dual)
            node_log.append((fix, lb_parent, res.dual))
            if lb_u >= UB * (1.0 - gap):
                continue
            z = relax.z_of_beta(res.beta, fix, lam0, lam2, M)
            if round_incumbent or not np.any(fix == relax.FREE):
                S = np.nonzero((fix == relax.F1) | ((fix == relax.FREE) & (z >= 0.5)))[0]
                obj, beta_s = ub.support_objective(X, y, S, lam0, lam2, M)
                if obj < UB:
                    UB, best = obj, beta_s
            if lb_u >= UB * (1.0 - gap):
                continue
            g = X.T @ res.r
            j = branch_index(z, fix, g)
            if j < 0:
                continue  # leaf: closed by its own upper bound
            for val in (relax.F0, relax.F1):
                child = fix.copy()
                child[j] = val
                wb = wv = None
                if warm_start:
                    wb = res.beta.copy()
                    wv = res.v.copy()
                    if val == relax.F0:
                        wb[j] = 0.0
                heapq.heappush(heap, (lb_u, next(counter), child, wb, wv, depth + 1))
        LB = min(min((e[0] for e in heap), default=UB), UB)
        history.append((nodes, UB, LB))
    if not heap:
        LB = UB
    return BnbResult(beta=best, ub=UB, lb=LB, nodes=nodes, status=status,
                     max_depth=max_depth, history=history, node_log=node_log)
