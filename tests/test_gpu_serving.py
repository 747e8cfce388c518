"""Serving: independent solves of different (n, p, lambda) arriving over time are
admitted under an HBM budget and interleaved on the GPU; each result equals the
result of the same request solved alone (same support, objective within 1e-8
relative, both certified to the requested gap), and agrees with the FP64 oracle:
the p = 16 request is the brute-force optimum, every other one is within the
certified gap of the oracle's own branch-and-bound and is the exact objective of
the support it returns."""
import numpy as np
import pytest

import datagen
from oracle import bnb as obnb, brute, ub as oub

pytestmark = pytest.mark.gpu
bnb = pytest.importorskip("paper_2602_04551_b300")
from paper_2602_04551_b300.serve import Request, Server, LibraryBackend, latency_summary  # noqa: E402


def _requests(early_branch=0):
    specs = [(120, 16, 0.1, 3, 0.05), (200, 40, 0.3, 4, 0.03), (150, 60, 0.5, 5, 0.05),
             (300, 30, 0.7, 3, 0.1), (200, 50, 0.1, 5, 0.04), (100, 24, 0.3, 3, 0.02)]
    reqs = []
    for i, (n, p, rho, k, frac) in enumerate(specs):
        inst = datagen.make_instance(n, p, rho, k, 5.0, 5000 + i)
        lam2 = 0.01
        M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
        lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
        reqs.append(Request(rid=i, X=inst.X, y=inst.y, lambda0=lam0, lambda2=lam2, M=M, gap=1e-6,
                            # (the early-branch stop solves these small trees in a few
                            # milliseconds: closer arrivals keep the solves overlapping)
                            arrival=(0.002 if early_branch else 0.02) * i,
                            options=dict(batch_K=64, node_tol=1e-7, max_admm_iter=5000,
                                         time_limit_s=60.0, early_branch=early_branch)))
    return reqs


@pytest.mark.parametrize("early_branch", [0, 1])
def test_each_result_same_alone_and_in_the_mix(early_branch):
    """With the paper's node stop and with the early-branch one the serving loop uses."""
    reqs = _requests(early_branch)
    alone = {}
    for r in reqs:
        o = bnb.bnb_options_default(M=r.M, batch_K=64, node_tol=1e-7, max_admm_iter=5000,
                                    queue_capacity=1 << 16, time_limit_s=60.0,
                                    early_branch=early_branch)
        with bnb.bnb_create(r.X, r.y, r.lambda0, r.lambda2, o) as h:
            alone[r.rid] = bnb.bnb_solve(h, r.gap)
    # a budget that holds only part of the stream at once forces admission waits
    be = LibraryBackend()
    fps = [be.footprint(r) for r in reqs]
    srv = Server(backend=be, budget_bytes=int(2.5 * max(fps)), rounds_per_step=2)
    mixed = srv.run(reqs)
    assert srv.peak_active >= 2            # solves overlapped on the device
    for res in mixed:
        a = alone[res.rid]
        assert res.status in ("optimal", "gap")
        assert tuple(np.nonzero(res.beta)[0]) == tuple(np.nonzero(a["beta"])[0])
        assert res.ub == pytest.approx(a["ub"], rel=1e-8)
        assert res.lb <= res.ub * (1 + 1e-12)
    s = latency_summary(mixed)
    assert s["solves"] == len(reqs) and s["p99_s"] >= s["p50_s"] > 0
    # against the oracle
    by_id = {res.rid: res for res in mixed}
    for r in reqs:
        res = by_id[r.rid]
        S = np.nonzero(res.beta)[0]
        obj, _ = oub.support_objective(r.X, r.y, S, r.lambda0, r.lambda2, r.M)
        assert res.ub == pytest.approx(obj, rel=1e-9)          # the support's exact value
        if r.X.shape[1] <= 16:
            br = brute.solve(r.X, r.y, r.lambda0, r.lambda2, r.M)
            assert tuple(S) == br.support
            assert res.ub == pytest.approx(br.objective, rel=1e-8)
        else:
            ref = obnb.solve(r.X, r.y, r.lambda0, r.lambda2, r.M, gap=r.gap)
            assert ref.status in ("optimal", "gap")
            # both certified to the gap: each is within it of the optimum, hence of the other
            assert abs(res.ub - ref.ub) <= 2 * r.gap * abs(ref.ub)
            assert res.lb <= ref.ub * (1 + 1e-12) and ref.lb <= res.ub * (1 + 1e-12)


def test_autotune_search_trial_times_the_tree_search():
    """The autotuner's search measurement on a real solve: a primed solve of the c2_small
    instance, timed rounds, a positive node rate; and autotune with search_top picks one of
    the searched candidates."""
    from paper_2602_04551_b300 import autotune
    inst = datagen.config_instance("c2_small", 0)
    lam2 = datagen.CONFIGS["c2_small"]["lam2"]
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.02 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    opts = dict(rho=0.3, relax_alpha=1.6, batch_K=64, check_every=10, precision=3)
    st = autotune.search_trial(inst.X, inst.y, lam0, lam2, M, opts, rounds=50, warm_rounds=20)
    if st is not None:                             # None only when the solve ends while priming
        assert st["search_nodes"] > 0 and st["search_nodes_per_s"] > 0
        assert st["search_rounds"] == 50 and st["prime_rounds"] <= 420
    grid = {"rho": [0.2, 0.3], "relax_alpha": [1.6], "batch_K": [64], "check_every": [10],
            "precision": [3]}
    best, entry = autotune.autotune(inst.X, inst.y, lam0, lam2, M, grid=grid, use_cache=False,
                                    tune_crossover=False, search_top=2)
    searched = [t for t in entry["trials"] if "search_nodes_per_s" in t]
    if searched:
        top = max(searched, key=lambda t: t["search_nodes_per_s"])
        assert best["rho"] == top["rho"]
