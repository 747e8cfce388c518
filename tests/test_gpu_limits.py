"""Solve-ending limits and the bounded device waits, on the GPU.

A solve that stops early (wall-clock limit, node limit, full node pool, a leaf whose
support is too large to evaluate) reports its own status and a lower bound that is
still valid: LB <= the brute-force optimum at p = 16.  The tensor-core kernels' bounded
mbarrier wait gives up, sets its error word and returns when nothing arrives (the
diagnostics library runs that wait alone with short limits; no TMA copy or MMA is in
flight), and the context stays usable afterwards.
"""
import numpy as np
import pytest

import datagen
from oracle import brute

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
bnb = pytest.importorskip("paper_2602_04551_b300")


def _p16(inst_id=1, frac=0.03):
    c = datagen.CONFIGS["c1_p16"]
    inst = datagen.config_instance("c1_p16", inst_id)
    lam2 = c["lam2"]
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    return inst, lam0, lam2, M


def _solve(inst, lam0, lam2, M, gap=1e-9, **kw):
    kw.setdefault("queue_capacity", 1 << 12)
    kw.setdefault("batch_K", 8)
    o = bnb.bnb_options_default(M=M, node_tol=1e-7, max_admm_iter=5000, **kw)
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
        return bnb.bnb_solve(h, gap), bnb.bnb_get_stats(h)


def _valid(res, br):
    assert res["lb"] <= br.objective * (1 + 1e-9), (res["lb"], br.objective)
    assert res["ub"] >= br.objective * (1 - 1e-12)
    assert res["lb"] <= res["ub"] * (1 + 1e-12)


def test_time_limit_status_keeps_a_valid_bound():
    inst, lam0, lam2, M = _p16()
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res, _ = _solve(inst, lam0, lam2, M, time_limit_s=1e-6, root_heuristic=0)
    assert res["status"] == "time_limit"
    _valid(res, br)


def test_node_limit_status_keeps_a_valid_bound():
    inst, lam0, lam2, M = _p16()
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res, st = _solve(inst, lam0, lam2, M, batch_K=1, max_nodes=3, root_heuristic=0)
    assert res["status"] == "node_limit"
    assert 3 <= res["nodes"] <= 4
    _valid(res, br)


def test_full_pool_status_keeps_a_valid_bound():
    """The smallest pool (4 K + 8 = 12 entries) with one slot: a solve stops once fewer
    than 2 K + 2 = 4 entries are free, i.e. beyond 8 open nodes.  An instance whose search
    needs at least 12 open nodes (a solve with a large pool shows how many) must end on
    the full pool."""
    for frac in (0.01, 0.005, 0.003, 0.002):
        inst, lam0, lam2, M = _p16(1, frac)
        br = brute.solve(inst.X, inst.y, lam0, lam2, M)
        big, st = _solve(inst, lam0, lam2, M, batch_K=1, root_heuristic=0)
        assert tuple(np.nonzero(big["beta"])[0]) == br.support
        if st["pool_peak"] >= 12:
            break
    assert st["pool_peak"] >= 12, st["pool_peak"]
    res, _ = _solve(inst, lam0, lam2, M, batch_K=1, queue_capacity=12, root_heuristic=0)
    assert res["status"] == "queue_full"
    _valid(res, br)


def test_oversized_leaf_support_status_keeps_a_valid_bound():
    """support_max = 1 with every feature fixable (max_depth >= p): a leaf with two or more
    features in F1 cannot have its upper bound taken, so the solve stops with its own
    status and keeps that leaf's bound in LB instead of dropping its objective."""
    inst, lam0, lam2, M = _p16(1, 0.002)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    assert len(br.support) >= 2
    res, _ = _solve(inst, lam0, lam2, M, batch_K=4, support_max=1, max_depth=16,
                    root_heuristic=0)
    assert res["status"] == "support_limit"
    _valid(res, br)


@pytest.mark.parametrize("polls,seconds", [(1 << 30, 0.02), (4096, 1.0)])
def test_bounded_mbarrier_wait_expires_sets_error_and_returns(polls, seconds):
    """First case: the time limit ends the wait (about 20 ms); second: the poll limit."""
    err, waited = bnb.bnb_diag_wait_expiry(polls, seconds)
    assert err == 1, err                      # every wait expired, none reported success
    if polls == 1 << 30:
        assert 0.015 <= waited <= 0.5, waited
    else:
        assert waited < 0.5, waited
    # the context is still usable
    x = torch.arange(1000, device="cuda", dtype=torch.float64)
    assert float(x.sum().item()) == 499500.0


def test_poll_before_the_first_round_does_not_end_the_solve():
    """bnb_solve_poll right after bnb_solve_start (no round launched yet) reports the root
    alone and an open solve -- it must not read a stale status as a closed tree -- and the
    solve then reaches the brute-force optimum as usual."""
    inst, lam0, lam2, M = _p16(1, 0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    o = bnb.bnb_options_default(M=M, node_tol=1e-7, max_admm_iter=5000, batch_K=8,
                                queue_capacity=1 << 12)
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
        for _ in range(2):                    # a second solve on the same handle as well
            bnb.bnb_solve_start(h, 1e-9)
            pr = bnb.bnb_solve_poll(h)
            assert not pr["done"] and pr["nodes"] == 0 and pr["open_nodes"] == 1
            assert pr["lb"] == -np.inf
            while not pr["done"]:
                bnb.bnb_solve_launch(h, 1)
                pr = bnb.bnb_solve_poll(h)
            res = bnb.bnb_solve_finish(h)
            assert tuple(np.nonzero(res["beta"])[0]) == br.support
            assert res["ub"] == pytest.approx(br.objective, rel=1e-8)
