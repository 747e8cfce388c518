"""Selection and cache logic of the autotuner with fake trials (no GPU): configurations
whose mean certified bound is weaker than the best by more than the tolerance are not
chosen for speed, the fastest of the rest on the batch measurement is unless the search
measurement of the top candidates ranks them otherwise, the narrow-form crossover is the
largest width at which it wins, and results are cached per (n, p) bucket and grid."""
import numpy as np

from paper_2602_04551_b300 import autotune


def _fake_trial(X, y, lam0, lam2, M, opts, device=0, seed=0, nodes=None):
    rho, prec = opts["rho"], opts["precision"]
    if nodes is not None:                          # crossover trials: narrow wins below 16
        narrow = opts.get("mv_crossover", 0) > 0
        ms = (1.0 if nodes <= 8 else 3.0) if narrow else 2.0
        return {"nodes_per_s": nodes / ms, "ms": ms, "mean_iters": 10.0, "lb_mean": 1.0}
    speed = {0.1: 100.0, 0.3: 300.0, 1.0: 200.0}[rho] * (5.0 if prec == 2 else 1.0)
    lb = 0.9 if prec == 2 else 1.0                 # the fast mode has weak bounds
    return {"nodes_per_s": speed, "ms": 1.0, "mean_iters": 50.0, "lb_mean": lb}


def _no_search(*a, **k):
    return None                                    # every solve ends before it is timed


def test_fastest_valid_configuration_and_crossover(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "trial", _fake_trial)
    monkeypatch.setattr(autotune, "search_trial", _no_search)
    monkeypatch.setenv("BNB_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    X = np.zeros((100, 500))
    grid = {"rho": [0.1, 0.3, 1.0], "precision": [3, 2], "batch_K": [64], "relax_alpha": [1.0]}
    best, entry = autotune.autotune(X, np.zeros(100), 0.1, 0.01, 1.0, grid=grid)
    assert best["rho"] == 0.3 and best["precision"] == 3      # BF16 is faster but weaker
    assert best["mv_crossover"] == 8
    assert [r["width"] for r in entry["crossover"]] == [4, 8, 16, 32]
    assert len(entry["trials"]) == 6


def test_cache_hit_and_key(monkeypatch, tmp_path):
    calls = []

    def counting(*a, **k):
        calls.append(1)
        return _fake_trial(*a, **k)

    monkeypatch.setattr(autotune, "trial", counting)
    monkeypatch.setattr(autotune, "search_trial", _no_search)
    monkeypatch.setenv("BNB_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    grid = {"rho": [0.3], "precision": [3], "batch_K": [64], "relax_alpha": [1.0]}
    X = np.zeros((100, 500))
    b1, _ = autotune.autotune(X, np.zeros(100), 0.1, 0.01, 1.0, grid=grid)
    n1 = len(calls)
    b2, _ = autotune.autotune(np.zeros((105, 520)), np.zeros(105), 0.1, 0.01, 1.0, grid=grid)
    assert b1 == b2 and len(calls) == n1           # same half-octave bucket: cached
    autotune.autotune(np.zeros((400, 500)), np.zeros(400), 0.1, 0.01, 1.0, grid=grid)
    assert len(calls) > n1                         # another bucket: measured
    assert autotune._key(100, 500, grid) != autotune._key(100, 500, dict(grid, rho=[0.1]))


def test_no_crossover_when_narrow_never_wins(monkeypatch, tmp_path):
    def slow_narrow(X, y, lam0, lam2, M, opts, device=0, seed=0, nodes=None):
        r = _fake_trial(X, y, lam0, lam2, M, opts, device, seed, nodes)
        if nodes is not None and opts.get("mv_crossover", 0) > 0:
            r["ms"] = 9.0
        return r

    monkeypatch.setattr(autotune, "trial", slow_narrow)
    monkeypatch.setattr(autotune, "search_trial", _no_search)
    monkeypatch.setenv("BNB_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    grid = {"rho": [0.3], "precision": [3], "batch_K": [64], "relax_alpha": [1.0]}
    best, _ = autotune.autotune(np.zeros((100, 500)), np.zeros(100), 0.1, 0.01, 1.0, grid=grid,
                                use_cache=False)
    assert best["mv_crossover"] == 0


def test_search_measurement_decides_among_top_candidates(monkeypatch, tmp_path):
    """Batch ranking 0.3 > 1.0 > 0.1 (> the weak BF16 modes, filtered); the search
    measurement of the top two prefers 1.0; 0.1 is outside the top two and is not searched
    even though its search score would be the highest."""
    searched = []

    def fake_search(X, y, lam0, lam2, M, opts, device=0, **k):
        searched.append(opts["rho"])
        return {"search_nodes_per_s": {0.1: 900.0, 0.3: 400.0, 1.0: 500.0}[opts["rho"]]}

    monkeypatch.setattr(autotune, "trial", _fake_trial)
    monkeypatch.setattr(autotune, "search_trial", fake_search)
    grid = {"rho": [0.1, 0.3, 1.0], "precision": [3, 2], "batch_K": [64], "relax_alpha": [1.0]}
    best, entry = autotune.autotune(np.zeros((100, 500)), np.zeros(100), 0.1, 0.01, 1.0,
                                    grid=grid, use_cache=False, tune_crossover=False,
                                    search_top=2)
    assert searched == [0.3, 1.0]
    assert best["rho"] == 1.0 and best["precision"] == 3
    assert entry["score"]["search_nodes_per_s"] == 500.0
    rows = {(t["rho"], t["precision"]): t for t in entry["trials"]}
    assert "search_nodes_per_s" in rows[(0.3, 3)] and "search_nodes_per_s" not in rows[(0.1, 3)]


def test_search_top_zero_keeps_batch_ranking(monkeypatch, tmp_path):
    def fail(*a, **k):
        raise AssertionError("search_trial called with search_top=0")

    monkeypatch.setattr(autotune, "trial", _fake_trial)
    monkeypatch.setattr(autotune, "search_trial", fail)
    grid = {"rho": [0.1, 0.3, 1.0], "precision": [3], "batch_K": [64], "relax_alpha": [1.0]}
    best, _ = autotune.autotune(np.zeros((100, 500)), np.zeros(100), 0.1, 0.01, 1.0, grid=grid,
                                use_cache=False, tune_crossover=False, search_top=0)
    assert best["rho"] == 0.3


def test_check_every_chosen_by_search(monkeypatch):
    """With check_every_values, the chosen configuration is searched again at each other
    interval and the fastest interval is kept; a solve that ends while priming (None) is
    skipped."""
    calls = []

    def fake_search(X, y, lam0, lam2, M, opts, device=0, **k):
        calls.append((opts["rho"], opts["check_every"]))
        if opts["check_every"] == 40:
            return None
        return {"search_nodes_per_s": {10: 100.0, 20: 130.0, 30: 120.0}[opts["check_every"]]
                * (2.0 if opts["rho"] == 0.3 else 1.0)}

    monkeypatch.setattr(autotune, "trial", _fake_trial)
    monkeypatch.setattr(autotune, "search_trial", fake_search)
    grid = {"rho": [0.1, 0.3], "precision": [3], "batch_K": [64], "relax_alpha": [1.0],
            "check_every": [10]}
    best, entry = autotune.autotune(np.zeros((100, 500)), np.zeros(100), 0.1, 0.01, 1.0,
                                    grid=grid, use_cache=False, tune_crossover=False,
                                    search_top=2, check_every_values=(10, 20, 30, 40))
    assert best["rho"] == 0.3 and best["check_every"] == 20
    assert calls[2:] == [(0.3, 20), (0.3, 30), (0.3, 40)]
    assert [r["check_every"] for r in entry["check_every"]] == [10, 20, 30]
    assert entry["score"]["search_nodes_per_s"] == 260.0


def test_steady_state_needs_a_certified_batch_and_a_batch_of_waiting_nodes():
    """autotune.steady, the priming rule of the bench and of the tree-search trial: a batch's
    worth of certified nodes and K open nodes besides the active slots; the active-slot
    count alone (read after a round's stop test has retired its converged slots) does not
    decide it."""
    K = 512
    pr = lambda nodes, open_nodes, active: {"nodes": nodes, "open_nodes": open_nodes,
                                             "active_slots": active}
    assert autotune.steady(pr(600, 1100, 437), K)          # slots refill from 663 waiting
    assert not autotune.steady(pr(400, 5000, 512), K)      # too few nodes certified yet
    assert not autotune.steady(pr(600, 900, 500), K)       # only 400 waiting: a refill runs short
    assert autotune.steady(pr(10**6, 2 * 10**6, 0), K)     # every slot retired at once (C3)
