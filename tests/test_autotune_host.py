"""Selection and cache logic of the autotuner with fake trials (no GPU): configurations
whose mean certified bound is weaker than the best by more than the tolerance are not
chosen for speed, the fastest of the rest is, the narrow-form crossover is the largest
width at which it wins, and results are cached per (n, p) bucket and grid."""
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


def test_fastest_valid_configuration_and_crossover(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "trial", _fake_trial)
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
    monkeypatch.setenv("BNB_AUTOTUNE_CACHE", str(tmp_path / "cache.json"))
    grid = {"rho": [0.3], "precision": [3], "batch_K": [64], "relax_alpha": [1.0]}
    best, _ = autotune.autotune(np.zeros((100, 500)), np.zeros(100), 0.1, 0.01, 1.0, grid=grid,
                                use_cache=False)
    assert best["mv_crossover"] == 0
