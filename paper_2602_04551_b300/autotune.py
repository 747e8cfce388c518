"""Autotuner for the node-batch solve: ADMM penalty rho, batch width K, stop-test
interval (check_every) and arithmetic mode, chosen per problem by measurement.

Each trial creates a handle with the candidate options, solves the root once and
then a batch of K child nodes warm-started from it (random fixings of small
depth, the shape of the nodes the tree produces) through bnb_relax_batch_device,
timed with CUDA events on the handle's stream.  The score is certified nodes per
second; the mean FP64 bound of the batch is recorded so that a mode whose bounds
are markedly weaker (e.g. plain BF16) is not chosen for speed alone.
The few best candidates of that batch measurement (search_top) are then timed on the
tree search itself (search_trial): a solve of the problem with the candidate options is
run until its node slots are busy, and the certified nodes of the next rounds per second
decide.  The batch measurement alone ranks candidates of close score unreliably: its
random children are not the nodes the search produces, and its time is set by the
slowest node of the batch, where the search refills each slot as its node finishes.
With check_every_values the stop-test interval is then chosen the same way, by search
measurements of the chosen configuration at each interval.
A second, short measurement picks the crossover below which a round runs the
narrow matrix-vector form instead of tensor-core tiles (mv_crossover): batches of 4 to
32 children are timed with the narrow form forced on and off, and the crossover is the
largest width at which it is faster.
Results are cached in a JSON file keyed by (n, p) bucket.
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

DEFAULT_GRID = {
    "rho": [0.1, 0.2, 0.3, 0.5, 1.0],
    "relax_alpha": [1.0, 1.6],
    "batch_K": [256, 512, 1024],
    "check_every": [10],
    "precision": [3],
}


def _cache_path():
    return os.environ.get("BNB_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bnb_autotune.json"))


def _key(n, p, grid):
    b = lambda v: round(2.0 * float(np.log2(max(v, 1)))) / 2.0      # half-octave buckets
    g = ",".join(f"{k}={grid[k]}" for k in sorted(grid))
    return f"{b(n)}x{b(p)}|{g}"


def _children(p, K, seed, depth=8):
    rng = np.random.default_rng(seed)
    fix = np.full((K, p), -1, np.int8)
    for k in range(K):
        d = int(rng.integers(1, depth + 1))
        idx = rng.choice(p, size=min(d, p), replace=False)
        fix[k, idx] = (rng.random(len(idx)) < 0.3).astype(np.int8)
    return fix


def trial(X, y, lam0, lam2, M, opts: dict, device=0, seed=0, nodes=None):
    """Time the root plus a batch of `nodes` (default batch_K) warm-started children."""
    import torch
    import paper_2602_04551_b300 as bnb
    K = int(opts["batch_K"]) if nodes is None else int(nodes)
    p = X.shape[1]
    s = torch.cuda.Stream(device=device)
    o = bnb.bnb_options_default(M=M, device=device, stream=s.cuda_stream, **opts)
    with bnb.bnb_create(X, y, lam0, lam2, o) as h:
        root = bnb.bnb_relax_batch(h, np.full((1, p), -1, np.int8), want_v=True)
        fix = _children(p, K, seed)
        wb = np.repeat(root["beta"], K, 0)
        wb[fix == 0] = 0.0
        dfix = torch.tensor(fix, device=f"cuda:{device}")
        dwb = torch.tensor(wb, device=f"cuda:{device}")
        dwv = torch.tensor(np.repeat(root["v"], K, 0), device=f"cuda:{device}")
        dlb = torch.empty(K, dtype=torch.float64, device=f"cuda:{device}")
        dit = torch.empty(K, dtype=torch.int32, device=f"cuda:{device}")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.synchronize()
        e0.record(s)
        bnb.bnb_relax_batch_device(h, K, dfix, dwb, dwv, 0, dlb, diters=dit)
        e1.record(s)
        s.synchronize()
        ms = e0.elapsed_time(e1)
        return {"nodes_per_s": K / (ms / 1e3), "ms": ms, "mean_iters": float(dit.float().mean()),
                "lb_mean": float(dlb.mean())}


def steady(pr: dict, K: int) -> bool:
    """A solve is in its steady state once a batch's worth of nodes has been certified
    and the pool holds at least K open nodes besides the active slots, so that every
    refill fills each free slot.  (The active-slot count itself is read after the round's
    stop test has retired its converged slots, so with a long stop-test interval it sits
    well below K even when the slots are all busy.)"""
    return pr["nodes"] >= K and pr["open_nodes"] - pr["active_slots"] >= K


def search_trial(X, y, lam0, lam2, M, opts: dict, device=0, rounds=300, prime_rounds=400,
                 warm_rounds=125, gap=1e-4):
    """Certified nodes per second of the tree search with the candidate options: a solve
    primed until 90 % of its slots are busy and a batch's worth of nodes is certified (at
    most prime_rounds rounds), `warm_rounds` more rounds, then `rounds` rounds timed with
    CUDA events on the handle's stream.  The rate changes as the tree grows (a setting
    that retires nodes faster in the first rounds can be the slower one a few hundred
    rounds later), so the timed rounds start where a long solve's steady state does.  None
    when the solve ends before the timed rounds."""
    import torch
    import paper_2602_04551_b300 as bnb
    K = int(opts["batch_K"])
    s = torch.cuda.Stream(device=device)
    o = bnb.bnb_options_default(M=M, device=device, stream=s.cuda_stream, time_limit_s=1e9,
                                **opts)
    with bnb.bnb_create(X, y, lam0, lam2, o) as h:
        bnb.bnb_solve_start(h, gap)
        primed = 0
        while primed < prime_rounds:
            bnb.bnb_solve_launch(h, 20)
            primed += 20
            pr = bnb.bnb_solve_poll(h)
            if pr["done"]:
                return None
            if steady(pr, K):
                break
        if warm_rounds > 0:
            bnb.bnb_solve_launch(h, warm_rounds)
            pr = bnb.bnb_solve_poll(h)
            if pr["done"]:
                return None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.synchronize()
        e0.record(s)
        bnb.bnb_solve_launch(h, rounds)
        e1.record(s)
        s.synchronize()
        after = bnb.bnb_solve_poll(h)
        ms = e0.elapsed_time(e1)
        bnb.bnb_solve_finish(h)
    nodes = after["nodes"] - pr["nodes"]
    return {"search_nodes_per_s": nodes / (ms / 1e3), "search_ms": ms, "search_nodes": nodes,
            "search_rounds": rounds, "prime_rounds": primed + warm_rounds}


def crossover(X, y, lam0, lam2, M, opts: dict, device=0, widths=(4, 8, 16, 32)):
    """Largest batch width (<= 32) at which the narrow matrix-vector form beats the
    tensor-core form on `widths`-node batches; 0 when it never does."""
    best = 0
    rows = []
    for w in widths:
        narrow = trial(X, y, lam0, lam2, M, dict(opts, mv_crossover=32), device=device, nodes=w)
        wide = trial(X, y, lam0, lam2, M, dict(opts, mv_crossover=0), device=device, nodes=w)
        rows.append({"width": w, "narrow_ms": narrow["ms"], "wide_ms": wide["ms"]})
        if narrow["ms"] < wide["ms"]:
            best = w
    return best, rows


def autotune(X, y, lam0, lam2, M, grid=None, device=0, use_cache=True, bound_tol=1e-3,
             tune_crossover=True, search_top=4, check_every_values=None):
    grid = dict(DEFAULT_GRID, **(grid or {}))
    n, p = X.shape
    key = _key(n, p, grid) + f"|search_top={search_top}|ce={check_every_values}"
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except Exception:
            cache = {}
        if key in cache:
            return cache[key]["best"], cache[key]
    names = list(grid)
    results = []
    t0 = time.time()
    for combo in itertools.product(*[grid[k] for k in names]):
        opts = dict(zip(names, combo))
        r = trial(X, y, lam0, lam2, M, opts, device=device)
        results.append((opts, r))
    best_lb = max(r["lb_mean"] for _, r in results)
    ok = [(o, r) for o, r in results if r["lb_mean"] >= best_lb - bound_tol * max(1.0, abs(best_lb))]
    ok.sort(key=lambda t: -t[1]["nodes_per_s"])
    best, br = ok[0]
    searched = []
    if search_top > 0:
        for o, r in ok[:search_top]:
            st = search_trial(X, y, lam0, lam2, M, o, device=device)
            if st is not None:
                r.update(st)
                searched.append((o, r))
        if searched:
            best, br = max(searched, key=lambda t: t[1]["search_nodes_per_s"])
    best = dict(best)
    ce_rows = []
    if check_every_values and "search_nodes_per_s" in br:
        # the stop-test interval, on the search alone: the batch measurement cannot see it
        # (a longer interval spreads each round's fixed work -- certificate, branching,
        # upper bound, selection -- over more iterations, but a converged node waits longer
        # for its test)
        ce_rows.append({"check_every": best.get("check_every"),
                        "search_nodes_per_s": br["search_nodes_per_s"]})
        for ce in check_every_values:
            if ce == best.get("check_every"):
                continue
            st = search_trial(X, y, lam0, lam2, M, dict(best, check_every=ce), device=device)
            if st is not None:
                ce_rows.append({"check_every": ce, "search_nodes_per_s": st["search_nodes_per_s"]})
        top = max(ce_rows, key=lambda r: r["search_nodes_per_s"])
        if top["check_every"] != best.get("check_every"):
            best["check_every"] = top["check_every"]
            br = dict(br, search_nodes_per_s=top["search_nodes_per_s"])
    cross_rows = []
    if tune_crossover and best.get("precision", 3) in (2, 3, 4):
        best["mv_crossover"], cross_rows = crossover(X, y, lam0, lam2, M, best, device=device)
    entry = {"best": best, "score": br, "trials": [dict(o, **r) for o, r in results],
             "check_every": ce_rows, "crossover": cross_rows, "seconds": time.time() - t0}
    if use_cache:
        cache[key] = entry
        os.makedirs(os.path.dirname(path), exist_ok=True)
        json.dump(cache, open(path, "w"), indent=1)
    return best, entry
