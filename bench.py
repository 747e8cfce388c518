#!/usr/bin/env python
"""Benchmark: certified branch-and-bound nodes per second on one B300.

Workload (default "c2"): n=1000, p=5000, Toeplitz rho=0.3, k=10 true ones,
SNR=5, lambda2=1e-3, M = 1.5 ||ridge on the true support||_inf, lambda0 from a
sweep relative to max_j (X_j^T y)^2 / (2(||X_j||^2 + 2 lambda2)), node-batch
width K=512, target gap 1e-4, FP32 ADMM with FP64 certificates.

A "step" is a fixed block of --rounds-per-step (default 25) device rounds of the
solve; a round refills free slots best-first, runs check_every ADMM iterations over
all K slots, certifies the nodes that stopped in FP64, picks branches and takes the
batched upper bound, and prunes/branches into the pool.
  value     nodes certified per second over the timed steps (device time, CUDA
            events on the solve's stream; L2 flushed with a 256 MiB write
            before every step, outside the timed interval)
  e2e       nodes certified per second through bnb_relax_batch with host
            buffers: each step uploads K nodes (fixings + warm starts) from
            pinned memory and reads back bounds, beta, z
  fp64_path the plain FP64 GPU path on the same batch of nodes (the comparator)
  fp32_path the same timed rounds with the FP32 CUDA-core ADMM (no tensor cores)
  roofline  the dominant kernel of a profiled round (CUDA events per launch)
  cpu_baseline the FP64 oracle's node solves on the host cores, bounded sample
  reverify  the certificates of a short logged solve of the same workload re-checked by
            the FP64 oracle at the logged residuals
  certified_solves  full solves to gap 1e-4 over five lambda0 values chosen so that
            the first incumbent has 5, 8, 12, 16 and 20 nonzeros, mixed precision
            and plain FP64, per instance, and where the mixed path certified, again
            with the early-branch node stop; with `reverify`: certificates of a real
            solve and every final support re-checked by the FP64 oracle
  serve     a short run of the serving workload (32 requests): p50/p99 latency,
            queueing and service time, certified count

`--impl reference` times the FP64 oracle itself (the reference arm for this
build): node solves of the same workload on the host cores.
Multi-GPU (torchrun): every rank solves its own instance (independent trees,
no collective on the data path); value = all ranks' nodes / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import datagen  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
PREC = {"fp32": 1, "bf16": 2, "tc3": 3, "fp64": 0, "bf16x2": 4}
DTYPE = {"fp32": "f32", "bf16": "bf16", "tc3": "bf16x3", "fp64": "f64", "bf16x2": "bf16x2"}
SM_COUNT, FP32_LANES = 148, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--mode", default="rounds", choices=["rounds", "solves", "serve", "kcurve"],
                    help="rounds: steady-state nodes/s (default); solves: full solves over a "
                         "lambda0 sweep; serve: Poisson request stream through the serving loop")
    ap.add_argument("--lam0-fracs", default="0.3,0.15,0.08,0.05,0.03")
    ap.add_argument("--solve-time-limit", type=float, default=120.0)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--arrival-rate", type=float, default=20.0)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--fp64-compare", action="store_true",
                    help="solves mode: also solve each instance with the plain FP64 path")
    ap.add_argument("--fp64-time-limit", type=float, default=60.0)
    ap.add_argument("--seeds", type=int, default=1, help="solves mode: instances per lambda0")
    ap.add_argument("--max-depth", type=int, default=1024)
    ap.add_argument("--fused-shape", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="fused X^T U' shape: 0 measured at setup, 1 one CTA per tile, "
                         "2 clusters of two sharing X, 3 transposed on CTA pairs, "
                         "4 untransposed on CTA pairs")
    ap.add_argument("--fused-width", type=int, default=0,
                    help="tile width of the fused X^T U' product (0: measured at setup)")
    ap.add_argument("--early-branch", type=int, default=0, choices=[0, 1],
                    help="solves: retire a node whose primal estimate is already below the "
                         "prune threshold (bnb_options.early_branch)")
    ap.add_argument("--exact-bounds", type=int, default=0, choices=[0, 1],
                    help="exact FP64 certificate terms for every branched node (1) or only "
                         "where they can change the prune decision (0)")
    ap.add_argument("--fused-select", type=int, default=0, choices=[0, 1],
                    help="the selection as one cooperative launch (1) or separate launches (0)")
    ap.add_argument("--u-shape", type=int, default=0, choices=[0, 1, 2, 3],
                    help="U' = H W'^T: 0 measured at setup, 1 cluster-reduced, 2 CTA pairs split-K, 3 CTA pairs in split-K clusters")
    ap.add_argument("--mv-crossover", type=int, default=-1,
                    help="narrow-form crossover (-1 default; 0 = tensor-core form only: graphs "
                         "without conditional nodes, which ncu can profile kernel by kernel)")
    ap.add_argument("--k-list", default="1,4,16,64,256,512",
                    help="kcurve mode: batch widths; each solve runs --solve-time-limit seconds")
    ap.add_argument("--lam0-frac", type=float, default=0.02)
    ap.add_argument("--K", type=int, default=512)
    ap.add_argument("--check-every", type=int, default=0,
                    help="ADMM iterations between stop tests (0: chosen by the autotuner among "
                         "10, 20 and 30 on search measurements, 10 when --rho is given)")
    ap.add_argument("--rounds-per-step", type=int, default=25,
                    help="device rounds in one timed step")
    ap.add_argument("--no-side", action="store_true",
                    help="skip the side measurements (fp32 path, certified solves, serve)")
    ap.add_argument("--cert-time-limit", type=float, default=8.0,
                    help="per-solve limit of the certified_solves side key (each path)")
    ap.add_argument("--serve-requests", type=int, default=32)
    ap.add_argument("--serve-time-limit", type=float, default=20.0)
    ap.add_argument("--fp32-steps", type=int, default=4)
    ap.add_argument("--reverify-nodes", type=int, default=128,
                    help="certificates of a short logged solve re-checked by the oracle (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--fp64-steps", type=int, default=4)
    ap.add_argument("--fp64-K", type=int, default=512,
                    help="nodes in the FP64-vs-mixed comparison batch (bounded for large shapes)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--prime-seconds", type=float, default=90.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", default="tc3", choices=["fp32", "tc3", "bf16", "bf16x2"])
    ap.add_argument("--rho", type=float, default=0.0, help="0: chosen by the autotuner")
    ap.add_argument("--alpha", type=float, default=1.0, help="ADMM over-relaxation (autotuned with rho)")
    args = ap.parse_args()
    # the interval is tuned only with rho (timed-rounds mode); elsewhere it defaults to 10
    args.check_every_auto = args.check_every <= 0 and args.rho <= 0 and args.mode == "rounds"
    if args.check_every <= 0:
        args.check_every = 10
    return args


METRIC = "certified BnB nodes/s"        # both arms report this metric on the same config


def note(msg):
    """Progress of the run on stderr (the JSON line goes to stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def line_config(cfg, args):
    """The `config` object of both arms' JSON lines: the workload, its batch width and
    target gap, and how the GPU arm keeps inputs out of L2 between timed steps."""
    return dict(cfg, K=args.K, gap=1e-4, parallelism="replicas",
                l2="GPU arm: a 256 MiB write flushes L2 before every timed step")


def workload(name, inst_id, lam0_frac):
    c = datagen.CONFIGS[name]
    inst = datagen.config_instance(name, inst_id)
    lam2 = c["lam2"]
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = lam0_frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    cfg = {"workload": name, "n": c["n"], "p": c["p"], "toeplitz_rho": c["rho"], "k_true": c["k"],
           "snr": c["snr"], "lambda2": lam2, "lambda0": lam0, "lambda0_frac": lam0_frac, "M": M,
           "seed": inst.seed}
    return inst, lam0, lam2, M, cfg


def node_sample(inst, K, seed, depth=8):
    """K child-like nodes: random fixings of depth <= `depth` (datagen recipe)."""
    rng = np.random.default_rng(seed)
    return datagen.random_fixings(inst.p, K, rng, depth)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {}


# --------------------------------------------------------------------------- mine


def run_mine(args, rank, world):
    import torch
    import paper_2602_04551_b300 as bnb

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    inst, lam0, lam2, M, cfg = workload(args.workload, rank, args.lam0_frac)
    tune = None
    if args.rho <= 0:
        from paper_2602_04551_b300 import autotune
        # (the timed rounds are wide batches: the narrow-form crossover does not enter)
        best, entry = autotune.autotune(inst.X, inst.y, lam0, lam2, M, device=dev, use_cache=False,
                                        grid={"batch_K": [args.K], "precision": [PREC[args.precision]],
                                              "check_every": [args.check_every]},
                                        tune_crossover=False,
                                        check_every_values=(10, 20, 30) if args.check_every_auto
                                        else None)
        args.rho = float(best["rho"])
        args.alpha = float(best.get("relax_alpha", 1.0))
        args.check_every = int(best["check_every"])
        note(f"autotune: rho {args.rho} alpha {args.alpha}")
        tune = {"chosen": best, "seconds": entry["seconds"], "check_every": entry["check_every"],
                "trials": [{k: t[k] for k in ("rho", "relax_alpha", "nodes_per_s", "mean_iters",
                                              "lb_mean", "search_nodes_per_s") if k in t}
                           for t in entry["trials"]]}
    s = torch.cuda.Stream()
    opt = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every,
                                  precision=PREC[args.precision], device=dev, stream=s.cuda_stream,
                                  queue_capacity=1 << 21, time_limit_s=1e9, rho=args.rho,
                                  relax_alpha=args.alpha, mv_crossover=args.mv_crossover,
                                  fused_shape=args.fused_shape, u_shape=args.u_shape,
                                  fused_width=args.fused_width, fused_select=args.fused_select,
                                  exact_bounds=args.exact_bounds)
    h = bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    gap = 1e-4
    bnb.bnb_solve_start(h, gap)
    # priming (untimed): grow the tree until a batch's worth of nodes has been certified
    # and the pool holds a batch of open nodes beside the slots, so that the timed rounds
    # measure the steady state of the solve (slots retiring and refilling) rather than its
    # first nodes, and not a pool grown to its capacity
    from paper_2602_04551_b300 import autotune
    t0 = time.time()
    prime_rounds = 0
    while True:
        bnb.bnb_solve_launch(h, 20)
        prime_rounds += 20
        pr = bnb.bnb_solve_poll(h)
        if pr["done"] or autotune.steady(pr, args.K) or time.time() - t0 > args.prime_seconds:
            break
    note(f"primed: {prime_rounds} rounds")
    clk = Clocks(dev)            # sampling spans the warm-up and the timed steps
    time.sleep(0.3)
    R = args.rounds_per_step
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            bnb.bnb_solve_launch(h, R)
    before = bnb.bnb_solve_poll(h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("bench_timed")
    with torch.cuda.stream(s):
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(s)
            bnb.bnb_solve_launch(h, R)
            ev[i][1].record(s)
    s.synchronize()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    clocks = clk.stop()
    after = bnb.bnb_solve_poll(h)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    nodes = after["nodes"] - before["nodes"]
    stats = bnb.bnb_get_stats(h)
    prof = bnb.bnb_profile_round(h)   # one extra round with per-stage CUDA events
    prog = bnb.bnb_solve_poll(h)
    kernels_per_round = stats.get("round_kernels", 0)
    res = bnb.bnb_solve_finish(h)
    h.close()
    shapes = {k: stats.get(k) for k in ("xw_tile_width", "xw_cluster", "fused_tile_width",
                                          "fused_clusters", "fused_pairs", "fused_transposed",
                                          "u_split", "u_cluster_pairs")}
    out = dict(ms=ms, nodes=nodes, prof=prof, prog=prog, clocks=clocks, cfg=cfg, tune=tune,
               setup_seconds=stats.get("setup_seconds"),
               kernels=kernels_per_round * args.steps * R, after=after, res=res, shapes=shapes,
               rounds=after["rounds"] - before["rounds"],
               prime={"rounds": prime_rounds, "seconds": time.time() - t0,
                      "active_slots": before["active_slots"], "open_nodes": before["open_nodes"]})
    note(f"timed: {nodes} nodes in {ms:.1f} ms")
    if rank == 0:
        out["e2e"] = run_e2e(args, inst, lam0, lam2, M, dev)
        note("e2e done")
        out["fp64"] = run_fp64(args, inst, lam0, lam2, M, dev)
        note("fp64 same-batch done")
        if world == 1 and args.reverify_nodes > 0:
            out["reverify"] = run_reverify(args, inst, lam0, lam2, M, dev)
            note("reverify done")
        if world == 1 and not args.no_side:
            out["fp32"] = run_fp32_side(args, inst, lam0, lam2, M, dev)
            note("fp32 side done")
            out["certified"] = run_certified(args, inst.seed - 1000 * datagen.CONFIGS[args.workload]["cfg_id"])
            note("certified solves done")
            out["serve"] = run_serve_side(args)
            note("serve side done")
    return out


def run_fp32_side(args, inst, lam0, lam2, M, dev):
    """The same workload and timed steps with the FP32 CUDA-core ADMM (BNB_PREC_FP32): the
    path that computes the FP32 ADMM literally, beside the tensor-core default."""
    import torch
    import paper_2602_04551_b300 as bnb
    from paper_2602_04551_b300 import autotune
    s = torch.cuda.Stream()
    opt = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every,
                                  precision=bnb.BNB_PREC_FP32, device=dev, stream=s.cuda_stream,
                                  queue_capacity=1 << 21, time_limit_s=1e9, rho=args.rho,
                                  relax_alpha=args.alpha)
    R = args.rounds_per_step
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt) as h:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
        bnb.bnb_solve_start(h, 1e-4)
        t0 = time.time()
        while True:
            bnb.bnb_solve_launch(h, 20)
            pr = bnb.bnb_solve_poll(h)
            if pr["done"] or autotune.steady(pr, args.K) or time.time() - t0 > args.prime_seconds:
                break
        with torch.cuda.stream(s):
            bnb.bnb_solve_launch(h, R)
        before = bnb.bnb_solve_poll(h)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.fp32_steps)]
        torch.cuda.synchronize()
        with torch.cuda.stream(s):
            for i in range(args.fp32_steps):
                flush.fill_(i & 0xff)
                ev[i][0].record(s)
                bnb.bnb_solve_launch(h, R)
                ev[i][1].record(s)
        s.synchronize()
        after = bnb.bnb_solve_poll(h)
        ms = sum(a.elapsed_time(b) for a, b in ev)
        bnb.bnb_solve_finish(h)
    nodes = after["nodes"] - before["nodes"]
    rounds = after["rounds"] - before["rounds"]
    return {"value": nodes / (ms / 1e3), "unit": "nodes/s", "precision": "fp32",
            "ms_per_round": ms / max(1, rounds), "rounds": rounds, "nodes": nodes,
            "how": f"{args.fp32_steps} steps of {R} rounds after priming, same workload, K, "
                   "rho and alpha; FP32 state and products on CUDA cores, FP64 certificates"}


def run_e2e(args, inst, lam0, lam2, M, dev):
    """bnb_relax_batch with pinned host buffers: K child nodes per step."""
    import torch
    import paper_2602_04551_b300 as bnb

    K = args.K
    opt = bnb.bnb_options_default(M=M, batch_K=K, check_every=args.check_every, device=dev,
                                  precision=PREC[args.precision], rho=args.rho,
                                  relax_alpha=args.alpha)
    h = bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt)
    p = inst.p
    root = bnb.bnb_relax_batch(h, np.full((1, p), -1, np.int8), want_v=True)
    pin = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    fix = pin((K, p), torch.int8)
    wb = pin((K, p), torch.float32)
    wv = pin((K, p), torch.float32)
    fix[:] = node_sample(inst, K, 7)
    wb[:] = root["beta"][0][None, :]
    wb[fix == 0] = 0.0
    wv[:] = root["v"][0][None, :]
    h2d = fix.nbytes + wb.nbytes + wv.nbytes
    d2h = K * 8 + 2 * K * p * 4 + K * 4 + K * 8 + K * 4
    bnb.bnb_relax_batch(h, fix, wb, wv)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        bnb.bnb_relax_batch(h, fix, wb, wv)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    h.close()
    return {"value": K * args.e2e_steps / dt, "unit": "nodes/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "call": "bnb_relax_batch (host buffers)",
            "nodes_per_step": K}


def run_fp64(args, inst, lam0, lam2, M, dev):
    """Plain FP64 GPU path vs the FP32 path on the same batch of K child nodes
    (bnb_relax_batch_device, device time with CUDA events on the handle stream)."""
    import torch
    import paper_2602_04551_b300 as bnb

    K, p = min(args.K, args.fp64_K), inst.p
    fix = node_sample(inst, K, 7)
    res = {}
    for name, prec in (("mixed", PREC[args.precision]), ("fp64", bnb.BNB_PREC_FP64)):
        s = torch.cuda.Stream()
        opt = bnb.bnb_options_default(M=M, batch_K=K, check_every=args.check_every, device=dev,
                                      precision=prec, stream=s.cuda_stream, rho=args.rho,
                                      relax_alpha=args.alpha)
        h = bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt)
        root = bnb.bnb_relax_batch(h, np.full((1, p), -1, np.int8), want_v=True)
        wb = np.repeat(root["beta"], K, 0)
        wb[fix == 0] = 0.0
        wv = np.repeat(root["v"], K, 0)
        dfix = torch.tensor(fix, device="cuda")
        dwb = torch.tensor(wb, device="cuda")
        dwv = torch.tensor(wv, device="cuda")
        dlb = torch.empty(K, dtype=torch.float64, device="cuda")
        dit = torch.empty(K, dtype=torch.int32, device="cuda")
        bnb.bnb_relax_batch_device(h, K, dfix, dwb, dwv, 0, dlb, diters=dit)  # warm-up
        steps = 1 if name == "fp64" else 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.synchronize()
        e0.record(s)
        for _ in range(steps):
            bnb.bnb_relax_batch_device(h, K, dfix, dwb, dwv, 0, dlb, diters=dit)
        e1.record(s)
        s.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res[name] = {"nodes_per_s": K / (ms / 1e3), "ms_per_batch": ms,
                     "mean_iters": float(dit.float().mean()), "lb_mean": float(dlb.mean()),
                     "lb": dlb.cpu().numpy()}
        h.close()
    # bound error of the mixed-precision certificates against the FP64 path, per node
    rel = np.abs(res["mixed"]["lb"] - res["fp64"]["lb"]) / np.maximum(1.0, np.abs(res["fp64"]["lb"]))
    bound_error = {"max_rel": float(rel.max()), "median_rel": float(np.median(rel)),
                   "mixed_minus_fp64_mean": float(np.mean(res["mixed"]["lb"] - res["fp64"]["lb"]))}
    for r in res.values():
        r.pop("lb")
    return {"value": res["fp64"]["nodes_per_s"], "unit": "nodes/s",
            "mixed_same_batch": res["mixed"], "fp64": res["fp64"], "bound_error": bound_error,
            "how": "K child nodes of the workload, warm start from the root, node tol 1e-4; "
                   "bnb_relax_batch_device, CUDA events"}


# ---------------------------------------------------------------------- oracle


def oracle_threads():
    """Threads the oracle's numpy arithmetic runs on: the BLAS pool's size (its node
    solves are matrix-vector products), else the host's core count."""
    try:
        from threadpoolctl import threadpool_info
        n = [d["num_threads"] for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def oracle_setup(args, inst=None, lam0=None, lam2=None, M=None, cfg=None):
    """The oracle's per-problem setup (its direct D = (X^T X + rho I)^-1 and the root
    relaxation, which the children warm-start from) and a sample of child fixings."""
    from oracle import admm
    if inst is None:
        inst, lam0, lam2, M, cfg = workload(args.workload, 0, args.lam0_frac)
    data = admm.AdmmData(inst.X, inst.y, 1.0)
    root = admm.solve_node(data, np.full(inst.p, -1, np.int8), lam0, lam2, M, tol=1e-4,
                           max_iter=400)
    return {"data": data, "root": root, "fix": node_sample(inst, 64, 7), "lam0": lam0,
            "lam2": lam2, "M": M, "cfg": cfg, "next": 0}


def oracle_nodes(st, seconds):
    """FP64 oracle child-node solves (as the oracle stands) until `seconds` have passed
    (at least one); returns (nodes, seconds)."""
    from oracle import admm
    fix = st["fix"]
    t0 = time.perf_counter()
    done = 0
    while True:
        k = st["next"] % fix.shape[0]
        st["next"] += 1
        wb = st["root"].beta.copy()
        wb[fix[k] == 0] = 0.0
        admm.solve_node(st["data"], fix[k], st["lam0"], st["lam2"], st["M"], beta0=wb,
                        v0=st["root"].v, tol=1e-4, max_iter=400)
        done += 1
        if time.perf_counter() - t0 > seconds:
            break
    return done, time.perf_counter() - t0


def oracle_sample_text(cfg, done, dt):
    return (f"{done} child nodes of the {cfg['workload']} workload (warm start from the "
            f"root, node tol 1e-4, <=400 ADMM iterations), FP64 numpy, {dt:.1f} s")


def run_oracle(args, seconds, inst=None, lam0=None, lam2=None, M=None, cfg=None):
    """FP64 oracle node solves (as the oracle stands) on a bounded sample."""
    st = oracle_setup(args, inst, lam0, lam2, M, cfg)
    done, dt = oracle_nodes(st, seconds)
    return {"value": done / dt, "unit": "nodes/s", "cores": oracle_threads(), "kind": "oracle",
            "sample": oracle_sample_text(st["cfg"], done, dt)}


def reference_arm(args):
    """The oracle timed on the host cores: one setup, then each step a bounded sample of
    child-node solves (at least one), sized so that the whole run stays within a few
    minutes whatever --steps and --warmup are."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    inst, lam0, lam2, M, cfg = workload(args.workload, 0, args.lam0_frac)
    st = oracle_setup(args, inst, lam0, lam2, M, cfg)
    budget = 150.0 / max(1, args.steps + args.warmup)
    for _ in range(args.warmup):
        oracle_nodes(st, budget * 0.2)
    nodes, secs = 0, 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        d, dt = oracle_nodes(st, budget)
        nodes += d
        secs += dt
    wall = time.perf_counter() - t0
    v = nodes / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "nodes/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": line_config(cfg, args),
            "cpu_baseline": {"value": v, "unit": "nodes/s", "cores": oracle_threads(),
                             "kind": "oracle", "sample": oracle_sample_text(cfg, nodes, secs)},
            "e2e": {"value": v, "unit": "nodes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------ main


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the dominant kernel per
# launch, from one ncu capture summarised under profiles/; it is reported only while the
# source that defines the captured kernel is unchanged (hash of the kernel template, its
# tile geometry, its epilogue, the epilogue warp count and the shared device helpers),
# else null.
_COMMON = (("common.cuh", "", None),)
_PERSIST = (("tc_gemm.cuh", "tc_gemm_persist_kernel(", "\n}\n"),
            ("tc_gemm.cuh", "template <int BN, int NSPLIT>\nstruct Geo {", "\n};\n"),
            ("admm_tc.cu", "struct TcEpiAdmm {", "\n};\n"),
            ("admm_tc.cu", "constexpr int FUSED_EPIW", "\n")) + _COMMON
_PAIR = (("tc_gemm.cuh", "tc_gemm_pair_kernel(", "\n}\n"),
         ("tc_gemm.cuh", "template <int BN, int NSPLIT>\nstruct PairGeo {", "\n};\n"),
         ("admm_tc.cu", "struct TcEpiAdmmT {", "\n};\n"),
         ("admm_tc.cu", "constexpr int PAIR_EPIW", "\n")) + _COMMON
_PAIR_NT = (("tc_gemm.cuh", "tc_gemm_pair_kernel(", "\n}\n"),
            ("tc_gemm.cuh", "template <int BN, int NSPLIT>\nstruct PairGeo {", "\n};\n"),
            ("admm_tc.cu", "struct TcEpiAdmm {", "\n};\n"),
            ("admm_tc.cu", "struct TcEpiAdmmPair {", "\n};\n"),
            ("admm_tc.cu", "constexpr int PAIR_EPIW", "\n")) + _COMMON
_NOTE = "ncu capture of {k} on the c2 workload (~500 active slots), profiles/{f}"
TRAFFIC = {
    # (stage, workload, K, precision, fused tile width, clusters of two sharing X, CTA pairs,
    #  transposed)
    ("gemm_xtu_prox", "c2", 512, "tc3", 176, False, True, False): {
        "blocks": _PAIR_NT, "sources": "50944af0a1ee1eec", "bytes": 45.185152e6 + 0.581760e6,
        "note": _NOTE.format(k="tc_gemm_pair_kernel<176, 3, TcEpiAdmmPair<176, 0>, 12>",
                             f="fused_pair_untransposed_c2_K512_tc3.md")},
}


def sources_hash(blocks):
    """Hash of the source text that defines one captured kernel."""
    import hashlib
    h = hashlib.sha256()
    for f, start, end in blocks:
        with open(os.path.join(ROOT, "paper_2602_04551_b300", "csrc", f)) as fh:
            text = fh.read()
        if start:
            i = text.index(start)
            text = text[i:text.index(end, i) + len(end)]
        h.update(text.encode())
    return h.hexdigest()[:16]


def roofline(out, args, pk):
    """Dominant contraction of the profiled round against its peak.

    CUDA-core path: FP32 FMA peak derived from 148 SMs x 128 lanes x 2 x 2032 MHz.
    Tensor-core paths: the measured sustained dense BF16 rate (the kernel is timed
    inside a long step).  `achieved` counts the algorithmic FLOPs (2 n p per node and
    product); the hi/lo path issues three tensor-core products per algorithmic one,
    reported as `achieved_hw`.
    """
    prof = out["prof"]
    cfg = out["cfg"]
    n, p = cfg["n"], cfg["p"]
    active = max(1, int(out["prog"]["active_slots"]))
    total = {k: v[0] * v[1] for k, v in prof.items()}
    flops = {"gemm_xw": 2.0 * n * p * active, "gemm_xtu_prox": 2.0 * n * p * active,
             "check_xbeta": 2.0 * n * p * active, "gemm_ginv_t": 2.0 * n * n * active}
    cand = {k: total[k] for k in flops if k in total}
    name = max(cand, key=cand.get)
    ms = prof[name][0]
    ach = flops[name] / (ms * 1e-3) / 1e12
    share = total[name] / max(1e-12, sum(total.values()))
    r = {"kernel": name, "achieved": ach, "unit": "TFLOP/s", "traffic": None,
         "share_of_round": share, "flops_per_launch": flops[name], "ms_per_launch": ms,
         "active_slots": active}
    sh = out.get("shapes") or {}
    tr = TRAFFIC.get((name, args.workload, args.K, args.precision, sh.get("fused_tile_width"),
                      bool(sh.get("fused_clusters")), bool(sh.get("fused_pairs")),
                      bool(sh.get("fused_transposed"))))
    if tr is not None and tr["sources"] == sources_hash(tr["blocks"]):
        r["traffic"] = tr["bytes"]
        r["traffic_note"] = tr["note"]
    if args.precision == "fp32":
        peak = SM_COUNT * FP32_LANES * 2 * 2032.0 * 1e6 / 1e12
        r.update(bound="alu", peak=peak, frac=ach / peak,
                 peak_note="FP32 FMA peak 148 SM x 128 lanes x 2 x 2032 MHz (derived)")
    else:
        # burst peak when the timed region ran at the maximum SM clock with no power cap
        # (the kernel is not power-limited there), else the sustained one
        clk = out.get("clocks") or {}
        burst = (clk.get("sm_mhz") and clk.get("sm_max_mhz")
                 and clk["sm_mhz"] >= 0.97 * clk["sm_max_mhz"]
                 and "sw_power_cap" not in (clk.get("reasons") or []))
        key = "bf16_tflops" if burst else "bf16_tflops_sustained"
        if key in pk:
            peak = float(pk[key])
            note = (f"measured {'burst' if burst else 'sustained'} dense BF16 (MEASURED_PEAKS.json); "
                    f"{'burst: SM clock at its maximum, no power cap in the timed region' if burst else 'sustained: clocks below maximum or power-capped'}")
        else:
            peak = 1800.0 if burst else 1400.0
            note = "fallback dense BF16 peak (no measured peaks file)"
        mult = {"tc3": 3.0, "bf16x2": 2.0}.get(args.precision, 1.0)
        r.update(bound="tensor", peak=peak, frac=ach / peak, achieved_hw=ach * mult,
                 frac_hw=ach * mult / peak, peak_note=note, peak_kind="burst" if burst else "sustained")
        other = "bf16_tflops_sustained" if burst else "bf16_tflops"
        if other in pk:
            r["frac_vs_" + ("sustained" if burst else "burst")] = ach / float(pk[other])
    if name == "gemm_xtu_prox" and "hbm_gbs" in pk:
        # the same launch against the copy bandwidth: its compulsory bytes are the data
        # operand (X as the precision stores it), U' and the node state the update reads
        # and writes (beta, V read and written, the fixing codes read, W' written: 21 bytes
        # per element in the tensor-core forms, 25 in FP32); most of it stays in L2
        ex = {"tc3": 4, "bf16x2": 2, "bf16": 2}.get(args.precision, 4)
        state = 21 if args.precision != "fp32" else 25
        nbytes = float(ex * n * p + ex * n * active + state * p * active)
        gbs = nbytes / (ms * 1e-3) / 1e9
        r["hbm_view"] = {"algorithmic_bytes": nbytes, "achieved_gbs": gbs,
                         "peak_gbs": float(pk["hbm_gbs"]), "frac": gbs / float(pk["hbm_gbs"]),
                         "note": "compulsory bytes of the launch over its time, against the "
                                 "measured copy bandwidth (the launch is not DRAM-bound: "
                                 "its working set stays largely in L2)"}
    return r


def combine_ranks(ms, nodes, world):
    """Whole-job figures from independent per-rank solves: the slowest rank's time
    and the total of the nodes every rank certified (host-side timing reduction;
    the solves themselves exchange nothing)."""
    if world <= 1:
        return ms, nodes
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms, float(nodes)], dtype=torch.float64, device=dev)
    mx = t.clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(mx[0]), float(t[1])


# lambda0 where the workload gives a nonzero count: fractions of
# max_j (X_j^T y)^2 / (2(||X_j||^2 + 2 lambda2)) on a geometric grid
LAM0_TARGETS = (5, 8, 12, 16, 20)
LAM0_GRID = tuple(float(x) for x in np.geomspace(1.0, 0.008, 28))


def lambda0_by_count(inst, lam2, M, targets=LAM0_TARGETS, grid=LAM0_GRID, dev=0):
    """lambda0 for each target count of nonzeros: on the geometric grid of fractions, the
    support size of the first incumbent (the library's matching-pursuit root heuristic,
    polished exactly in FP64); per target, the geometric midpoint of the grid points that
    give that count, else the grid point whose count is nearest (ties to the larger
    lambda0).  Returns (picks, counts per grid point)."""
    import paper_2602_04551_b300 as bnb
    sc = datagen.lambda0_scale(inst.X, inst.y, lam2)
    counts = []
    for f in grid:
        o = bnb.bnb_options_default(M=M, batch_K=16, precision=bnb.BNB_PREC_FP32, device=dev,
                                    queue_capacity=1 << 12)
        with bnb.bnb_create(inst.X, inst.y, f * sc, lam2, o) as h:
            b, _ = bnb.bnb_root_heuristic(h)
        counts.append(int(np.count_nonzero(b)))
    picks = [dict(pk, lambda0=pk["lambda0_frac"] * sc) for pk in pick_lambda0(counts, grid, targets)]
    return picks, counts


def pick_lambda0(counts, grid, targets):
    """Per target count: the geometric midpoint of the grid fractions whose count equals it,
    else the fraction whose count is nearest (ties to the larger lambda0, the earlier grid
    point: the grid runs from large to small)."""
    picks = []
    for t in targets:
        hit = [i for i, c in enumerate(counts) if c == t]
        if hit:
            f = float(np.sqrt(grid[hit[0]] * grid[hit[-1]]))
        else:
            f = float(grid[min(range(len(grid)), key=lambda i: (abs(counts[i] - t), i))])
        picks.append({"target_nnz": t, "lambda0_frac": f})
    return picks


def greedy_lambda0(X, y, lam2, M, k):
    """Per-request lambda0 of the serving workload for a target of k nonzeros: forward
    single-coordinate steps from beta = 0 (each adds the coordinate whose fit on the current
    residual lowers 1/2||r||^2 + lam2 beta^2 most, then refits the ridge on the support),
    recording each step's drop; the greedy path stops at k nonzeros for lambda0 between the
    k-th and (k+1)-th drops, and their geometric mean is returned."""
    d = np.einsum("ij,ij->j", X, X) + 2.0 * lam2
    S, drops = [], []
    r = y.copy()
    for _ in range(k + 1):
        c = X.T @ r
        b = np.clip(c / d, -M, M)
        gain = c * b - 0.5 * d * b * b
        gain[S] = -np.inf
        j = int(np.argmax(gain))
        drops.append(float(gain[j]))
        S.append(j)
        XS = X[:, S]
        bs = np.clip(np.linalg.solve(XS.T @ XS + 2.0 * lam2 * np.eye(len(S)), XS.T @ y), -M, M)
        r = y - XS @ bs
    return float(np.sqrt(max(drops[k - 1], 1e-300) * max(drops[k], 1e-300)))


def solve_record(args, inst, lam0, lam2, M, rho, alpha, prec, time_limit, log_nodes=0,
                 early_branch=None, check_every=None):
    """One full solve to gap 1e-4; its record (and the node log when requested).  The node
    stop settings default to the command line's."""
    import torch
    import paper_2602_04551_b300 as bnb
    o = bnb.bnb_options_default(M=M, batch_K=args.K,
                                check_every=args.check_every if check_every is None else check_every,
                                precision=prec, rho=rho, relax_alpha=alpha,
                                queue_capacity=1 << 21, max_depth=args.max_depth,
                                time_limit_s=time_limit, log_nodes=log_nodes,
                                early_branch=args.early_branch if early_branch is None
                                else early_branch)
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = bnb.bnb_solve(h, 1e-4)
        dt = time.perf_counter() - t0
        st = bnb.bnb_get_stats(h)
        log = bnb.bnb_get_node_log(h) if log_nodes else None
    rec = {"status": res["status"], "seconds": dt, "nodes": res["nodes"],
           "nnz": int(np.count_nonzero(res["beta"])), "ub": res["ub"], "lb": res["lb"],
           "gap": (res["ub"] - res["lb"]) / res["ub"], "nodes_per_s": res["nodes"] / dt,
           "max_depth": st["max_depth"], "setup_seconds": st.get("setup_seconds"),
           "certified": res["status"] in ("optimal", "gap")}
    return rec, res["beta"], log


def reverify_logs(inst, lam0, lam2, M, logs):
    """Logged certificates of real solves against the oracle's Eq. dual at the logged r:
    exact ones by relative error, screened ones by the excess D(r) - bound against their
    recorded interval width (a valid screened bound has 0 <= excess <= width)."""
    from oracle import relax
    rel, ratio, loose, n_ex, n_sc, bad = [], [], [], 0, 0, 0
    for log in logs:
        for k in range(log["count"]):
            d = relax.dual_value(inst.X, inst.y, log["r"][k], log["fix"][k], lam0, lam2, M)
            tol = 1e-10 * max(1.0, abs(d))
            if log["exact"][k] == 1.0:
                n_ex += 1
                rel.append(abs(log["lb"][k] - d) / max(1.0, abs(d)))
                bad += int(abs(log["lb"][k] - d) > tol)
            else:
                n_sc += 1
                ex = d - log["lb"][k]
                ratio.append(ex / log["width"][k] if log["width"][k] > 0 else 0.0)
                loose.append(ex / max(1.0, abs(d)))
                bad += int(ex < -tol or ex > log["width"][k] * (1 + 1e-9) + tol)
    return {"n_certs": n_ex + n_sc, "exact": n_ex, "screened": n_sc,
            "exact_max_rel": float(max(rel)) if rel else None,
            "exact_median_rel": float(np.median(rel)) if rel else None,
            "screened_max_excess_over_width": float(max(ratio)) if ratio else None,
            # how far a screened bound sits below the exact FP64 D(r) at the same r
            "screened_max_rel_below_exact": float(max(loose)) if loose else None,
            "screened_median_rel_below_exact": float(np.median(loose)) if loose else None,
            "violations": bad}


def run_reverify(args, inst, lam0, lam2, M, dev):
    """A short solve of the timed workload that logs its first --reverify-nodes certified
    nodes; each logged certificate is re-checked by the FP64 oracle's Eq. dual at the
    logged residual (reverify_logs)."""
    import paper_2602_04551_b300 as bnb
    o = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every, device=dev,
                                precision=PREC[args.precision], rho=args.rho,
                                relax_alpha=args.alpha, queue_capacity=1 << 20,
                                time_limit_s=60.0, log_nodes=args.reverify_nodes,
                                exact_bounds=args.exact_bounds)
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
        bnb.bnb_solve_start(h, 1e-4)
        while True:
            bnb.bnb_solve_launch(h, 5)
            pr = bnb.bnb_solve_poll(h)
            if pr["done"] or pr["nodes"] >= args.reverify_nodes:
                break
        log = bnb.bnb_get_node_log(h)
        bnb.bnb_solve_finish(h)
    t0 = time.perf_counter()
    out = reverify_logs(inst, lam0, lam2, M, [log])
    out["oracle_seconds"] = time.perf_counter() - t0
    return out


def run_certified(args, seed):
    """The certified_solves side key: the workload instance `seed`, lambda0 for 5, 8, 12,
    16 and 20 nonzeros, each solved to gap 1e-4 by the mixed-precision path (with a node
    log) and by the plain FP64 path under the same time limit; every final support
    re-checked by the oracle's exact objective, and the logged certificates by its Eq. dual."""
    import paper_2602_04551_b300 as bnb
    from oracle import ub as oub
    inst, _, lam2, M, cfg = workload(args.workload, seed, 0.1)
    t0 = time.perf_counter()
    picks, counts = lambda0_by_count(inst, lam2, M)
    t_grid = time.perf_counter() - t0
    rows, logs = [], []
    for pk in picks:
        lam0 = pk["lambda0"]
        row = dict(pk)
        for name, prec in (("mixed", PREC[args.precision]), ("fp64", bnb.BNB_PREC_FP64)):
            rec, beta, log = solve_record(args, inst, lam0, lam2, M, args.rho, args.alpha, prec,
                                          args.cert_time_limit, 128 if name == "mixed" else 0)
            S = np.nonzero(beta)[0]
            obj, _ = oub.support_objective(inst.X, inst.y, S, lam0, lam2, M)
            rec["support_objective_rel_diff"] = abs(obj - rec["ub"]) / abs(obj)
            row[name] = rec
            row[name + "_support"] = [int(i) for i in S]
            if name == "mixed":
                row["mixed_support_list"] = [int(i) for i in S]
            if log is not None:
                logs.append((lam0, log))
            note(f"certified target {pk['target_nnz']} {name}: {rec['status']} {rec['seconds']:.2f} s")
        row["same_support"] = row.pop("mixed_support") == row.pop("fp64_support")
        if row["mixed"]["certified"] and row["fp64"]["certified"]:
            row["speedup_time_to_certificate"] = row["fp64"]["seconds"] / row["mixed"]["seconds"]
        if row["mixed"]["certified"]:
            # the same instance with the early-branch node stop (a node whose primal estimate
            # is below the prune threshold is branched at once) and a stop test every 10
            # iterations: run where the default path certified, to time the same certificate
            rec, beta, _ = solve_record(args, inst, lam0, lam2, M, args.rho, args.alpha,
                                        PREC[args.precision], args.cert_time_limit,
                                        early_branch=1, check_every=10)
            S = np.nonzero(beta)[0]
            obj, _ = oub.support_objective(inst.X, inst.y, S, lam0, lam2, M)
            rec["support_objective_rel_diff"] = abs(obj - rec["ub"]) / abs(obj)
            rec["same_support_as_mixed"] = [int(i) for i in S] == row["mixed_support_list"]
            if rec["certified"]:
                rec["speedup_vs_mixed"] = row["mixed"]["seconds"] / rec["seconds"]
                if row["fp64"]["certified"]:
                    rec["speedup_vs_fp64"] = row["fp64"]["seconds"] / rec["seconds"]
            row["mixed_early_branch"] = rec
            # the plain FP64 path with the same node stop (same algorithm, FP64 everywhere)
            r64, b64, _ = solve_record(args, inst, lam0, lam2, M, args.rho, args.alpha,
                                       bnb.BNB_PREC_FP64, args.cert_time_limit,
                                       early_branch=1, check_every=10)
            r64["same_support_as_mixed"] = [int(i) for i in np.nonzero(b64)[0]] == \
                row["mixed_support_list"]
            if rec["certified"] and r64["certified"]:
                rec["speedup_vs_fp64_early_branch"] = r64["seconds"] / rec["seconds"]
            row["fp64_early_branch"] = r64
            note(f"certified target {pk['target_nnz']} fp64_early_branch: {r64['status']} "
                 f"{r64['seconds']:.3f} s")
            note(f"certified target {pk['target_nnz']} mixed_early_branch: {rec['status']} "
                 f"{rec['seconds']:.3f} s")
        row.pop("mixed_support_list", None)
        rows.append(row)
    cert = {}
    for name in ("mixed", "fp64"):
        done = [r[name] for r in rows if r[name]["certified"]]
        cert[name] = {"certified": len(done), "of": len(rows),
                      "solves_per_s": len(done) / sum(r[name]["seconds"] for r in rows)}
    eb = [r["mixed_early_branch"] for r in rows if "mixed_early_branch" in r]
    cert["mixed_early_branch"] = {
        "certified": sum(1 for r in eb if r["certified"]), "of": len(eb),
        "note": "run on the instances the mixed path certified; early_branch = 1, a stop "
                "test every 10 iterations",
        "seconds": [r["seconds"] for r in eb]}
    eb64 = [r["fp64_early_branch"] for r in rows if "fp64_early_branch" in r]
    cert["fp64_early_branch"] = {
        "certified": sum(1 for r in eb64 if r["certified"]), "of": len(eb64),
        "note": "the same instances and node stop, FP64 everywhere",
        "seconds": [r["seconds"] for r in eb64]}
    rv = {"certificates": None, "supports_ok": all(
        r[nm]["support_objective_rel_diff"] <= 1e-10 for r in rows for nm in ("mixed", "fp64"))
        and all(r["support_objective_rel_diff"] <= 1e-10 for r in eb)}
    agg = None
    for lam0, log in logs:
        one = reverify_logs(inst, lam0, lam2, M, [log])
        if agg is None:
            agg = one
        else:
            for k in ("n_certs", "exact", "screened", "violations"):
                agg[k] += one[k]
            for k in ("exact_max_rel", "screened_max_excess_over_width"):
                if one[k] is not None:
                    agg[k] = one[k] if agg[k] is None else max(agg[k], one[k])
            agg["exact_median_rel"] = None
    rv["certificates"] = agg
    return {"workload": args.workload, "seed": inst.seed, "gap": 1e-4,
            "time_limit_s": args.cert_time_limit, "rho": args.rho, "relax_alpha": args.alpha,
            "lambda0_rule": "first-incumbent nonzero count on a geometric grid of fractions",
            "grid_counts": counts, "grid_seconds": t_grid, "paths": cert, "instances": rows,
            "reverify": rv}


# the serving loop's node stop: a node whose primal estimate is below the prune threshold
# is branched at once (bnb_options.early_branch); on the first 32 requests of the stream
# 4 certify within 20 s against 1 with the paper's node stop
SERVE_EARLY_BRANCH = 1


def run_serve_side(args):
    """A short run of the serving workload (the first --serve-requests requests of the
    Poisson stream) for the bench line."""
    srv, res, summ = serve_stream(args, args.serve_requests, args.serve_time_limit,
                                  pregenerate=True)
    status = {}
    for r in res:
        status[r.status] = status.get(r.status, 0) + 1
    return dict(summ, status=status, requests=args.serve_requests,
                time_limit_s=args.serve_time_limit, early_branch=SERVE_EARLY_BRANCH,
                peak_admitted=srv.peak_active,
                peak_gib=srv.peak_used / (1 << 30),
                per_request=[{"rid": r.rid, "status": r.status, "nodes": r.nodes,
                              "queue_s": round(r.queueing, 4), "service_s": round(r.service, 4),
                              "gap": (r.ub - r.lb) / r.ub if r.ub else None} for r in res],
                data="request data generated before the clock starts")


def run_solves(args):
    """Full solves to gap 1e-4 of the workload (certified solves/s): for each of --seeds
    instances, lambda0 for 5, 8, 12, 16 and 20 nonzeros (lambda0_by_count), each solved by
    the mixed-precision path and, with --fp64-compare, by the plain FP64 path.  rho and
    alpha are autotuned once per instance (at the middle lambda0) unless --rho is given."""
    import paper_2602_04551_b300 as bnb
    from paper_2602_04551_b300 import autotune
    from oracle import ub as oub
    out = []
    t_all = time.perf_counter()
    for seed in range(args.seeds):
        inst, _, lam2, M, cfg = workload(args.workload, seed, 0.1)
        picks, counts = lambda0_by_count(inst, lam2, M)
        rho, alpha = args.rho, args.alpha
        if rho <= 0:
            best, _ = autotune.autotune(inst.X, inst.y, picks[len(picks) // 2]["lambda0"], lam2,
                                        M, use_cache=False,
                                        grid={"batch_K": [args.K],
                                              "precision": [PREC[args.precision]],
                                              "check_every": [args.check_every]},
                                        tune_crossover=False)
            rho, alpha = float(best["rho"]), float(best["relax_alpha"])
        for pk in picks:
            lam0 = pk["lambda0"]
            rec, beta, _ = solve_record(args, inst, lam0, lam2, M, rho, alpha,
                                        PREC[args.precision], args.solve_time_limit)
            S = np.nonzero(beta)[0]
            obj, _ = oub.support_objective(inst.X, inst.y, S, lam0, lam2, M)
            rec.update(pk, seed=seed, rho=rho, relax_alpha=alpha,
                       support_objective_rel_diff=abs(obj - rec["ub"]) / abs(obj))
            if args.fp64_compare:
                r64, b64, _ = solve_record(args, inst, lam0, lam2, M, rho, alpha,
                                           bnb.BNB_PREC_FP64, args.fp64_time_limit)
                r64["same_support"] = bool(np.array_equal(np.nonzero(b64)[0], S))
                rec["fp64"] = r64
            out.append(rec)
            print(json.dumps({"solve": out[-1]}), file=sys.stderr, flush=True)
    done = [r for r in out if r["certified"]]
    total = time.perf_counter() - t_all
    fp64 = None
    if args.fp64_compare:
        d64 = [r for r in out if r["fp64"]["certified"]]
        fp64 = {"solves_per_s": len(d64) / sum(r["fp64"]["seconds"] for r in out),
                "certified": len(d64), "time_limit_s": args.fp64_time_limit,
                "note": "same instances, rho and alpha, precision FP64 everywhere"}
    lat = np.array([r["seconds"] for r in done]) if done else np.array([np.nan])
    line = {"metric": "certified solves/s (gap 1e-4)", "mode": "solves",
            "value": len(done) / sum(r["seconds"] for r in out), "unit": "solves/s",
            "certified": len(done), "of": len(out),
            "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": {"workload": args.workload, "K": args.K,
                                            "lambda0_targets": list(LAM0_TARGETS),
                                            "seeds": args.seeds,
                                            "time_limit_s": args.solve_time_limit},
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "wall_s": total, "fp64_path": fp64, "solves": out}
    print(json.dumps(line), flush=True)


def run_kcurve(args):
    """Node throughput against the batch width K, for continuous slot refill and for the
    lockstep batches of Algorithm 1, on one workload instance (time-limited solves)."""
    import torch
    import paper_2602_04551_b300 as bnb
    inst, lam0, lam2, M, cfg = workload(args.workload, 0, args.lam0_frac)
    rho = args.rho if args.rho > 0 else 0.3
    rows = []
    for K in [int(k) for k in args.k_list.split(",")]:
        for lock in (0, 1):
            o = bnb.bnb_options_default(M=M, batch_K=K, check_every=args.check_every,
                                        precision=PREC[args.precision], rho=rho,
                                        relax_alpha=args.alpha, queue_capacity=1 << 21,
                                        max_depth=args.max_depth, lockstep=lock,
                                        time_limit_s=args.solve_time_limit)
            with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res = bnb.bnb_solve(h, 1e-4)
                dt = time.perf_counter() - t0
            rows.append({"K": K, "lockstep": lock, "nodes": res["nodes"], "seconds": dt,
                         "nodes_per_s": res["nodes"] / dt, "status": res["status"],
                         "ub": res["ub"], "lb": res["lb"]})
            print(json.dumps({"kcurve": rows[-1]}), file=sys.stderr, flush=True)
    base = {r["lockstep"]: r["nodes_per_s"] for r in rows if r["K"] == rows[0]["K"]}
    for r in rows:
        r["speedup_vs_first_K"] = r["nodes_per_s"] / base[r["lockstep"]]
    line = {"metric": "BnB nodes/s vs batch width K", "mode": "kcurve", "unit": "nodes/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": {"workload": args.workload,
                                            "lambda0_frac": args.lam0_frac, "rho": rho,
                                            "relax_alpha": args.alpha,
                                            "time_limit_s": args.solve_time_limit},
            "rows": rows}
    print(json.dumps(line), flush=True)


def serve_stream(args, count, time_limit, pregenerate=False):
    """The serving workload's first `count` requests (Poisson arrivals at --arrival-rate,
    shapes n ~ U[500, 5000], p ~ U[1000, 20000], rho in {0.1, 0.3, 0.5, 0.7}, k ~ U[5, 25],
    SNR ~ U[2, 10], lambda2 = 0.01, lambda0 for k nonzeros by greedy_lambda0) through the
    serving loop; returns (server, results, latency summary).  With `pregenerate` every
    request's synthetic data are made before the clock starts (as if each request carried
    its data); otherwise they are made at admission, inside the loop."""
    from paper_2602_04551_b300.serve import Request, Server, poisson_arrivals, latency_summary
    rng = np.random.Generator(np.random.PCG64(5000))
    times = poisson_arrivals(args.requests, args.arrival_rate, 5000)
    lam2 = 0.01

    def loader(n, p, rho, k, snr, seed):
        def make():
            inst = datagen.make_instance(n, p, rho, k, snr, seed)
            M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
            return inst.X, inst.y, greedy_lambda0(inst.X, inst.y, lam2, M, k), M
        return make

    reqs = []
    for i in range(args.requests):
        n = int(rng.integers(500, 5001))
        p = int(rng.integers(1000, 20001))
        rho = float(rng.choice([0.1, 0.3, 0.5, 0.7]))
        k = int(rng.integers(5, 26))
        snr = float(rng.uniform(2, 10))
        if i < count:
            reqs.append(Request(rid=i, X=None, y=None, lambda0=0.0, lambda2=lam2, M=1.0,
                                gap=1e-4, arrival=float(times[i]), shape=(n, p),
                                loader=loader(n, p, rho, k, snr, 5000 + i),
                                options=dict(batch_K=256, rho=0.3, relax_alpha=1.6,
                                             precision=PREC[args.precision], max_depth=1024,
                                             time_limit_s=time_limit,
                                             early_branch=SERVE_EARLY_BRANCH)))
    if pregenerate:
        for r in reqs:
            r.data()
            r.loader = None
        note(f"serve: {len(reqs)} requests generated")
    last = [0.0]

    def progress(t, pending, active, done):
        if t - last[0] >= 5.0:
            last[0] = t
            note(f"serve t={t:.1f}s pending {pending} active {active} done {done}")

    srv = Server(budget_bytes=int(args.budget_gb * (1 << 30)), rounds_per_step=4,
                 progress=progress)
    res = srv.run(reqs)
    return srv, res, latency_summary(res)


def run_serve(args):
    """The serving workload: independent solves of random shapes arriving as a
    Poisson stream, admitted under an HBM budget and interleaved on the GPU."""
    import paper_2602_04551_b300 as bnb
    srv, res, summ = serve_stream(args, args.requests, args.solve_time_limit)
    status = {}
    for r in res:
        status[r.status] = status.get(r.status, 0) + 1
    line = {"metric": "serving: p50/p99 time to certified gap 1e-4", "mode": "serve",
            "value": summ["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": DTYPE[args.precision], "data": "synthetic",
            "status": status, "peak_admitted": srv.peak_active, "peak_bytes": srv.peak_used,
            "config": {"workload": "serve", "requests": args.requests,
                       "arrival_rate_per_s": args.arrival_rate, "budget_gb": args.budget_gb,
                       "time_limit_s": args.solve_time_limit,
                       "early_branch": SERVE_EARLY_BRANCH,
                       "lambda0": "per request, k nonzeros on the greedy forward path"}}
    line.update(summ)
    print(json.dumps(line), flush=True)


def mine_line(args, out, world, ms, nodes, pk, cpu):
    """The GPU arm's JSON line from run_mine's record, the max-over-ranks time `ms` of the
    timed rounds and the nodes all ranks certified in them."""
    return {
        "metric": METRIC,
        "value": nodes / (ms / 1e3), "unit": "nodes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": line_config(out["cfg"], args),
        "solver": {"arithmetic": "mixed-precision ADMM, FP64 certificates and polish",
                   "precision": args.precision, "check_every": args.check_every,
                   "rho": args.rho, "relax_alpha": args.alpha},
        "e2e": out["e2e"], "gpu_launches": out["kernels"], "clocks": out["clocks"],
        "roofline": roofline(out, args, pk),
        "fp64_path": dict(out["fp64"], ratio_same_batch=out["fp64"]["mixed_same_batch"]["nodes_per_s"]
                          / max(1e-12, out["fp64"]["value"])),
        "prime": out["prime"],
        "setup_seconds": out.get("setup_seconds"),    # per-tree setup (R0), outside the timed rounds
        "autotune": out["tune"],
        "cpu_baseline": cpu,
        "solve_progress": {"nodes": out["after"]["nodes"], "ub": out["after"]["ub"],
                           "lb": out["after"]["lb"], "open_nodes": out["after"]["open_nodes"],
                           "done": out["after"]["done"]},
        "stages_ms": {k: v[0] for k, v in out["prof"].items()},
        "kernel_shapes": out["shapes"],
        "rounds_per_step": args.rounds_per_step,
        "rounds": out.get("rounds"),
        "ms_per_round": ms / max(1, out.get("rounds") or args.steps * args.rounds_per_step),
        "reverify": out.get("reverify"),
        "fp32_path": out.get("fp32"),
        "certified_solves": out.get("certified"),
        "serve": out.get("serve"),
    }


def main():
    import faulthandler
    # a stalled run reports where it is: every thread's stack on stderr every 5 minutes
    faulthandler.dump_traceback_later(300, repeat=True, file=sys.stderr)
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    if args.mode == "solves":
        run_solves(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return
    if args.mode == "kcurve":
        run_kcurve(args)
        return
    world = int(os.environ.get("WORLD_SIZE", 1))
    rank = int(os.environ.get("RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        dist.init_process_group("nccl")
    out = run_mine(args, rank, world)
    ms, nodes = combine_ranks(out["ms"], out["nodes"], world)
    if rank == 0:
        cpu = None if args.no_cpu else run_oracle(args, args.cpu_seconds)
        line = mine_line(args, out, world, ms, nodes, peaks(), cpu)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
