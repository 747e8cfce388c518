#!/usr/bin/env python
"""Benchmark: certified branch-and-bound nodes per second on one B300.

Workload (default "c2"): n=1000, p=5000, Toeplitz rho=0.3, k=10 true ones,
SNR=5, lambda2=1e-3, M = 1.5 ||ridge on the true support||_inf, lambda0 from a
sweep relative to max_j (X_j^T y)^2 / (2(||X_j||^2 + 2 lambda2)), node-batch
width K=512, target gap 1e-4, FP32 ADMM with FP64 certificates.

A "step" is one device round of the solve: refill free slots best-first,
check_every ADMM iterations over all K slots, FP64 certificates of the nodes
that stopped, branch pick + batched upper bound, prune/branch into the pool.
  value     nodes certified per second over the timed steps (device time, CUDA
            events on the solve's stream; L2 flushed with a 256 MiB write
            before every step, outside the timed interval)
  e2e       nodes certified per second through bnb_relax_batch with host
            buffers: each step uploads K nodes (fixings + warm starts) from
            pinned memory and reads back bounds, beta, z
  fp64_path the same rounds on the plain FP64 GPU path (the comparator)
  roofline  the dominant kernel of a profiled round (CUDA events per launch)
  cpu_baseline the FP64 oracle's node solves on the host cores, bounded sample

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
    ap.add_argument("--serve-lam0-frac", type=float, default=0.3,
                    help="serve mode: lambda0 = frac x max_j (X_j^T y)^2 / (2 (||X_j||^2 + 2 lambda2))")
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
    ap.add_argument("--u-shape", type=int, default=0, choices=[0, 1, 2],
                    help="U' = H W'^T: 0 measured at setup, 1 cluster-reduced, 2 CTA pairs split-K")
    ap.add_argument("--mv-crossover", type=int, default=-1,
                    help="narrow-form crossover (-1 default; 0 = tensor-core form only: graphs "
                         "without conditional nodes, which ncu can profile kernel by kernel)")
    ap.add_argument("--k-list", default="1,4,16,64,256,512",
                    help="kcurve mode: batch widths; each solve runs --solve-time-limit seconds")
    ap.add_argument("--lam0-frac", type=float, default=0.02)
    ap.add_argument("--K", type=int, default=512)
    ap.add_argument("--check-every", type=int, default=10)
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
    return ap.parse_args()


METRIC = "certified BnB nodes/s"        # both arms report this metric on the same config


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
                                        tune_crossover=False)
        args.rho = float(best["rho"])
        args.alpha = float(best.get("relax_alpha", 1.0))
        tune = {"chosen": best, "seconds": entry["seconds"],
                "trials": [{k: t[k] for k in ("rho", "nodes_per_s", "mean_iters", "lb_mean")}
                           for t in entry["trials"]]}
    s = torch.cuda.Stream()
    opt = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every,
                                  precision=PREC[args.precision], device=dev, stream=s.cuda_stream,
                                  queue_capacity=1 << 21, time_limit_s=1e9, rho=args.rho,
                                  relax_alpha=args.alpha, mv_crossover=args.mv_crossover,
                                  fused_shape=args.fused_shape, u_shape=args.u_shape)
    h = bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    gap = 1e-4
    bnb.bnb_solve_start(h, gap)
    # priming (untimed): grow the tree until the slots are busy and a batch's worth of
    # nodes has been certified, so that the timed rounds measure the steady state of the
    # solve (slots retiring and refilling) rather than its first nodes
    t0 = time.time()
    prime_rounds = 0
    while True:
        bnb.bnb_solve_launch(h, 20)
        prime_rounds += 20
        pr = bnb.bnb_solve_poll(h)
        busy = pr["active_slots"] >= 0.9 * args.K and pr["nodes"] >= args.K
        if pr["done"] or busy or time.time() - t0 > args.prime_seconds:
            break
    clk = Clocks(dev)            # sampling spans the warm-up and the timed steps
    time.sleep(0.3)
    with torch.cuda.stream(s):
        for _ in range(args.warmup):
            bnb.bnb_solve_launch(h, 1)
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
            bnb.bnb_solve_launch(h, 1)
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
                                          "u_split")}
    out = dict(ms=ms, nodes=nodes, prof=prof, prog=prog, clocks=clocks, cfg=cfg, tune=tune,
               setup_seconds=stats.get("setup_seconds"),
               kernels=kernels_per_round * args.steps, after=after, res=res, shapes=shapes,
               prime={"rounds": prime_rounds, "seconds": time.time() - t0,
                      "active_slots": before["active_slots"], "open_nodes": before["open_nodes"]})
    if rank == 0:
        out["e2e"] = run_e2e(args, inst, lam0, lam2, M, dev)
        out["fp64"] = run_fp64(args, inst, lam0, lam2, M, dev)
    return out


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
        "blocks": _PAIR_NT, "sources": "cbfa68214a12d6bb", "bytes": 45.185024e6 + 0.526592e6,
        "note": _NOTE.format(k="tc_gemm_pair_kernel<176, 3, TcEpiAdmmPair<176, 0>, 12>",
                             f="fused_pair_untransposed_c2_K512_tc3.md")},
    ("gemm_xtu_prox", "c2", 512, "tc3", 64, False, False, False): {
        "blocks": _PERSIST, "sources": "445fd8171ad98c9b", "bytes": 45.183232e6 + 0.606976e6,
        "note": _NOTE.format(k="tc_gemm_persist_kernel<64, 3, TcEpiAdmm<64, 0>, 12>",
                             f="fused_xtu_prox_shapes_c2_K512_tc3.md")},
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
        if "bf16_tflops_sustained" in pk:
            peak = float(pk["bf16_tflops_sustained"])
            note = "measured sustained dense BF16 (MEASURED_PEAKS.json)"
        else:
            peak = 1400.0
            note = "fallback: 1.4 PFLOP/s sustained dense BF16 (no measured peaks file)"
        mult = {"tc3": 3.0, "bf16x2": 2.0}.get(args.precision, 1.0)
        r.update(bound="tensor", peak=peak, frac=ach / peak, achieved_hw=ach * mult,
                 frac_hw=ach * mult / peak, peak_note=note)
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


def run_solves(args):
    """Full solves to gap 1e-4 of the workload over a lambda0 sweep (certified solves/s)."""
    import torch
    import paper_2602_04551_b300 as bnb
    from paper_2602_04551_b300 import autotune
    out = []
    t_all = time.perf_counter()
    jobs = [(float(f), sd) for f in args.lam0_fracs.split(",") for sd in range(args.seeds)]
    for frac, seed in jobs:
        inst, lam0, lam2, M, cfg = workload(args.workload, seed, frac)
        best, _ = autotune.autotune(inst.X, inst.y, lam0, lam2, M, use_cache=False,
                                    grid={"batch_K": [args.K], "precision": [PREC[args.precision]],
                                          "check_every": [args.check_every]})
        o = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every,
                                    precision=PREC[args.precision], rho=best["rho"],
                                    relax_alpha=best["relax_alpha"], queue_capacity=1 << 21,
                                    mv_crossover=int(best.get("mv_crossover", -1)),
                                    max_depth=args.max_depth, time_limit_s=args.solve_time_limit)
        with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o) as h:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res = bnb.bnb_solve(h, 1e-4)
            dt = time.perf_counter() - t0
            st = bnb.bnb_get_stats(h)
            dh, sh = bnb.bnb_get_histograms(h, args.max_depth + 1, 202)
        rec = {"lambda0_frac": frac, "seed": seed, "lambda0": lam0, "seconds": dt,
               "setup_seconds": st.get("setup_seconds"),
               "status": res["status"], "nodes": res["nodes"],
               "nnz": int(np.count_nonzero(res["beta"])), "ub": res["ub"], "lb": res["lb"],
               "gap": (res["ub"] - res["lb"]) / res["ub"], "nodes_per_s": res["nodes"] / dt,
               "rho": best["rho"], "relax_alpha": best["relax_alpha"],
               "mv_crossover": best.get("mv_crossover"), "max_depth": st["max_depth"],
               # solved nodes by depth 0..40 (+ deeper) and by rounded-support size 0..200 (+ larger)
               "depth_hist": [int(x) for x in dh[:41]] + [int(dh[41:].sum())],
               "support_hist": [int(x) for x in sh[:201]] + [int(sh[201:].sum())]}
        if args.fp64_compare:
            o64 = bnb.bnb_options_default(M=M, batch_K=args.K, check_every=args.check_every,
                                          precision=0, rho=best["rho"],
                                          relax_alpha=best["relax_alpha"], queue_capacity=1 << 21,
                                          max_depth=args.max_depth,
                                          time_limit_s=args.fp64_time_limit)
            with bnb.bnb_create(inst.X, inst.y, lam0, lam2, o64) as h:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r64 = bnb.bnb_solve(h, 1e-4)
                d64 = time.perf_counter() - t0
            rec["fp64"] = {"seconds": d64, "status": r64["status"], "nodes": r64["nodes"],
                           "ub": r64["ub"], "lb": r64["lb"], "nodes_per_s": r64["nodes"] / d64,
                           "same_support": bool(np.array_equal(np.nonzero(r64["beta"])[0],
                                                               np.nonzero(res["beta"])[0]))}
        out.append(rec)
        print(json.dumps({"solve": out[-1]}), file=sys.stderr, flush=True)
    done = [r for r in out if r["status"] in ("optimal", "gap")]
    total = time.perf_counter() - t_all
    fp64 = None
    if args.fp64_compare:
        d64 = [r for r in out if r["fp64"]["status"] in ("optimal", "gap")]
        fp64 = {"solves_per_s": len(d64) / sum(r["fp64"]["seconds"] for r in out),
                "time_limit_s": args.fp64_time_limit,
                "note": "same instances, autotuned rho and K, precision FP64 everywhere"}
    lat = np.array([r["seconds"] for r in done]) if done else np.array([np.nan])
    line = {"metric": "certified solves/s (gap 1e-4)", "mode": "solves",
            "value": len(done) / sum(r["seconds"] for r in out), "unit": "solves/s",
            "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE[args.precision],
            "data": "synthetic", "config": {"workload": args.workload, "K": args.K,
                                            "lambda0_fracs": args.lam0_fracs, "seeds": args.seeds,
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


def run_serve(args):
    """The serving workload: independent solves of random shapes arriving as a
    Poisson stream, admitted under an HBM budget and interleaved on the GPU."""
    import paper_2602_04551_b300 as bnb
    from paper_2602_04551_b300.serve import Request, Server, poisson_arrivals, latency_summary
    rng = np.random.Generator(np.random.PCG64(5000))
    times = poisson_arrivals(args.requests, args.arrival_rate, 5000)
    reqs = []
    lam2 = 0.01

    def loader(n, p, rho, k, snr, seed):
        def make():
            inst = datagen.make_instance(n, p, rho, k, snr, seed)
            M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
            lam0 = args.serve_lam0_frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
            return inst.X, inst.y, lam0, M
        return make

    for i in range(args.requests):
        n = int(rng.integers(500, 5001))
        p = int(rng.integers(1000, 20001))
        rho = float(rng.choice([0.1, 0.3, 0.5, 0.7]))
        k = int(rng.integers(5, 26))
        snr = float(rng.uniform(2, 10))
        reqs.append(Request(rid=i, X=None, y=None, lambda0=0.0, lambda2=lam2, M=1.0, gap=1e-4,
                            arrival=float(times[i]), shape=(n, p),
                            loader=loader(n, p, rho, k, snr, 5000 + i),
                            options=dict(batch_K=256, rho=0.3, relax_alpha=1.6,
                                         precision=PREC[args.precision],
                                         time_limit_s=args.solve_time_limit)))
    srv = Server(budget_bytes=int(args.budget_gb * (1 << 30)), rounds_per_step=4)
    res = srv.run(reqs)
    summ = latency_summary(res)
    status = {}
    for r in res:
        status[r.status] = status.get(r.status, 0) + 1
    # a sample of requests re-solved alone: same support and objective
    check = []
    for r in res[: min(4, len(res))]:
        q = reqs[r.rid]
        X, y, lam0, M = q.loader()
        o = bnb.bnb_options_default(M=M, batch_K=256, rho=0.3, relax_alpha=1.6,
                                    precision=PREC[args.precision],
                                    time_limit_s=args.solve_time_limit, queue_capacity=1 << 18,
                                    warm_capacity=1 << 14)
        with bnb.bnb_create(X, y, lam0, q.lambda2, o) as h:
            a = bnb.bnb_solve(h, q.gap)
        check.append({"rid": r.rid, "same_support": bool(np.array_equal(np.nonzero(a["beta"])[0],
                                                                          np.nonzero(r.beta)[0])),
                      "ub_rel_diff": abs(a["ub"] - r.ub) / abs(a["ub"])})
    line = {"metric": "serving: p50/p99 time to certified gap 1e-4", "mode": "serve",
            "value": summ["solves_per_s"], "unit": "solves/s", "p50_s": summ["p50_s"],
            "p99_s": summ["p99_s"], "mean_s": summ["mean_s"], "makespan_s": summ["makespan_s"],
            "solves": summ["solves"], "status": status, "nodes": summ["nodes"],
            "peak_admitted": srv.peak_active, "peak_bytes": srv.peak_used, "n_gpus": 1,
            "higher_is_better": True, "dtype": DTYPE[args.precision], "data": "synthetic",
            "config": {"workload": "serve", "requests": args.requests,
                       "arrival_rate_per_s": args.arrival_rate, "budget_gb": args.budget_gb,
                       "time_limit_s": args.solve_time_limit,
                       "lambda0_frac": args.serve_lam0_frac},
            "alone_vs_mix": check}
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
    }


def main():
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
