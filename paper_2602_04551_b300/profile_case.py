"""Profiling harness: a solve primed to steady state, then a few rounds, for ncu.

    python -m paper_2602_04551_b300.profile_case --workload c4 --rounds 3

Used for the ncu captures of the top kernels (small enough that the capture ends in
a minute or two; the c4 shape keeps X and the node state larger than the L2 cache).
ncu does not profile the kernels of a CUDA graph that contains conditional nodes, so
captures run with --mv-crossover 0 (wide rounds: the tensor-core form, no conditional
node) or --no-graphs (the narrow matrix-vector form launched directly).
"""
import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="c4")
    ap.add_argument("--lam0-frac", type=float, default=0.02)
    ap.add_argument("--K", type=int, default=512)
    ap.add_argument("--rho", type=float, default=0.3)
    ap.add_argument("--precision", type=int, default=3)
    ap.add_argument("--rounds", type=int, default=3)
    ap.add_argument("--prime-seconds", type=float, default=30.0)
    ap.add_argument("--mv-crossover", type=int, default=-1)
    ap.add_argument("--fused-shape", type=int, default=0, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--u-shape", type=int, default=0, choices=[0, 1, 2, 3])
    ap.add_argument("--fused-width", type=int, default=0)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--tma-stream", action="store_true",
                    help="time the TMA operand ring alone (bnb_diag_tma_stream) over CTA "
                         "counts and pass counts, one JSON line per case, and exit")
    return ap


def tma_stream_table() -> None:
    """The operand ring of the fused product's pair tile alone (A hi/lo 128 rows, B hi/lo
    88 rows per CTA, three stages): one pass of 16 K steps (the c2 main loop: 864 KB per
    CTA) and eight passes (the steady rate), on 30 to 148 SMs."""
    import json
    import paper_2602_04551_b300 as bnb
    for ctas, stages, b_rows, reps in [(120, 3, 88, 1), (120, 3, 88, 8), (148, 3, 88, 8),
                                       (60, 3, 88, 8), (30, 3, 88, 8), (120, 4, 64, 8)]:
        r = bnb.bnb_diag_tma_stream(ctas, stages, b_rows, reps, launches=5)
        print(json.dumps(dict(ctas=ctas, stages=stages, b_rows=b_rows, reps=reps,
                              kb_per_cta=r["bytes"] / ctas / 1024, **r)), flush=True)


def main():
    import torch
    import datagen
    import paper_2602_04551_b300 as bnb
    from paper_2602_04551_b300 import autotune

    a = parser().parse_args()
    if a.tma_stream:
        tma_stream_table()
        return
    c = datagen.CONFIGS[a.workload]
    inst = datagen.config_instance(a.workload, 0)
    M = datagen.big_m(inst.X, inst.y, inst.support_true, c["lam2"])
    lam0 = a.lam0_frac * datagen.lambda0_scale(inst.X, inst.y, c["lam2"])
    o = bnb.bnb_options_default(M=M, batch_K=a.K, rho=a.rho, precision=a.precision,
                                queue_capacity=1 << 20, time_limit_s=1e9,
                                mv_crossover=a.mv_crossover, use_graphs=0 if a.no_graphs else 1,
                                fused_shape=a.fused_shape, u_shape=a.u_shape,
                                fused_width=a.fused_width)
    with bnb.bnb_create(inst.X, inst.y, lam0, c["lam2"], o) as h:
        bnb.bnb_solve_start(h, 1e-4)
        t0 = time.time()
        while True:
            bnb.bnb_solve_launch(h, 10)
            pr = bnb.bnb_solve_poll(h)
            if pr["done"] or autotune.steady(pr, a.K) or time.time() - t0 > a.prime_seconds:
                break
        torch.cuda.nvtx.range_push("profiled_rounds")
        bnb.bnb_solve_launch(h, a.rounds)
        pr = bnb.bnb_solve_poll(h)
        torch.cuda.nvtx.range_pop()
        print({k: pr[k] for k in ("nodes", "active_slots", "open_nodes", "ub", "lb")})
        bnb.bnb_solve_finish(h)


if __name__ == "__main__":
    main()
