"""Host logic of bench.py (no GPU): the roofline figures of the dominant kernel and the
provenance rule of its DRAM traffic (reported only while the captured kernel's source is
unchanged)."""
import importlib.util
import os
import shutil
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    argv = sys.argv
    sys.argv = ["bench.py"]
    try:
        spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def _out(key, ms_fused=0.036, ms_u=0.028, active=491):
    _, workload, K, prec, width, mc, pairs, transposed = key
    return {"prof": {"gemm_xtu_prox": [ms_fused, 10], "gemm_xw": [ms_u, 10], "certificate": [0.08, 1]},
            "cfg": {"n": 1000, "p": 5000}, "prog": {"active_slots": active},
            "shapes": {"fused_tile_width": width, "fused_clusters": 74 if mc else 0,
                       "fused_pairs": 74 if pairs else 0, "fused_transposed": int(transposed)}}


def _args(key):
    _, workload, K, prec, *_ = key
    return types.SimpleNamespace(workload=workload, K=K, precision=prec)


def test_roofline_figures(bench):
    key = next(iter(bench.TRAFFIC))
    r = bench.roofline(_out(key), _args(key), {"bf16_tflops_sustained": 1390.1})
    assert r["kernel"] == "gemm_xtu_prox"
    flops = 2.0 * 1000 * 5000 * 491
    assert r["flops_per_launch"] == flops
    assert r["achieved"] == pytest.approx(flops / 0.036e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1390.1)
    assert r["achieved_hw"] == pytest.approx(3 * r["achieved"])
    assert r["bound"] == "tensor" and r["peak"] == 1390.1
    assert r["share_of_round"] == pytest.approx(0.36 / (0.36 + 0.28 + 0.08))
    # the committed capture matches the committed kernel source
    assert r["traffic"] == bench.TRAFFIC[key]["bytes"]


def test_roofline_hbm_view_of_the_fused_product(bench):
    """The fused product's compulsory bytes (X and U' as BF16 pairs, 21 bytes of node state
    per active element) over its launch time, against the measured copy bandwidth."""
    key = next(iter(bench.TRAFFIC))
    r = bench.roofline(_out(key), _args(key), {"bf16_tflops_sustained": 1390.1, "hbm_gbs": 6480.8})
    n, p, a = 1000, 5000, 491
    nbytes = 4.0 * n * p + 4.0 * n * a + 21.0 * p * a
    hv = r["hbm_view"]
    assert hv["algorithmic_bytes"] == nbytes
    assert hv["achieved_gbs"] == pytest.approx(nbytes / 0.036e-3 / 1e9)
    assert hv["frac"] == pytest.approx(hv["achieved_gbs"] / 6480.8)
    assert "hbm_view" not in bench.roofline(_out(key), _args(key), {"bf16_tflops_sustained": 1.0})


def test_fallback_peak_is_labelled(bench):
    key = next(iter(bench.TRAFFIC))
    r = bench.roofline(_out(key), _args(key), {})
    assert r["peak"] == 1400.0 and "fallback" in r["peak_note"]


def test_traffic_needs_the_captured_shape(bench):
    key = next(iter(bench.TRAFFIC))
    other = key[:4] + (999,) + key[5:]
    r = bench.roofline(_out(other), _args(other), {"bf16_tflops_sustained": 1390.1})
    assert r["traffic"] is None


def test_traffic_dropped_when_the_kernel_source_changes(bench, tmp_path, monkeypatch):
    key = next(iter(bench.TRAFFIC))
    csrc = tmp_path / "paper_2602_04551_b300" / "csrc"
    shutil.copytree(os.path.join(ROOT, "paper_2602_04551_b300", "csrc"), csrc)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r = bench.roofline(_out(key), _args(key), {"bf16_tflops_sustained": 1390.1})
    assert r["traffic"] is not None                      # an identical copy still matches
    f, start, _ = bench.TRAFFIC[key]["blocks"][0]
    text = (csrc / f).read_text()
    i = text.index(start)
    (csrc / f).write_text(text[:i] + start + " /* edited */" + text[i + len(start):])
    r = bench.roofline(_out(key), _args(key), {"bf16_tflops_sustained": 1390.1})
    assert r["traffic"] is None


def test_reference_arm_line(bench, monkeypatch, capsys):
    """The reference arm (the oracle on the host cores) prints one contract line with the
    GPU arm's metric, unit and config; ranks other than 0 print nothing."""
    import json
    calls = []
    monkeypatch.setattr(bench, "oracle_setup", lambda *a, **k: "state")
    monkeypatch.setattr(bench, "oracle_nodes", lambda st, sec: calls.append(sec) or (3, 0.5))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"])
    args = bench.parse()
    monkeypatch.setenv("RANK", "1")
    bench.reference_arm(args)
    assert capsys.readouterr().out == "" and not calls
    monkeypatch.setenv("RANK", "0")
    bench.reference_arm(args)
    line = json.loads(capsys.readouterr().out.strip())
    assert len(calls) == 5
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "nodes/s" and line["higher_is_better"] is True
    assert line["value"] == pytest.approx(3 * 2 / (0.5 * 2))
    _, _, _, _, cfg = bench.workload(args.workload, 0, args.lam0_frac)
    assert line["config"] == bench.line_config(cfg, args)
    assert line["config"]["workload"] == "c2" and line["config"]["K"] == 512
    for key in ("n_gpus", "steps", "warmup", "ms_per_step", "scaling", "vs_baseline", "dtype", "data"):
        assert key in line
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert 1 <= line["cpu_baseline"]["cores"] <= os.cpu_count()
    assert line["cpu_baseline"]["cores"] == bench.oracle_threads()
    assert line["e2e"] == {"value": line["value"], "unit": "nodes/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_gpu_arm_line_has_the_contract_keys(bench, monkeypatch):
    """The GPU arm's line, built from a record shaped like the one the timed run returns:
    every contract key, the same metric and config as the reference arm, value = nodes
    certified over the timed seconds."""
    import json
    key = next(iter(bench.TRAFFIC))
    monkeypatch.setattr(sys, "argv", ["bench.py", "--steps", "80", "--warmup", "3"])
    args = bench.parse()
    args.rho, args.alpha = 0.2, 1.6                  # as the autotuner sets them
    _, _, _, _, cfg = bench.workload(args.workload, 0, args.lam0_frac)
    out = _out((key[0], args.workload, args.K, args.precision) + key[4:])
    out["cfg"] = cfg
    out.update(
        kernels=40 * 80, tune={"rho": 0.2, "relax_alpha": 1.6},
        clocks={"sm_mhz": 2032, "sm_max_mhz": 2032, "reasons": [], "samples": 50},
        e2e={"value": 28000.0, "unit": "nodes/s", "h2d_bytes_per_step": 23 << 20,
             "d2h_bytes_per_step": 20 << 20, "call": "bnb_relax_batch (host buffers)"},
        fp64={"value": 300.0, "unit": "nodes/s", "mixed_same_batch": {"nodes_per_s": 36000.0},
              "fp64": {"nodes_per_s": 300.0}, "bound_error": {"max_rel": 3e-5}},
        prime={"rounds": 200, "seconds": 2.0, "active_slots": 500, "open_nodes": 9000},
        after={"nodes": 50000, "ub": 1.0, "lb": 0.99, "open_nodes": 20000, "done": 0},
        shapes={"fused_tile_width": key[4], "fused_clusters": 0, "fused_pairs": 74,
                "fused_transposed": 0, "xw_tile_width": 128, "xw_cluster": 4, "u_split": 0})
    cpu = {"value": 3.0, "unit": "nodes/s", "cores": 16, "kind": "oracle", "sample": "s"}
    line = json.loads(json.dumps(bench.mine_line(args, out, 1, 64.0, 2688, {"bf16_tflops_sustained": 1390.1},
                                                 cpu)))
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks",
              "roofline", "cpu_baseline"):
        assert k in line, k
    assert line["metric"] == bench.METRIC and line["unit"] == "nodes/s"
    assert line["config"] == bench.line_config(cfg, args)
    assert line["value"] == pytest.approx(2688 / 0.064)
    assert line["ms_per_step"] == pytest.approx(64.0 / 80)
    assert set(line["roofline"]) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
    assert set(line["e2e"]) >= {"value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"}
    assert line["fp64_path"]["ratio_same_batch"] == pytest.approx(120.0)
    assert line["solver"]["rho"] == 0.2
    assert line["setup_seconds"] is None             # absent from the fake record
    out["setup_seconds"] = 0.9
    assert bench.mine_line(args, out, 1, 64.0, 2688, {}, cpu)["setup_seconds"] == 0.9


def test_burst_peak_when_the_timed_region_ran_at_full_clock(bench):
    """At the maximum SM clock with no power cap the kernel is compared with the burst
    peak; otherwise with the sustained one; the other fraction is reported beside it."""
    key = next(iter(bench.TRAFFIC))
    pk = {"bf16_tflops": 1790.8, "bf16_tflops_sustained": 1386.4}
    out = _out(key)
    out["clocks"] = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": []}
    r = bench.roofline(out, _args(key), pk)
    assert r["peak"] == 1790.8 and r["peak_kind"] == "burst"
    assert r["frac_vs_sustained"] == pytest.approx(r["achieved"] / 1386.4)
    out["clocks"] = {"sm_mhz": 2032.0, "sm_max_mhz": 2032.0, "reasons": ["sw_power_cap"]}
    r = bench.roofline(out, _args(key), pk)
    assert r["peak"] == 1386.4 and r["peak_kind"] == "sustained"
    out["clocks"] = {"sm_mhz": 1600.0, "sm_max_mhz": 2032.0, "reasons": []}
    assert bench.roofline(out, _args(key), pk)["peak_kind"] == "sustained"


def test_lambda0_pick_rule(bench):
    grid = [1.0, 0.5, 0.25, 0.125, 0.0625]
    counts = [3, 5, 5, 8, 13]
    picks = bench.pick_lambda0(counts, grid, (5, 8, 12, 20, 1))
    fr = [p["lambda0_frac"] for p in picks]
    assert fr[0] == pytest.approx((0.5 * 0.25) ** 0.5)     # midpoint of the points giving 5
    assert fr[1] == 0.125                                   # the one point giving 8
    assert fr[2] == 0.0625                                  # nearest count to 12 is 13
    assert fr[3] == 0.0625
    assert fr[4] == 1.0                                     # nearest to 1 is 3 (largest lambda0)


def test_greedy_lambda0_orthonormal_design(bench):
    """Orthonormal columns: each forward step's drop is c_j^2 / (2 (1 + 2 lam2)) of the
    untouched coefficient (box loose), so the returned lambda0 lies strictly between the
    k-th and (k+1)-th largest of them."""
    import numpy as np
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 12)))
    beta = np.array([3.0, -2.6, 2.2, 1.9, -1.5, 1.2, 0.9, 0.7, 0.5, 0.3, 0.2, 0.1])
    y = Q @ beta
    lam2, M = 0.01, 10.0
    drops = np.sort((Q.T @ y) ** 2 / (2 * (1 + 2 * lam2)))[::-1]
    for k in (1, 4, 7):
        lam0 = bench.greedy_lambda0(Q, y, lam2, M, k)
        assert drops[k] < lam0 < drops[k - 1]


def test_reverify_logs_counts_and_flags(bench):
    """reverify_logs against the oracle on a fabricated log: an exact bound equal to D(r),
    a screened bound inside its interval, and one claiming more than D(r) (a violation)."""
    import numpy as np
    import datagen
    from oracle import relax
    inst = datagen.config_instance("c1", 0)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.05 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    rng = np.random.default_rng(2)
    fix = datagen.random_fixings(inst.p, 3, rng, 5)
    r = inst.y[None, :] * 0.9 + rng.normal(0, 0.05, (3, inst.n))
    d = np.array([relax.dual_value(inst.X, inst.y, r[k], fix[k], lam0, lam2, M) for k in range(3)])
    log = {"count": 3, "fix": fix, "r": r, "lb": np.array([d[0], d[1] - 0.01, d[2] + 0.01]),
           "exact": np.array([1.0, 0.0, 0.0]), "width": np.array([0.0, 0.02, 0.02])}
    out = bench.reverify_logs(inst, lam0, lam2, M, [log])
    assert out["n_certs"] == 3 and out["exact"] == 1 and out["screened"] == 2
    assert out["violations"] == 1
    assert out["exact_max_rel"] <= 1e-15
    assert out["screened_max_rel_below_exact"] == pytest.approx(0.01 / max(1.0, abs(d[1])))


def test_certified_side_times_the_early_branch_stop_where_the_mixed_path_certified(bench, monkeypatch):
    """run_certified (the bench line's certified_solves): every target lambda0 is solved by
    the mixed and the FP64 paths; where the mixed path certified, once more with the
    early-branch node stop and a stop test every 10 iterations, with its speed-ups; the
    instances the mixed path did not certify get no third solve."""
    import numpy as np
    from oracle import ub as oub
    calls = []
    picks = [{"target_nnz": 5, "lambda0": 0.5}, {"target_nnz": 12, "lambda0": 0.05}]
    monkeypatch.setattr(bench, "lambda0_by_count", lambda inst, lam2, M: (picks, [5, 12]))

    def fake_solve(args, inst, lam0, lam2, M, rho, alpha, prec, tl, log_nodes=0,
                   early_branch=None, check_every=None):
        calls.append((lam0, prec, early_branch, check_every))
        beta = np.zeros(inst.p)
        beta[[0, 3]] = 0.5
        obj, _ = oub.support_objective(inst.X, inst.y, np.array([0, 3]), lam0, lam2, M)
        cert = lam0 > 0.1
        secs = {None: 2.0 if prec == 0 else 0.04, 1: 0.02}[early_branch]
        rec = {"status": "optimal" if cert else "time_limit", "seconds": secs, "nodes": 100,
               "nnz": 2, "ub": obj, "lb": obj, "gap": 0.0, "certified": cert}
        return rec, beta, None

    monkeypatch.setattr(bench, "solve_record", fake_solve)
    args = types.SimpleNamespace(workload="c1_p16", rho=0.3, alpha=1.6, precision="tc3",
                                 cert_time_limit=1.0)
    out = bench.run_certified(args, 0)
    rows = out["instances"]
    assert [c[1:] for c in calls] == [(3, None, None), (0, None, None), (3, 1, 10),
                                      (0, 1, 10), (3, None, None), (0, None, None)]
    eb = rows[0]["mixed_early_branch"]
    assert eb["same_support_as_mixed"] and eb["speedup_vs_mixed"] == pytest.approx(2.0)
    assert eb["speedup_vs_fp64"] == pytest.approx(100.0)
    assert eb["speedup_vs_fp64_early_branch"] == pytest.approx(1.0)
    assert rows[0]["fp64_early_branch"]["same_support_as_mixed"]
    assert out["paths"]["fp64_early_branch"]["of"] == 1
    assert "mixed_early_branch" not in rows[1] and "mixed_support_list" not in rows[0]
    assert out["paths"]["mixed_early_branch"]["certified"] == 1
    assert out["paths"]["mixed_early_branch"]["of"] == 1
    assert out["reverify"]["supports_ok"]
