"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (stated per precision):
  * certificates (Proposition 1 bound for a given r): FP64 on both sides, only the
    summation order differs -> |LB_gpu - LB_oracle| <= 1e-10 max(1, |LB|);
  * one ADMM iteration: FP64 path 1e-8; FP32 path (FP32 Woodbury b-update with a
    Newton-Schulz G^-1) 2e-4 * max(1, |ref|);
  * converged node bound: valid (<= the relaxation optimum of the independent
    second solver) and within the node tolerance of it;
  * upper bound on a support: FP64 polish -> 1e-10 relative objective, 1e-7 in beta;
  * full solve: identical optimal support, objective within 1e-8 relative.
"""
import json
import os

import numpy as np
import pytest

import datagen
from oracle import relax, admm, pgd, ub as oub, brute

pytestmark = pytest.mark.gpu

bnb = pytest.importorskip("paper_2602_04551_b300")
PRECS = [pytest.param(1, id="fp32"), pytest.param(0, id="fp64"), pytest.param(3, id="tc3"),
         pytest.param(2, id="bf16"), pytest.param(4, id="bf16x2")]
# one-iteration tolerance per precision (relative to max(1, |ref|))
ITER_TOL = {0: 1e-8, 1: 2e-4, 3: 3e-4, 2: 3e-2, 4: 1e-2}
# node tolerance used for converged-bound checks per precision
NODE_TOL = {0: 1e-7, 1: 1e-5, 3: 1e-5, 2: 1e-3, 4: 1e-3}
GOLD = os.path.join(os.path.dirname(__file__), "golden", "c1_optimum.json")


def _inst(name, inst_id=0, frac=0.05, mfac=1.5):
    c = datagen.CONFIGS[name]
    inst = datagen.config_instance(name, inst_id)
    lam2 = c["lam2"]
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2, mfac)
    lam0 = frac * datagen.lambda0_scale(inst.X, inst.y, lam2)
    return inst, lam0, lam2, M


def _handle(inst, lam0, lam2, M, prec, K=64, **kw):
    kw.setdefault("time_limit_s", 60.0)
    kw.setdefault("queue_capacity", 1 << 16)
    o = bnb.bnb_options_default(M=M, precision=prec, batch_K=K, **kw)
    return bnb.bnb_create(inst.X, inst.y, lam0, lam2, o)


# ------------------------------------------------------------------ certificate


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mfac", [1.5, 0.3])
def test_dual_bound_matches_oracle(prec, mfac):
    inst, lam0, lam2, M = _inst("c2_small", 0, mfac=mfac)
    rng = np.random.default_rng(11)
    K = 37  # ragged against every tile width
    fix = datagen.random_fixings(inst.p, K, rng, 12)
    fix[0] = -1
    fix[1] = 0          # every coordinate in F0
    fix[2] = 1          # every coordinate in F1 (a leaf)
    r = inst.y[None, :] * rng.uniform(0.2, 1.2, (K, 1)) + rng.normal(0, 0.3, (K, inst.n))
    with _handle(inst, lam0, lam2, M, prec, K=48) as h:
        lb = bnb.bnb_dual_bound(h, fix, r)
    for k in range(K):
        ref = relax.dual_value(inst.X, inst.y, r[k], fix[k], lam0, lam2, M)
        assert abs(lb[k] - ref) <= 1e-10 * max(1.0, abs(ref)), (k, lb[k], ref)


@pytest.mark.parametrize("prec", PRECS)
def test_dual_bound_full_size_sampled(prec):
    """C2 shape (n=1000, p=5000) in the bench launch width K=512; eight nodes checked."""
    inst, lam0, lam2, M = _inst("c2", 0)
    rng = np.random.default_rng(12)
    K = 8
    fix = datagen.random_fixings(inst.p, K, rng, 30)
    r = inst.y[None, :] * rng.uniform(0.5, 1.0, (K, 1)) + rng.normal(0, 0.05, (K, inst.n))
    with _handle(inst, lam0, lam2, M, prec, K=512) as h:
        lb = bnb.bnb_dual_bound(h, fix, r)
    for k in range(K):
        ref = relax.dual_value(inst.X, inst.y, r[k], fix[k], lam0, lam2, M)
        assert abs(lb[k] - ref) <= 1e-10 * max(1.0, abs(ref))


# ------------------------------------------------------------------ ADMM iteration


def _one_iteration_check(inst, lam0, lam2, M, prec, K, Kopt, rows, seed, tol=None, rho=1.0,
                         alpha=1.0, iters=1, stats=None, **kw):
    """`iters` ADMM iterations (penalty rho, over-relaxation alpha; one round of that many
    iterations, so all but the last take the fused update without the stop-test sums)
    through the C ABI against the oracle's direct-D iterations, element by element.  The
    b-update's operator D = (X^T X + rho I)^-1 has norm 1/rho on the null space of X (p > n),
    so the error of the low-precision products in b grows as 1/rho, and the iterations add
    their errors: the tolerance is iters * ITER_TOL / min(1, rho).  `stats`: entries the
    handle's bnb_get_stats must show."""
    rng = np.random.default_rng(seed)
    fix = datagen.random_fixings(inst.p, K, rng, 20)
    wb = (rng.uniform(-M, M, (K, inst.p)) * (rng.random((K, inst.p)) < 0.05)).astype(np.float32)
    wb[fix == 0] = 0.0
    wv = rng.normal(0, 0.05, (K, inst.p)).astype(np.float32)
    with _handle(inst, lam0, lam2, M, prec, K=Kopt, check_every=iters, rho=rho,
                 relax_alpha=alpha, **kw) as h:
        out = bnb.bnb_relax_batch(h, fix, wb, wv, max_iter=iters, want_v=True)
        st = bnb.bnb_get_stats(h)
    for key, want in (stats or {}).items():
        assert st[key] == want, (key, st[key], want)
    assert np.all(out["iters"] == iters)
    data = admm.AdmmData(inst.X, inst.y, rho)
    tol = iters * (ITER_TOL[prec] if tol is None else tol) / min(1.0, rho)
    for k in rows:
        beta, v = wb[k].astype(np.float64), wv[k].astype(np.float64)
        for _ in range(iters):
            b, beta, v = admm.admm_iteration(data, beta, v, fix[k], lam0, lam2, M, alpha=alpha)
        sb = max(1.0, np.max(np.abs(beta)))
        sv = max(1.0, np.max(np.abs(v)))
        np.testing.assert_allclose(out["beta"][k], beta, atol=tol * sb)
        np.testing.assert_allclose(out["v"][k], v, atol=tol * sv)
        assert np.all(out["beta"][k][fix[k] == 0] == 0.0)
        assert np.all(np.abs(out["beta"][k]) <= M * (1 + 1e-7))


@pytest.mark.parametrize("prec", PRECS)
def test_one_admm_iteration_matches_oracle(prec):
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=45, Kopt=64, rows=range(45), seed=3)


@pytest.mark.parametrize("prec", PRECS)
def test_one_admm_iteration_full_size_sampled(prec):
    """C2 shape at the bench width K=512; four sampled nodes against the oracle."""
    inst, lam0, lam2, M = _inst("c2", 0)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=512, Kopt=512, rows=[0, 131, 300, 511], seed=4)


@pytest.mark.parametrize("prec", PRECS)
def test_one_admm_iteration_benchmarked_rho_alpha(prec):
    """The penalty and over-relaxation the benchmark's autotuner picks (rho = 0.3,
    alpha = 1.6), element by element against the oracle's over-relaxed iteration: the
    rho-scaled terms of the fused update (v / rho, rho beta - V, the shifted W') and
    the alpha-mix of b and beta are exercised with rho != 1."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=45, Kopt=64, rows=range(45), seed=13,
                         rho=0.3, alpha=1.6)


@pytest.mark.parametrize("prec", [3, 1])
def test_one_admm_iteration_benchmarked_rho_alpha_full_size(prec):
    """The same at the benchmark's c2 shape and launch width (K = 512), sampled rows."""
    inst, lam0, lam2, M = _inst("c2", 0, frac=0.02)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=512, Kopt=512, rows=[0, 77, 256, 511],
                         seed=14, rho=0.3, alpha=1.6)


@pytest.mark.parametrize("prec", [3, 2])
def test_one_admm_iteration_narrow_batch_benchmarked_rho_alpha(prec):
    """Narrow batches (matrix-vector form) at rho = 0.3, alpha = 1.6."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=12, Kopt=64, rows=range(12), seed=15,
                         tol=ITER_TOL[1], rho=0.3, alpha=1.6)


def _threshold_targets(lam0, lam2, M, rho, fix, rng):
    """Per coordinate, a target for beta~ = b + v / rho on a breakpoint of the prox of
    Eq. minbetalower: free coordinates cycle over +-a, +-tau (the ridge switch) and
    +-(a + M) (the box) in the perspective regime, or +-a_lin and +-(a_lin + M) in the
    linear regime (sqrt(lam0/lam2) > M); F1 coordinates sit where the ridge value reaches
    the box, +-M (rho + 2 lam2) / rho; F0 coordinates get arbitrary values."""
    s0 = np.sqrt(lam0 / lam2)
    if s0 > M:
        a = (lam0 / M + lam2 * M) / rho
        pts = [a, a + M]
    else:
        a = 2.0 * np.sqrt(lam0 * lam2) / rho
        pts = [a, a + s0, a + M] if a + s0 < a + M else [a, a + M]
    p = len(fix)
    t = np.empty(p)
    for i in range(p):
        sg = 1.0 if i % 2 == 0 else -1.0
        if fix[i] == 1:
            t[i] = sg * M * (rho + 2.0 * lam2) / rho
        elif fix[i] == 0:
            t[i] = rng.normal(0, 0.5)
        else:
            t[i] = sg * pts[(i // 2) % len(pts)]
    return t


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("frac", [pytest.param(0.01, id="perspective"),
                                  pytest.param(0.1, id="linear")])
def test_one_iteration_at_prox_breakpoints(prec, frac):
    """A warm start crafted so that beta~ lands on the prox's breakpoints (within the FP32
    rounding of the warm start) for F0, F1 and free coordinates, in both psi regimes; the
    GPU's beta and v after one iteration match the oracle's element by element.  With
    n > p (the c1 shape) I/rho - D is invertible, so v can be solved for any target:
    beta~ = D (c + rho beta) + (I/rho - D) v."""
    inst, lam0, lam2, M = _inst("c1", 0, frac=frac)
    rho = 0.7
    assert (np.sqrt(lam0 / lam2) > M) == (frac == 0.1)
    rng = np.random.default_rng(17)
    K, p = 6, inst.p
    fix = np.full((K, p), -1, np.int8)
    for k in range(1, K):
        idx = rng.permutation(p)
        fix[k, idx[: 4 * k]] = 0
        fix[k, idx[4 * k: 6 * k]] = 1
    data = admm.AdmmData(inst.X, inst.y, rho)
    A = np.eye(p) / rho - data.D
    wb = np.zeros((K, p), np.float32)
    wv = np.zeros((K, p), np.float32)
    for k in range(K):
        tgt = _threshold_targets(lam0, lam2, M, rho, fix[k], rng)
        b0 = rng.uniform(-M, M, p) * (rng.random(p) < 0.3)
        b0[fix[k] == 0] = 0.0
        wb[k] = b0.astype(np.float32)
        v = np.linalg.solve(A, tgt - data.D @ (data.c + rho * wb[k].astype(np.float64)))
        wv[k] = v.astype(np.float32)
        # the crafted start reaches its targets up to the FP32 rounding of v
        b = data.D @ (data.c + rho * wb[k].astype(np.float64) - wv[k].astype(np.float64))
        bt = b + wv[k].astype(np.float64) / rho
        assert np.max(np.abs(bt - tgt)) <= 1e-5 * max(1.0, np.max(np.abs(tgt)))
    with _handle(inst, lam0, lam2, M, prec, K=8, check_every=1, rho=rho) as h:
        out = bnb.bnb_relax_batch(h, fix, wb, wv, max_iter=1, want_v=True)
    tol = ITER_TOL[prec] / min(1.0, rho)
    for k in range(K):
        _, beta, v = admm.admm_iteration(data, wb[k].astype(np.float64), wv[k].astype(np.float64),
                                         fix[k], lam0, lam2, M)
        # the crafted v is a few times larger than the iterates it produces (v_new = v +
        # rho (b - beta) cancels), so the rounding of the products scales with |v|
        sc = max(1.0, float(np.max(np.abs(wv[k]))))
        np.testing.assert_allclose(out["beta"][k], beta, atol=tol * sc)
        np.testing.assert_allclose(out["v"][k], v, atol=tol * sc)
        assert np.all(out["beta"][k][fix[k] == 0] == 0.0)
        assert np.all(np.abs(out["beta"][k]) <= M * (1 + 1e-7))


@pytest.mark.parametrize("prec", [3, 2])
def test_one_admm_iteration_narrow_batch_matches_oracle(prec):
    """12 active nodes in a tensor-core handle: the matrix-vector round form (FP32 on the
    FP32 data, so the FP32 tolerance applies in both precisions)."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=12, Kopt=64, rows=range(12), seed=8,
                         tol=ITER_TOL[1])


def test_one_admm_iteration_narrow_batch_full_size():
    """c2 shape, 9 active nodes (partial slot group) through the matrix-vector form."""
    inst, lam0, lam2, M = _inst("c2", 0)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=9, Kopt=512, rows=[0, 4, 8], seed=9,
                         tol=ITER_TOL[1], mv_crossover=32)


def test_narrow_and_wide_forms_agree_on_converged_bounds():
    """The same 20 nodes relaxed with the matrix-vector form (crossover 32) and with the
    tensor-core form (crossover 0): both bounds valid, equal within the node tolerance."""
    inst, lam0, lam2, M = _inst("c2_small", 2)
    rng = np.random.default_rng(21)
    fix = datagen.random_fixings(inst.p, 20, rng, 10)
    outs = []
    for cross in (32, 0):
        with _handle(inst, lam0, lam2, M, 3, K=32, node_tol=1e-5, max_admm_iter=20000,
                     mv_crossover=cross) as h:
            outs.append(bnb.bnb_relax_batch(h, fix, max_iter=20000))
    for k in range(20):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        for out in outs:
            assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
            assert out["lb"][k] >= opt - 20 * 1e-5 * max(1.0, abs(opt))


@pytest.mark.parametrize("cross", [0, 8, 32])
def test_solve_same_answer_with_any_crossover(cross):
    """Solves whose rounds switch between the narrow and wide forms on the device (CUDA-
    graph conditional) return the stored optimum."""
    case = json.load(open(GOLD))["cases"][0]
    inst = datagen.config_instance("c1", case["instance"])
    o = bnb.bnb_options_default(M=case["M"], precision=3, batch_K=32, node_tol=1e-7,
                                max_admm_iter=5000, queue_capacity=1 << 16, time_limit_s=60.0,
                                mv_crossover=cross)
    with bnb.bnb_create(inst.X, inst.y, case["lambda0"], case["lambda2"], o) as h:
        res = bnb.bnb_solve(h, case["gap"])
    assert [int(i) for i in np.nonzero(res["beta"])[0]] == case["support"]
    assert res["ub"] == pytest.approx(case["objective"], rel=1e-8)


@pytest.mark.parametrize("prec", [3, 2])
def test_one_admm_iteration_full_size_wide_batch(prec):
    """C2 shape at K=1024 (other tile widths of the fused and cluster-reduced products);
    the last slot of the last column tile and a ragged middle one are sampled."""
    inst, lam0, lam2, M = _inst("c2", 0)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=1000, Kopt=1024, rows=[0, 517, 999], seed=5)


SHAPES = [pytest.param(1, id="single"), pytest.param(2, id="clusters_of_two"),
          pytest.param(3, id="cta_pairs_transposed"), pytest.param(4, id="cta_pairs")]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", [3, 4, 2])
def test_one_admm_iteration_every_fused_shape(shape, prec):
    """Each shape of the fused X^T U' product (one CTA per tile, clusters of two sharing
    the X tile, the product on CTA pairs transposed and not) gives the oracle's iteration."""
    if shape == 4 and prec == 4:
        pytest.skip("the untransposed pair product has no two-term (BF16X2) form")
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=45, Kopt=128, rows=range(45), seed=13,
                         fused_shape=shape)


@pytest.mark.parametrize("shape", [3, 4])
def test_one_admm_iteration_cta_pairs_full_size(shape):
    """c2 at K=512 on CTA pairs: transposed, slots on both CTAs of both row tiles are
    sampled (0, 127, 128 and 255 of the first tile, 256 and 511 of the second);
    untransposed, the same slots fall in the three 176-wide column tiles, and every
    feature (both CTAs of all 20 row tiles, the ragged last one included) is compared."""
    inst, lam0, lam2, M = _inst("c2", 0)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=512, Kopt=512,
                         rows=[0, 127, 128, 255, 256, 511], seed=14, fused_shape=shape)


PAIR_WIDTHS = [80, 96, 128, 176]


@pytest.mark.parametrize("width", PAIR_WIDTHS)
@pytest.mark.parametrize("prec", [3, 2])
def test_one_admm_iteration_untransposed_pair_widths(width, prec):
    """The untransposed CTA-pair product at every tile width it offers (80, 96 and 128 hold
    two accumulators and put several tiles on a pair; 176 one), forced with fused_width:
    at c2_small (K = 45 of 128 slots: ragged slot tiles) and at c2 (K = 512) with slots in
    every slot tile and the ragged last feature tile compared."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=45, Kopt=128, rows=range(45), seed=13,
                         fused_shape=4, fused_width=width)
    if prec == 3:
        inst, lam0, lam2, M = _inst("c2", 0)
        rows = sorted({0, width - 1, width, 2 * width + 3, 300, 511})
        _one_iteration_check(inst, lam0, lam2, M, 3, K=512, Kopt=512, rows=rows, seed=14,
                             fused_shape=4, fused_width=width)


@pytest.mark.parametrize("rho,alpha", [(1.0, 1.0), (0.2, 1.6)])
def test_admm_iterations_one_round_untransposed_pairs(rho, alpha):
    """Three iterations in one round on the 256 x 176 pair tile (TC3): the first two take
    the fused update without the stop-test sums, the third the one with them; at c2_small
    (K = 45 of 128 slots: inactive and past-K slots, ragged feature tile) and at the
    benchmark's c2 shape (K = 512: the second CTA of every pair, every slot tile, the last
    feature tile), element by element against the oracle's three iterations, at rho = 1
    and at the benchmarked rho = 0.2, alpha = 1.6."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=45, Kopt=128, rows=range(45), seed=31,
                         rho=rho, alpha=alpha, iters=3, fused_shape=4, fused_width=176,
                         mv_crossover=0, stats={"fused_tile_width": 176, "fused_transposed": 0})
    inst, lam0, lam2, M = _inst("c2", 0, frac=0.02)
    rows = [0, 15, 16, 175, 176, 191, 352, 500, 511]
    _one_iteration_check(inst, lam0, lam2, M, 3, K=512, Kopt=512, rows=rows, seed=32,
                         rho=rho, alpha=alpha, iters=3, fused_shape=4, fused_width=176,
                         mv_crossover=0, stats={"fused_tile_width": 176, "fused_transposed": 0})


@pytest.mark.parametrize("width", PAIR_WIDTHS)
def test_converged_bounds_untransposed_pair_widths(width):
    """Converged bounds (both instantiations of the fused update: the round's last
    iteration with the stop-test sums, the others without) at each pair width: valid and
    within 20 node tolerances of the second solver's optimum."""
    inst, lam0, lam2, M = _inst("c2_small", 2)
    rng = np.random.default_rng(22)
    fix = datagen.random_fixings(inst.p, 40, rng, 10)
    with _handle(inst, lam0, lam2, M, 3, K=128, node_tol=1e-5, max_admm_iter=20000,
                 mv_crossover=0, fused_shape=4, fused_width=width) as h:
        out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
        st = bnb.bnb_get_stats(h)
    assert st["fused_pairs"] > 0 and not st["fused_transposed"] and st["fused_tile_width"] == width
    for k in range(40):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
        assert out["lb"][k] >= opt - 20 * 1e-5 * max(1.0, abs(opt))


@pytest.mark.parametrize("shape", SHAPES)
def test_converged_bounds_and_solve_every_fused_shape(shape):
    """Converged node bounds (the stop-test sums of the fused epilogue decide when a node
    retires) stay valid and tight, and a solve returns the stored optimum, whatever the
    shape of the fused product."""
    inst, lam0, lam2, M = _inst("c2_small", 2)
    rng = np.random.default_rng(22)
    fix = datagen.random_fixings(inst.p, 20, rng, 10)
    with _handle(inst, lam0, lam2, M, 3, K=128, node_tol=1e-5, max_admm_iter=20000,
                 mv_crossover=0, fused_shape=shape) as h:
        out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
    for k in range(20):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
        assert out["lb"][k] >= opt - 20 * 1e-5 * max(1.0, abs(opt))
    case = json.load(open(GOLD))["cases"][0]
    ci = datagen.config_instance("c1", case["instance"])
    o = bnb.bnb_options_default(M=case["M"], precision=3, batch_K=128, node_tol=1e-7,
                                max_admm_iter=5000, queue_capacity=1 << 16, time_limit_s=60.0,
                                mv_crossover=0, fused_shape=shape)
    with bnb.bnb_create(ci.X, ci.y, case["lambda0"], case["lambda2"], o) as h:
        res = bnb.bnb_solve(h, case["gap"])
        st = bnb.bnb_get_stats(h)
        assert (st["fused_pairs"] > 0) == (shape >= 3)
        assert st["fused_transposed"] == (1 if shape == 3 else 0)
        assert (st["fused_clusters"] > 0) == (shape == 2)
    assert [int(i) for i in np.nonzero(res["beta"])[0]] == case["support"]
    assert res["ub"] == pytest.approx(case["objective"], rel=1e-8)


def _inst_odd():
    """A c2-recipe instance with n and p that are not multiples of 4 or 8: the scalar
    forms of the vectorised kernels (matrix-vector products, fused updates, W' formation)
    and ragged operand boxes."""
    inst = datagen.make_instance(101, 503, 0.3, 10, 5.0, 2077)
    lam2 = 1e-3
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2, 1.5)
    lam0 = 0.05 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    return inst, lam0, lam2, M


@pytest.mark.parametrize("shape", SHAPES)
def test_one_admm_iteration_odd_sizes_every_fused_shape(shape):
    inst, lam0, lam2, M = _inst_odd()
    _one_iteration_check(inst, lam0, lam2, M, 3, K=45, Kopt=128, rows=range(45), seed=31,
                         fused_shape=shape, mv_crossover=0)


def test_one_admm_iteration_odd_sizes_narrow_batch():
    inst, lam0, lam2, M = _inst_odd()
    _one_iteration_check(inst, lam0, lam2, M, 3, K=11, Kopt=64, rows=range(11), seed=32,
                         tol=ITER_TOL[1], mv_crossover=32)


def test_converged_bounds_odd_sizes():
    """Converged bounds on the odd instance in both round forms stay valid and tight."""
    inst, lam0, lam2, M = _inst_odd()
    rng = np.random.default_rng(33)
    fix = datagen.random_fixings(inst.p, 12, rng, 10)
    for cross in (32, 0):
        with _handle(inst, lam0, lam2, M, 3, K=64, node_tol=1e-5, max_admm_iter=20000,
                     mv_crossover=cross) as h:
            out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
        for k in range(12):
            _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
            assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
            assert out["lb"][k] >= opt - 20 * 1e-5 * max(1.0, abs(opt))


U_SHAPES = [pytest.param(1, id="cluster_reduced"), pytest.param(2, id="pairs_split_k"),
            pytest.param(3, id="pairs_in_clusters")]


@pytest.mark.parametrize("ushape", U_SHAPES)
@pytest.mark.parametrize("prec", [3, 2])
def test_one_admm_iteration_every_u_shape(ushape, prec):
    """Every form of U' = H W'^T (K split over a cluster; K chunks on CTA pairs added by
    a second kernel; CTA pairs in clusters that split K) gives the oracle's iteration."""
    inst, lam0, lam2, M = _inst("c2_small", 1)
    _one_iteration_check(inst, lam0, lam2, M, prec, K=45, Kopt=128, rows=range(45), seed=41,
                         u_shape=ushape, mv_crossover=0)


def test_one_admm_iteration_pairs_split_k_full_size():
    """c2 at K = 512 with U' on CTA pairs in 9 K chunks: slots of both slot tiles and both
    halves of a tile sampled."""
    inst, lam0, lam2, M = _inst("c2", 0)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=512, Kopt=512,
                         rows=[0, 127, 128, 255, 256, 511], seed=42, u_shape=2, mv_crossover=0)


@pytest.mark.parametrize("rho,alpha", [(1.0, 1.0), (0.2, 1.6)])
def test_admm_iterations_pairs_in_clusters_full_size(rho, alpha):
    """c2 at K = 512 with U' on 256 x 128 tiles, each on a cluster of CTA pairs splitting
    the K range (samples of both CTAs of a pair: rows 0-127 and 128-255 of each tile lie in
    different CTAs, every pair's partial tile summed in distributed shared memory), over a
    round of three iterations (the last one also forms U and the stop-test sums), against
    the oracle's iterations."""
    inst, lam0, lam2, M = _inst("c2", 0, frac=0.02)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=512, Kopt=512,
                         rows=[0, 63, 64, 127, 128, 255, 256, 383, 511], seed=44, rho=rho,
                         alpha=alpha, iters=3, u_shape=3, mv_crossover=0,
                         stats={"u_cluster_pairs": 4})


def test_admm_iterations_pairs_in_clusters_of_two():
    """U' on CTA pairs in split-K clusters with two pairs per cluster (the form the setup
    picks at C3): p = 300 gives 5 K steps, too few for four pairs, so the forced form takes
    two; three iterations in one round against the oracle's."""
    inst = datagen.make_instance(100, 300, 0.3, 5, 5.0, 2601)
    lam2 = 1e-3
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.05 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    _one_iteration_check(inst, lam0, lam2, M, 3, K=200, Kopt=256, rows=range(0, 200, 7),
                         seed=45, rho=0.3, alpha=1.6, iters=3, u_shape=3, mv_crossover=0,
                         stats={"u_cluster_pairs": 2})


@pytest.mark.parametrize("ushape", U_SHAPES)
def test_converged_bounds_every_u_shape(ushape):
    """Converged node bounds (the stop-test sums of U come from either form of U') stay
    valid and tight against the independent second solver."""
    inst, lam0, lam2, M = _inst("c2_small", 2)
    rng = np.random.default_rng(43)
    fix = datagen.random_fixings(inst.p, 20, rng, 10)
    with _handle(inst, lam0, lam2, M, 3, K=128, node_tol=1e-5, max_admm_iter=20000,
                 mv_crossover=0, u_shape=ushape) as h:
        out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
        st = bnb.bnb_get_stats(h)
        assert (st["u_split"] > 0) == (ushape == 2)
        assert (st["u_cluster_pairs"] > 0) == (ushape == 3)
    for k in range(20):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
        assert out["lb"][k] >= opt - 20 * 1e-5 * max(1.0, abs(opt))


# ------------------------------------------------------------------ converged node


@pytest.mark.parametrize("prec", PRECS)
def test_relaxation_bound_valid_and_tight(prec):
    inst, lam0, lam2, M = _inst("c1", 0, frac=0.05)
    rng = np.random.default_rng(5)
    K = 10
    fix = datagen.random_fixings(inst.p, K, rng, 6)
    tol = NODE_TOL[prec]
    with _handle(inst, lam0, lam2, M, prec, K=16, node_tol=tol, max_admm_iter=20000) as h:
        out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
    for k in range(K):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))          # valid (Prop. 1.1)
        assert out["lb"][k] >= opt - 20 * tol * max(1.0, abs(opt))      # tight at convergence
        if prec == 2:
            continue  # BF16 iterates: z/branch checked on the FP32-class paths
        z = out["z"][k]
        zref = relax.z_of_beta(out["beta"][k].astype(np.float64), fix[k], lam0, lam2, M)
        np.testing.assert_allclose(z, zref, atol=1e-6)
        free = np.nonzero(fix[k] == -1)[0]
        frac = np.minimum(z[free], 1 - z[free])
        if frac.max() > 0:
            assert out["branch"][k] == free[int(np.argmax(frac))]


# ------------------------------------------------------------------ upper bound


@pytest.mark.parametrize("prec", PRECS[:2])
@pytest.mark.parametrize("mfac", [1.5, 0.25])   # box loose / binding
def test_upper_batch_matches_oracle(prec, mfac):
    inst, lam0, lam2, M = _inst("c2_small", 2, mfac=mfac)
    rng = np.random.default_rng(6)
    K = 21
    sup = np.zeros((K, inst.p), np.uint8)
    for k in range(1, K):
        sup[k, rng.choice(inst.p, size=int(rng.integers(1, 15)), replace=False)] = 1
    sup[K - 1, inst.support_true] = 1
    with _handle(inst, lam0, lam2, M, prec, K=32) as h:
        ubv, beta = bnb.bnb_upper_batch(h, sup)
    for k in range(K):
        S = np.nonzero(sup[k])[0]
        obj, bref = oub.support_objective(inst.X, inst.y, S, lam0, lam2, M)
        assert ubv[k] == pytest.approx(obj, rel=1e-10), k
        np.testing.assert_allclose(beta[k], bref, atol=1e-7)


@pytest.mark.parametrize("prec", [1, 3, 0])
@pytest.mark.parametrize("mfac", [1.5, 0.3])
def test_projected_gradient_upper_bound_matches_oracle(prec, mfac):
    """The projected-gradient upper bound on its own (options.ub_polish = 0: no FP64
    re-solve), the value that decides inside a solve which supports get polished.  Against
    the oracle: the returned point is feasible (box, support) and its reported value is its
    exact objective; the value is within the method's stopping accuracy of the exact box
    ridge optimum and of the oracle's own run of Eqs. fpg_extrapolate..fpg_armijo with the
    same stopping rule (relative decrease below 1e-7, or 1e-13 on the FP64 path, within
    200 iterations).  Tolerance: an objective gap delta leaves beta within
    sqrt(2 delta / lambda_min(Q)) of the minimiser; delta <= 1e-5 relative here."""
    inst, lam0, lam2, M = _inst("c2_small", 2, mfac=mfac)
    rng = np.random.default_rng(16)
    K = 21
    sup = np.zeros((K, inst.p), np.uint8)
    for k in range(1, K):
        sup[k, rng.choice(inst.p, size=int(rng.integers(1, 15)), replace=False)] = 1
    sup[K - 1, inst.support_true] = 1
    with _handle(inst, lam0, lam2, M, prec, K=32, ub_polish=0) as h:
        ubv, beta = bnb.bnb_upper_batch(h, sup)
    rtol = 1e-7 if prec else 1e-13
    for k in range(K):
        S = np.nonzero(sup[k])[0]
        assert np.all(beta[k][sup[k] == 0] == 0.0)
        assert np.all(np.abs(beta[k]) <= M)
        assert ubv[k] == pytest.approx(relax.mip_objective(inst.X, inst.y, beta[k], lam0, lam2),
                                       rel=1e-12)
        obj, bref = oub.support_objective(inst.X, inst.y, S, lam0, lam2, M)
        if k == 0:
            assert ubv[k] == pytest.approx(obj, rel=1e-12)       # empty support
            continue
        assert ubv[k] >= obj * (1 - 1e-12)
        assert ubv[k] <= obj * (1 + 1e-5), (k, ubv[k], obj)
        bf = oub.fista_backtracking(inst.X, inst.y, S, lam2, M, tol=rtol, max_iter=200)
        full = np.zeros(inst.p)
        full[S] = bf
        ofista = relax.mip_objective(inst.X, inst.y, full, lam0, lam2)
        assert abs(ubv[k] - ofista) <= 1e-5 * abs(obj), (k, ubv[k], ofista)
        Q = inst.X[:, S].T @ inst.X[:, S] + 2 * lam2 * np.eye(len(S))
        lmin = float(np.linalg.eigvalsh(Q)[0])
        dev = np.sqrt(2 * max(ubv[k] - obj, 0.0) / lmin) + 1e-6
        assert np.max(np.abs(beta[k][S] - bref[S])) <= dev * 1.01 + 1e-6, k


def test_solve_after_upper_batch_reports_its_own_incumbent():
    """Upper bounds left on the handle by an earlier bnb_upper_batch call never become the
    solve's incumbent: the returned beta's objective is the returned UB, and both are
    the brute-force optimum."""
    inst, lam0, lam2, M = _inst("c1_p16", 0, frac=0.05)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    sup = np.zeros((8, inst.p), np.uint8)
    sup[0, list(br.support)] = 1
    sup[1, :3] = 1
    with _handle(inst, lam0, lam2, M, 3, K=8, node_tol=1e-7, max_admm_iter=5000) as h:
        bnb.bnb_upper_batch(h, sup)
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    obj = 0.5 * np.sum((inst.y - inst.X @ res["beta"]) ** 2) + lam0 * np.count_nonzero(res["beta"]) \
        + lam2 * np.sum(res["beta"] ** 2)
    assert obj == pytest.approx(res["ub"], rel=1e-10)
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)


# ------------------------------------------------------------------ full solve


@pytest.mark.parametrize("prec", PRECS)
def test_solve_c1_golden(prec):
    cases = json.load(open(GOLD))["cases"]
    for case in cases:
        inst = datagen.config_instance("c1", case["instance"])
        o = bnb.bnb_options_default(M=case["M"], precision=prec, batch_K=64, node_tol=1e-7,
                                    max_admm_iter=5000, queue_capacity=1 << 16,
                                    time_limit_s=60.0)
        with bnb.bnb_create(inst.X, inst.y, case["lambda0"], case["lambda2"], o) as h:
            res = bnb.bnb_solve(h, case["gap"])
        assert [int(i) for i in np.nonzero(res["beta"])[0]] == case["support"]
        assert res["ub"] == pytest.approx(case["objective"], rel=1e-8)
        assert res["lb"] <= res["ub"] * (1 + 1e-12)
        assert (res["ub"] - res["lb"]) <= case["gap"] * res["ub"] * (1 + 1e-9)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("frac", [0.2, 0.02])
def test_solve_matches_brute_force_p16(prec, frac):
    inst, lam0, lam2, M = _inst("c1_p16", 0, frac=frac)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, prec, K=8, node_tol=1e-7, max_admm_iter=5000) as h:
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)


@pytest.mark.parametrize("prec", [3, 1, 0])
@pytest.mark.parametrize("frac", [0.2, 0.03])
def test_early_branch_reaches_the_brute_force_optimum(prec, frac):
    """early_branch = 1 (a node whose primal estimate is already below the prune threshold
    is certified and branched at once): the same brute-force optimum, a final lower bound
    that is valid, and a C1 golden solve unchanged."""
    inst, lam0, lam2, M = _inst("c1_p16", 0, frac=frac)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, prec, K=8, node_tol=1e-7, max_admm_iter=5000,
                 early_branch=1) as h:
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)
    assert res["lb"] <= br.objective * (1 + 1e-9)
    case = json.load(open(GOLD))["cases"][0]
    inst = datagen.config_instance("c1", case["instance"])
    o = bnb.bnb_options_default(M=case["M"], precision=prec, batch_K=64, node_tol=1e-7,
                                max_admm_iter=5000, queue_capacity=1 << 16, time_limit_s=60.0,
                                early_branch=1)
    with bnb.bnb_create(inst.X, inst.y, case["lambda0"], case["lambda2"], o) as h:
        res = bnb.bnb_solve(h, case["gap"])
    assert [int(i) for i in np.nonzero(res["beta"])[0]] == case["support"]
    assert res["ub"] == pytest.approx(case["objective"], rel=1e-8)


def test_histograms_count_every_solved_node_and_depth_limit_is_reported():
    inst, lam0, lam2, M = _inst("c1_p16", 1, frac=0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, 3, K=8, node_tol=1e-7, max_admm_iter=5000) as h:
        res = bnb.bnb_solve(h, 1e-9)
        dh, sh = bnb.bnb_get_histograms(h, 300, 300)
        st = bnb.bnb_get_stats(h)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert dh.sum() == res["nodes"] == sh.sum()
    assert dh[0] == 1                                  # the root, once
    assert np.nonzero(dh)[0].max() <= st["max_depth"]
    assert sh[17:].sum() == 0                          # p = 16: no support is larger
    # a depth limit below the tree's depth ends the solve with its own status and a
    # lower bound that is still valid
    with _handle(inst, lam0, lam2, M, 3, K=8, node_tol=1e-7, max_admm_iter=5000, max_depth=8) as h:
        r8 = bnb.bnb_solve(h, 1e-9)
    if r8["status"] == "depth_limit":
        assert r8["lb"] <= br.objective * (1 + 1e-9)
    else:
        assert tuple(np.nonzero(r8["beta"])[0]) == br.support


@pytest.mark.parametrize("K", [1, 8])
def test_lockstep_batches_reach_the_same_optimum(K):
    """Algorithm 1's select-solve-branch batches (lockstep) against brute force."""
    inst, lam0, lam2, M = _inst("c1_p16", 1, frac=0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, 3, K=K, node_tol=1e-7, max_admm_iter=5000, lockstep=1) as h:
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)
    assert res["lb"] <= br.objective * (1 + 1e-9)


@pytest.mark.parametrize("K", [1, 3, 128])
def test_solve_batch_width_does_not_change_the_answer(K):
    inst, lam0, lam2, M = _inst("c1_p16", 1, frac=0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, 1, K=K, node_tol=1e-7, max_admm_iter=5000) as h:
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)


@pytest.mark.parametrize("prec", [1, 3])
def test_over_relaxed_admm_keeps_bounds_valid_and_answers_exact(prec):
    """relax_alpha > 1 changes the iterates, not the certificate: bounds stay below
    the relaxation optimum and the solve returns the brute-force optimum."""
    inst, lam0, lam2, M = _inst("c1", 0, frac=0.05)
    rng = np.random.default_rng(9)
    fix = datagen.random_fixings(inst.p, 8, rng, 6)
    with _handle(inst, lam0, lam2, M, prec, K=16, node_tol=1e-5, max_admm_iter=20000,
                 relax_alpha=1.6) as h:
        out = bnb.bnb_relax_batch(h, fix, max_iter=20000)
    for k in range(8):
        _, opt = pgd.solve_node(inst.X, inst.y, fix[k], lam0, lam2, M)
        assert out["lb"][k] <= opt + 1e-9 * max(1.0, abs(opt))
        assert out["lb"][k] >= opt - 2e-4 * max(1.0, abs(opt))
    inst, lam0, lam2, M = _inst("c1_p16", 0, frac=0.02)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, prec, K=8, node_tol=1e-7, max_admm_iter=5000,
                 relax_alpha=1.6) as h:
        res = bnb.bnb_solve(h, 1e-9)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)


@pytest.mark.parametrize("prec", [0, 3])
def test_root_heuristic_matches_oracle(prec):
    """Matching pursuit + exact polish: in FP64 the same greedy decisions as the
    oracle (same support, objective within 1e-10); in the mixed path a feasible
    point whose reported objective is its exact FP64 value."""
    from oracle import mp as omp
    for name, frac in (("c1", 0.05), ("c2_small", 0.05), ("c1_p16", 0.02)):
        inst, lam0, lam2, M = _inst(name, 0, frac=frac)
        with _handle(inst, lam0, lam2, M, prec, K=16) as h:
            beta, ubv = bnb.bnb_root_heuristic(h)
        assert np.all(np.abs(beta) <= M * (1 + 1e-12))
        assert ubv == pytest.approx(relax.mip_objective(inst.X, inst.y, beta, lam0, lam2), rel=1e-12)
        (obj, bref), S = omp.root_incumbent(inst.X, inst.y, lam0, lam2, M)
        if prec == 0:
            assert tuple(np.nonzero(beta)[0]) == tuple(np.nonzero(bref)[0])
            assert ubv == pytest.approx(obj, rel=1e-10)
        else:
            assert ubv <= relax.mip_objective(inst.X, inst.y, np.zeros(inst.p), lam0, lam2)


# ------------------------------------------------------------------ node log re-verification


def _reverify(inst, lam0, lam2, M, log):
    """Every logged certificate against the oracle's Eq. dual at the logged r: exact ones to
    1e-10 relative; screened ones are below D(r) by at most their recorded width."""
    assert log["count"] == len(log["lb"]) > 0
    for k in range(log["count"]):
        d = relax.dual_value(inst.X, inst.y, log["r"][k], log["fix"][k], lam0, lam2, M)
        tol = 1e-10 * max(1.0, abs(d))
        if log["exact"][k] == 1.0:
            assert abs(log["lb"][k] - d) <= tol, (k, log["lb"][k], d)
            assert log["width"][k] == 0.0
        else:
            assert log["lb"][k] <= d + tol, (k, log["lb"][k], d)
            assert d - log["lb"][k] <= log["width"][k] * (1 + 1e-9) + tol, (k, d, log["width"][k])
        assert log["node_lb"][k] == max(log["lb"][k], log["parent_lb"][k])


@pytest.mark.parametrize("prec", [3, 0])
def test_node_log_certificates_match_oracle(prec):
    """A solve that records its first certified nodes (options.log_nodes): each logged bound
    is the oracle's Eq. dual at the logged residual (exact terms) or a rigorous lower bound
    within its logged interval width (screened terms)."""
    inst, lam0, lam2, M = _inst("c2_small", 0, frac=0.1)
    with _handle(inst, lam0, lam2, M, prec, K=32, log_nodes=200, time_limit_s=5.0) as h:
        res = bnb.bnb_solve(h, 1e-4)
        log = bnb.bnb_get_node_log(h)
    assert log["count"] == min(200, res["nodes"])
    assert np.all(log["depth"][:1] == 0)          # the root is certified first
    _reverify(inst, lam0, lam2, M, log)


def test_node_log_certificates_match_oracle_odd_sizes():
    """The node log of a solve on the n = 101, p = 503 instance: the certificate screen
    takes its 4-byte-copy form there (n not a multiple of 4), and every logged bound is
    still the oracle's Eq. dual at the logged residual, or below it within the width."""
    inst, lam0, lam2, M = _inst_odd()
    with _handle(inst, lam0, lam2, M, 3, K=64, log_nodes=150, time_limit_s=5.0) as h:
        res = bnb.bnb_solve(h, 1e-4)
        log = bnb.bnb_get_node_log(h)
    assert log["count"] == min(150, res["nodes"]) > 0
    _reverify(inst, lam0, lam2, M, log)


def test_node_log_certificates_match_oracle_full_size():
    """The same at the benchmark's c2 shape and width (K = 512, TC3): 128 certificates of a
    real solve re-checked by the oracle."""
    inst, lam0, lam2, M = _inst("c2", 0, frac=0.02)
    with _handle(inst, lam0, lam2, M, 3, K=512, log_nodes=128, time_limit_s=3.0, rho=0.3,
                 relax_alpha=1.6, queue_capacity=1 << 18) as h:
        bnb.bnb_solve(h, 1e-4)
        log = bnb.bnb_get_node_log(h)
    assert log["count"] == 128
    _reverify(inst, lam0, lam2, M, log)


@pytest.mark.parametrize("lockstep", [0, 1])
@pytest.mark.parametrize("K", [1, 8, 64])
def test_fused_selection_same_answer_as_separate_launches(K, lockstep):
    """The round's selection as one cooperative launch (options.fused_select = 1) and as
    separate launches (the default): both reach the brute-force optimum at p = 16, with
    continuous refill and with Algorithm 1's lockstep batches."""
    inst, lam0, lam2, M = _inst("c1_p16", 1, frac=0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    for fused in (1, 0):
        with _handle(inst, lam0, lam2, M, 3, K=K, node_tol=1e-7, max_admm_iter=5000,
                     lockstep=lockstep, fused_select=fused) as h:
            res = bnb.bnb_solve(h, 1e-9)
        assert tuple(np.nonzero(res["beta"])[0]) == br.support, fused
        assert res["ub"] == pytest.approx(br.objective, rel=1e-8)
        assert res["lb"] <= br.objective * (1 + 1e-9)


def test_exact_bounds_option_same_answer_and_exact_certificates():
    """options.exact_bounds = 1: a branched node's certificate is the exact FP64 value at its
    residual (the node log shows every logged bound exact and equal to the oracle's Eq. dual),
    and the solve returns the brute-force optimum as with the default."""
    inst, lam0, lam2, M = _inst("c1_p16", 1, frac=0.03)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    with _handle(inst, lam0, lam2, M, 3, K=8, node_tol=1e-7, max_admm_iter=5000,
                 exact_bounds=1, log_nodes=64) as h:
        res = bnb.bnb_solve(h, 1e-9)
        log = bnb.bnb_get_node_log(h)
    assert tuple(np.nonzero(res["beta"])[0]) == br.support
    assert res["ub"] == pytest.approx(br.objective, rel=1e-8)
    thr_pruned = log["lb"] >= log["threshold"]
    assert np.all(log["exact"][~thr_pruned] == 1.0)
    _reverify(inst, lam0, lam2, M, log)
