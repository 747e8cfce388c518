"""Allocation-free dual bound (bnb_dual_bound_static) against bnb_dual_bound and the oracle.

Some callers cannot allocate device memory (for example code running under
another framework that already owns the GPU's memory through its own allocator,
or a loop that cannot afford cudaMalloc's synchronisation).  The static variant
keeps its scratch in a fixed array inside the library; this test calls it twice
in a row through the C ABI, with different node counts and inputs, and checks
each result against the handle-based bnb_dual_bound and against the FP64
oracle's Eq. dual (oracle.relax.dual_value) within the certificate tolerance of
the other tests (1e-10 relative).  It lives in its own file so that it is
collected last.
"""
import numpy as np
import pytest

import datagen
from oracle import relax

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
bnb = pytest.importorskip("paper_2602_04551_b300")


def _case(inst, K, seed):
    rng = np.random.default_rng(seed)
    fix = datagen.random_fixings(inst.p, K, rng, 12)
    r = inst.y[None, :] * rng.uniform(0.2, 1.2, (K, 1)) + rng.normal(0, 0.3, (K, inst.n))
    return fix, r


def _close(got, want):
    return np.all(np.abs(got - want) <= 1e-10 * np.maximum(1.0, np.abs(want)))


def test_static_dual_bound_matches_handle_version_and_oracle_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    inst = datagen.config_instance("c2_small", 0)
    lam2 = datagen.CONFIGS["c2_small"]["lam2"]
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.05 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    opt = bnb.bnb_options_default(M=M, batch_K=64, precision=bnb.BNB_PREC_FP64,
                                  queue_capacity=1 << 12)
    dX = torch.tensor(np.asfortranarray(inst.X).T.copy(), dtype=torch.float64, device="cuda")
    dy = torch.tensor(inst.y, dtype=torch.float64, device="cuda")
    with bnb.bnb_create(inst.X, inst.y, lam0, lam2, opt) as h:
        for K, seed in ((37, 1), (9, 2)):
            fix, r = _case(inst, K, seed)
            ref = bnb.bnb_dual_bound(h, fix, r)
            orc = np.array([relax.dual_value(inst.X, inst.y, r[k], fix[k], lam0, lam2, M)
                            for k in range(K)])
            dfix = torch.tensor(fix, device="cuda")
            dr = torch.tensor(r, dtype=torch.float64, device="cuda")
            dlb = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
            bnb.bnb_dual_bound_static(dX, dy, inst.n, inst.p, lam0, lam2, M, dfix, dr, dlb)
            torch.cuda.synchronize()
            got = dlb.cpu().numpy()
            assert _close(got, ref), (got - ref)
            assert _close(got, orc), (got - orc)


def test_static_dual_bound_rejects_oversized_request():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    # K * (ceil(p/256) + 2) = 257 * 4096 > 2^20 doubles of scratch; the buffers have the
    # full sizes, so a missing size check would still stay inside them
    n, p, K = 4, 256 * 4094, 257
    dX = torch.zeros(n * p, dtype=torch.float64, device="cuda")
    dy = torch.zeros(n, dtype=torch.float64, device="cuda")
    dfix = torch.zeros((K, p), dtype=torch.int8, device="cuda")
    dr = torch.zeros((K, n), dtype=torch.float64, device="cuda")
    dlb = torch.zeros(K, dtype=torch.float64, device="cuda")
    with pytest.raises(bnb.BnbError) as ei:
        bnb.bnb_dual_bound_static(dX, dy, n, p, 0.1, 0.1, 1.0, dfix, dr, dlb)
    assert ei.value.code == bnb.BNB_EINVAL


def test_static_dual_bound_wrapper_rejects_mismatched_tensors():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    n, p, K = 8, 300, 3
    dX = torch.zeros(n * p, dtype=torch.float64, device="cuda")
    dy = torch.zeros(n, dtype=torch.float64, device="cuda")
    dfix = torch.zeros((K, p), dtype=torch.int8, device="cuda")
    dr = torch.zeros((K, n), dtype=torch.float64, device="cuda")
    dlb = torch.zeros(K, dtype=torch.float64, device="cuda")
    for bad in (dict(dr=torch.zeros((K, n - 1), dtype=torch.float64, device="cuda")),
                dict(dlb=torch.zeros(K, dtype=torch.float32, device="cuda")),
                dict(dfix=torch.zeros((K, p), dtype=torch.int8)),
                dict(dX=torch.zeros((p, n), dtype=torch.float64, device="cuda").t())):
        args = dict(dX=dX, dy=dy, dfix=dfix, dr=dr, dlb=dlb)
        args.update(bad)
        with pytest.raises(ValueError):
            bnb.bnb_dual_bound_static(args["dX"], args["dy"], n, p, 0.1, 0.1, 1.0, args["dfix"],
                                      args["dr"], args["dlb"])
