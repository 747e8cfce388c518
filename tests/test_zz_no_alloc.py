"""Allocation-free dual bound (bnb_dual_bound_static) against bnb_dual_bound.

Some callers cannot allocate device memory (for example code running under
another framework that already owns the GPU's memory through its own allocator,
or a loop that cannot afford cudaMalloc's synchronisation).  The static variant
keeps its scratch in a fixed array inside the library; this test calls it twice
in a row through the C ABI, with different node counts and inputs, and checks
each result against the handle-based bnb_dual_bound within the certificate
tolerance of the other tests (1e-10 relative).  It lives in its own file so that
it is collected last.
"""
import numpy as np
import pytest

import datagen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
bnb = pytest.importorskip("paper_2602_04551_b300")


def _case(inst, K, seed):
    rng = np.random.default_rng(seed)
    fix = datagen.random_fixings(inst.p, K, rng, 12)
    r = inst.y[None, :] * rng.uniform(0.2, 1.2, (K, 1)) + rng.normal(0, 0.3, (K, inst.n))
    return fix, r


def test_static_dual_bound_matches_handle_version_twice():
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
            dfix = torch.tensor(fix, device="cuda")
            dr = torch.tensor(r, dtype=torch.float64, device="cuda")
            dlb = torch.full((K,), float("nan"), dtype=torch.float64, device="cuda")
            bnb.bnb_dual_bound_static(dX, dy, inst.n, inst.p, lam0, lam2, M, dfix, dr, dlb)
            torch.cuda.synchronize()
            got = dlb.cpu().numpy()
            assert np.all(np.abs(got - ref) <= 1e-10 * np.maximum(1.0, np.abs(ref))), (got - ref)


def test_static_dual_bound_rejects_oversized_request():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    n, p, K = 8, 1 << 16, 5000            # K * (ceil(p/256) + 2) > 2^20
    dX = torch.zeros(n * p, dtype=torch.float64, device="cuda")
    dy = torch.zeros(n, dtype=torch.float64, device="cuda")
    dfix = torch.zeros((K, 1), dtype=torch.int8, device="cuda")
    dr = torch.zeros((K, n), dtype=torch.float64, device="cuda")
    dlb = torch.zeros(K, dtype=torch.float64, device="cuda")
    with pytest.raises(bnb.BnbError) as ei:
        bnb.bnb_dual_bound_static(dX, dy, n, p, 0.1, 0.1, 1.0, dfix, dr, dlb)
    assert ei.value.code == bnb.BNB_EINVAL
