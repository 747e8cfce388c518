"""The C-ABI library loads on a machine without a GPU, exports every symbol that
include/bnb.h declares, and refuses work cleanly when no device is present."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2602_04551_b300 import build
    build.build()
    import paper_2602_04551_b300 as b
    return b


def _declared():
    txt = open(os.path.join(ROOT, "include", "bnb.h")).read()
    return set(re.findall(r"\b(bnb_[a-z_0-9]+)\s*\(", txt)) - {"bnb_handle"}


def test_header_symbols_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (bnb_[a-z_0-9]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    assert declared <= exported, declared - exported
    assert set(lib.SYMBOLS) == declared


def test_options_default_and_errors(lib):
    o = lib.bnb_options_default()
    assert o.M == 0.0 and o.rho == 1.0 and o.batch_K == 512 and o.node_tol == 1e-4
    import torch
    if torch.cuda.is_available():
        pytest.skip("device present: the no-device error path is not reachable")
    with pytest.raises(lib.BnbError) as ei:
        lib.bnb_create(np.ones((4, 3)), np.ones(4), 0.1, 0.1, lib.bnb_options_default(M=1.0))
    assert ei.value.code in (lib.BNB_ENODEV, lib.BNB_EINVAL)
