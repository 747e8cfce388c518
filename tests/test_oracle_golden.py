"""The stored C1 optimum (written by tests/golden/make_golden.py from the oracle)
is reproduced, and the p = 16 variant of the same recipe agrees with brute force."""
import json
import os

import numpy as np
import pytest

import datagen
from oracle import bnb, brute

GOLD = os.path.join(os.path.dirname(__file__), "golden", "c1_optimum.json")


def _cases():
    with open(GOLD) as fh:
        return json.load(fh)["cases"]


@pytest.mark.parametrize("case", _cases()[:1], ids=lambda c: f"seed{c['seed']}")
def test_c1_golden_reproduced(case):
    inst = datagen.config_instance("c1", case["instance"])
    res = bnb.solve(inst.X, inst.y, case["lambda0"], case["lambda2"], case["M"], gap=case["gap"])
    assert [int(i) for i in np.nonzero(res.beta)[0]] == case["support"]
    assert res.ub == pytest.approx(case["objective"], rel=1e-10)
    assert len(case["support"]) == 5


def test_c1_recipe_p16_brute_force():
    inst = datagen.config_instance("c1_p16", 0)
    lam2 = 0.01
    M = datagen.big_m(inst.X, inst.y, inst.support_true, lam2)
    lam0 = 0.1 * datagen.lambda0_scale(inst.X, inst.y, lam2)
    br = brute.solve(inst.X, inst.y, lam0, lam2, M)
    res = bnb.solve(inst.X, inst.y, lam0, lam2, M, gap=1e-6)
    assert tuple(np.nonzero(res.beta)[0]) == br.support
    assert res.ub == pytest.approx(br.objective, rel=1e-8)
