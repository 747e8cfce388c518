"""Pins for the oracle's closed forms against 1-D numeric optimisation.

Each closed form in oracle.relax is checked against the optimisation problem it
solves, evaluated by numeric search (dense grid + bounded Brent refinement)
rather than by retyping the formula:
  * psi (Eq. psi)           = min over (z, s) of the coordinate problem of Eq. relaxnode
  * prox (Eq. minbetalower) = argmin over |b| <= M of rho/2 (b - bt)^2 + psi(b)
  * nu (Eq. nudef)          = max over |b| <= M of x b - psi(b)   (the conjugate)
  * z recovery (App. A.1)   = argmin over z of lambda0 z + lambda2 b^2 / z
"""
import numpy as np
import pytest
from scipy.optimize import minimize_scalar

from oracle import relax

# parameter sets covering both regimes: sqrt(l0/l2) <= M and sqrt(l0/l2) > M
PARAMS = [
    (0.05, 0.01, 3.0),    # sqrt(l0/l2) = 2.24 <= 3
    (0.05, 0.01, 1.5),    # 2.24 > 1.5 (linear regime)
    (0.3, 0.5, 1.0),      # 0.77 <= 1
    (1e-3, 1e-3, 0.7),    # 1.0 > 0.7
    (0.0, 0.01, 2.0),     # lambda0 = 0
]


def _grid_min(fvec, lo, hi, n=40001):
    """Minimum of a 1-D function given vectorised; grid, then Brent on the bracket."""
    xs = np.linspace(lo, hi, n)
    vals = fvec(xs)
    i = int(np.argmin(vals))
    xb, fb = xs[i], vals[i]
    a, b = xs[max(i - 1, 0)], xs[min(i + 1, n - 1)]
    if b > a:
        res = minimize_scalar(lambda x: float(fvec(np.array([x]))[0]), bounds=(a, b),
                              method="bounded", options={"xatol": 1e-14})
        if res.fun < fb:
            xb, fb = res.x, res.fun
    return xb, fb


def test_T_definition_values():
    # Eq. Tdef at hand-picked points: below, inside and beyond the threshold band
    assert relax.T(0.3, 0.5, 1.0) == 0.0
    assert relax.T(-0.5, 0.5, 1.0) == 0.0
    assert relax.T(1.2, 0.5, 1.0) == pytest.approx(0.7)
    assert relax.T(-1.2, 0.5, 1.0) == pytest.approx(-0.7)
    assert relax.T(1.5, 0.5, 1.0) == pytest.approx(1.0)
    assert relax.T(-4.0, 0.5, 1.0) == pytest.approx(-1.0)


@pytest.mark.parametrize("lam0,lam2,M", PARAMS)
def test_psi_is_min_over_z_s(lam0, lam2, M):
    rng = np.random.default_rng(1)
    for b in list(rng.uniform(-M, M, 40)) + [0.0, M, -M, 0.999 * M]:
        # free coordinate: min lam0 z + lam2 s  s.t. b^2 <= s z, |b| <= M z, 0 <= z <= 1
        if b == 0.0:
            best = 0.0
        else:
            _, best = _grid_min(lambda z: lam0 * z + lam2 * b * b / z, max(abs(b) / M, 1e-12), 1.0)
        got = relax.psi(np.array([b]), np.array([relax.FREE]), lam0, lam2, M)[0]
        assert got == pytest.approx(best, rel=1e-9, abs=1e-12)
        # F1: z = 1, s = b^2
        got1 = relax.psi(np.array([b]), np.array([relax.F1]), lam0, lam2, M)[0]
        assert got1 == pytest.approx(lam0 + lam2 * b * b, rel=1e-12)
    assert relax.psi(np.array([0.1]), np.array([relax.F0]), lam0, lam2, M)[0] == np.inf
    assert relax.psi(np.array([0.0]), np.array([relax.F0]), lam0, lam2, M)[0] == 0.0
    assert relax.psi(np.array([M * 1.01]), np.array([relax.FREE]), lam0, lam2, M)[0] == np.inf


@pytest.mark.parametrize("lam0,lam2,M", PARAMS)
@pytest.mark.parametrize("rho", [0.3, 1.0, 4.0])
def test_prox_is_numeric_argmin(lam0, lam2, M, rho):
    rng = np.random.default_rng(2)
    s0 = np.sqrt(lam0 / lam2)
    thr = [2 * np.sqrt(lam0 * lam2) / rho + s0, 2 * np.sqrt(lam0 * lam2) / rho,
           (lam0 / M + lam2 * M) / rho, (lam0 / M + lam2 * M) / rho + M]
    pts = list(rng.normal(0, 2 * M, 30)) + [t * f for t in thr for f in (0.999, 1.0, 1.001, -1.0)]
    for code in (relax.FREE, relax.F1):
        for bt in pts:
            def f(b):
                b = np.asarray(b, dtype=np.float64)
                return 0.5 * rho * (b - bt) ** 2 + relax.psi(b, np.full(b.shape, code), lam0, lam2, M)
            xb, fb = _grid_min(f, -M, M)
            got = relax.prox(np.array([bt]), np.array([code]), lam0, lam2, M, rho)[0]
            assert abs(got) <= M
            assert f(np.array([got]))[0] <= fb + 1e-11 * max(1.0, abs(fb))
            assert got == pytest.approx(xb, abs=2e-6)
    assert relax.prox(np.array([3.0]), np.array([relax.F0]), lam0, lam2, M, rho)[0] == 0.0


@pytest.mark.parametrize("lam0,lam2,M", PARAMS)
def test_nu_is_conjugate_of_psi(lam0, lam2, M):
    xs = list(np.linspace(0, 6 * M * max(lam2, 0.1), 37)) + [2 * M * lam2, 2 * np.sqrt(lam0 * lam2),
                                                                lam0 / M + lam2 * M]
    for code in (relax.FREE, relax.F1, relax.F0):
        for x in xs:
            if code == relax.F0:
                best = 0.0
            else:
                def g(b):
                    b = np.asarray(b, dtype=np.float64)
                    return -(x * b - relax.psi(b, np.full(b.shape, code), lam0, lam2, M))
                _, fb = _grid_min(g, -M, M)
                best = -fb
            got = relax.nu(np.array([x]), np.array([code]), lam0, lam2, M)[0]
            assert got == pytest.approx(best, rel=1e-9, abs=1e-11)


def test_h_continuous_at_kink():
    lam0, lam2, M = 0.2, 0.03, 1.7
    x = 2 * M * lam2
    left = relax.h(np.array([x * (1 - 1e-12)]), lam0, lam2, M)[0]
    right = relax.h(np.array([x * (1 + 1e-12)]), lam0, lam2, M)[0]
    assert left == pytest.approx(right, abs=1e-9)


@pytest.mark.parametrize("lam0,lam2,M", [p for p in PARAMS if p[0] > 0])
def test_z_recovery_is_argmin(lam0, lam2, M):
    rng = np.random.default_rng(3)
    for b in list(rng.uniform(-M, M, 30)) + [M, -M]:
        if b == 0:
            continue
        zb, _ = _grid_min(lambda z: lam0 * z + lam2 * b * b / z, abs(b) / M, 1.0)
        got = relax.z_of_beta(np.array([b]), np.array([relax.FREE]), lam0, lam2, M)[0]
        assert got == pytest.approx(zb, abs=1e-6)
    assert relax.z_of_beta(np.array([0.4]), np.array([relax.F1]), lam0, lam2, M)[0] == 1.0
    assert relax.z_of_beta(np.array([0.0]), np.array([relax.F0]), lam0, lam2, M)[0] == 0.0
