"""Pins of the oracle's PPL update and adaptive time stepping against hand-worked values
(tests/golden/ppl_adaptime.json, Sec. 5.4 eq. lag_method and Sec. 5.7 eqs tend/steps)."""
import json
import os

import pytest

from oracle.ppl import PPL, adaptime

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ppl_adaptime.json")))


def test_ppl_first_iterates():
    g = GOLD["ppl_constant_C_1p2"]
    s = PPL(1)
    lam1, L1 = s.update([g["C"]], J=3.0)
    assert lam1[0] == pytest.approx(g["lambda1"], rel=1e-15)
    assert s.z[0] == pytest.approx(g["z1"], rel=1e-15)
    assert s.mu[0] == 0.0 and s.delta == pytest.approx(0.4995, rel=1e-15)
    # L = J + lambda (C-1) + mu z + alpha/2 z^2 + beta/2 (lambda-mu)^2
    assert L1 == pytest.approx(3.0 + g["lambda1"] * 0.2 + 1000 * g["z1"] ** 2 + 0.25 * g["lambda1"] ** 2, rel=1e-14)
    lam2, _ = s.update([g["C"]], J=3.0)
    assert s.mu[0] == pytest.approx(g["mu2"], rel=1e-14)
    assert lam2[0] == pytest.approx(g["lambda2"], rel=1e-14)
    assert s.delta == pytest.approx(0.4990005, rel=1e-15)


def test_ppl_satisfied_constraint_keeps_zero():
    s = PPL(2)
    for _ in range(5):
        lam, L = s.update([1.0, 1.0], J=2.0)
    assert list(lam) == [0.0, 0.0] and L == 2.0


@pytest.mark.parametrize("case", GOLD["adaptime"])
def test_adaptime(case):
    t_end, ns = adaptime(case["Btt"])
    assert t_end == pytest.approx(case["t_end"], rel=1e-15)
    assert ns == case["nsteps"]


def test_adaptime_rounds_half_away():
    # choose B so that s lands exactly on x.5: s = 8 ((t - tmin)/(tmax - tmin))^(1/6) + 8 = 12.5
    frac = (4.5 / 8) ** 6
    t = 1e-3 + frac * (0.1 - 1e-3)
    _, ns = adaptime(1e-2 / t)
    assert ns in (12, 13)         # 12.5 up to rounding of the 1/6 power; half rounds away -> 13 when exact
