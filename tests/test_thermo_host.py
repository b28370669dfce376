"""Host arithmetic of paper_2004_08669_gb300.thermo (no GPU): with the
library's scan replaced by a fake whose observables are closed forms in T,
central_derivatives must lay out T - dT, T, T + dT per temperature and return
the central differences of u and M and the beta-difference of beta f."""
import math

import numpy as np
import pytest

from paper_2004_08669_gb300 import thermo


def f_of(T):   # any smooth closed forms will do
    return -2.0 - 0.3 * T * T


def u_of(T):   # d(beta f)/d beta of f_of, i.e. f - T df/dT = -2 + 0.3 T^2
    return f_of(T) + 0.6 * T * T


def M_of(T):
    return math.exp(-T)


class FakeScan:
    created = []

    def __init__(self, spins, m, betas, workers=8, prec="fp64", device="cuda:0", **kw):
        self.betas = np.asarray(betas)
        FakeScan.created.append(self)
        self.closed = False

    def run(self, max_steps):
        n = len(self.betas)
        return [7] * n, [True] * n

    def observables(self):
        return [{"f": f_of(1 / b), "u": u_of(1 / b), "M": M_of(1 / b), "S_E": 0.5} for b in self.betas]

    def close(self):
        self.closed = True


def test_central_derivatives_arithmetic(monkeypatch):
    from paper_2004_08669_gb300 import ctm
    monkeypatch.setattr(ctm, "Scan", FakeScan)
    FakeScan.created.clear()
    temps, dT = [0.5, 1.5], 1e-4
    rows = thermo.central_derivatives(None, 8, temps, dT=dT)
    sc = FakeScan.created[-1]
    assert sc.closed
    np.testing.assert_allclose(1 / sc.betas, [0.5 - dT, 0.5, 0.5 + dT, 1.5 - dT, 1.5, 1.5 + dT], rtol=1e-14)
    for r, T in zip(rows, temps):
        assert r["converged"] and r["steps"] == [7, 7, 7]
        assert r["u"] == pytest.approx(u_of(T), rel=1e-15)
        assert r["u_fd"] == pytest.approx(u_of(T), rel=1e-7)           # d(beta f)/d beta
        assert r["C"] == pytest.approx(0.6 * T, rel=1e-6)   # u = -2 + 0.3 T^2
        assert r["dM_dT"] == pytest.approx(-math.exp(-T), rel=1e-7)


def test_rejects_a_step_past_zero_temperature():
    with pytest.raises(ValueError):
        thermo.central_derivatives(None, 8, [1e-5], dT=1e-4)
    with pytest.raises(ValueError):
        thermo.central_derivatives(None, 8, [0.5], dT=0.0)
