"""Host-side plumbing of paper_2004_08669_gb300.autograd (no GPU): with the
library replaced by a fake whose f(beta) and df/dbeta are closed forms, the
autograd function must return f and route the gradient through df/dbeta."""
import math

import pytest
import torch

from paper_2004_08669_gb300 import autograd as AG


class _FakeHandle:
    calls = []

    def __init__(self, spins, m, beta, device="cuda:0"):
        self.beta = beta
        _FakeHandle.calls.append(("init", m, beta))

    def run(self, max_steps):
        _FakeHandle.calls.append(("run", max_steps))

    def observables(self):
        return {"f": math.sin(self.beta), "converged": 1}

    def df_dbeta(self):
        _FakeHandle.calls.append(("df",))
        return math.cos(self.beta)

    def close(self):
        _FakeHandle.calls.append(("close",))


class _FakeLib:
    CTMRG = _FakeHandle


def test_forward_and_backward_route_through_the_library(monkeypatch):
    monkeypatch.setattr(AG, "_library", lambda: _FakeLib)
    _FakeHandle.calls.clear()
    beta = torch.tensor(0.7, dtype=torch.float64, requires_grad=True)
    f = AG.free_energy(beta, spins=None, m=8, max_steps=17)
    assert f.item() == pytest.approx(math.sin(0.7), rel=1e-15)
    (g,) = torch.autograd.grad(3.0 * f, beta)
    assert g.item() == pytest.approx(3.0 * math.cos(0.7), rel=1e-15)
    assert ("run", 17) in _FakeHandle.calls and ("df",) in _FakeHandle.calls
    assert _FakeHandle.calls[-1] == ("close",)


def test_no_derivative_without_requires_grad(monkeypatch):
    monkeypatch.setattr(AG, "_library", lambda: _FakeLib)
    _FakeHandle.calls.clear()
    f = AG.free_energy(torch.tensor(0.3, dtype=torch.float64), spins=None, m=4)
    assert f.item() == pytest.approx(math.sin(0.3))
    assert ("df",) not in _FakeHandle.calls


def test_unconverged_run_raises_and_closes(monkeypatch):
    class Slow(_FakeHandle):
        def observables(self):
            return {"f": 0.0, "converged": 0}

    class Lib:
        CTMRG = Slow

    monkeypatch.setattr(AG, "_library", lambda: Lib)
    _FakeHandle.calls.clear()
    with pytest.raises(RuntimeError):
        AG.free_energy(torch.tensor(0.5, dtype=torch.float64, requires_grad=True), spins=None, m=4)
    assert _FakeHandle.calls[-1] == ("close",)
