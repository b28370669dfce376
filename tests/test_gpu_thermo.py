"""Temperature derivatives through the scan (paper_2004_08669_gb300.thermo)
against the exact Ising ones.

q = 2 is the Ising model at K = 1/T; Onsager's energy u(K) and Yang's
magnetisation M(K) are closed forms, so their central differences with the
same dT are what the scan's central differences must give: the specific
heat C = du/dT and dM/dT agree up to the CTMRG error of u and M (about
1e-11) divided by 2 dT.  The GPU's bond-expectation energy must also equal
its own d(beta f)/d beta.

q = 20 has no closed form: there the scan's central differences are held
against the oracle's forward-mode derivative of the fixed point
(oracle/tangent.py), which the CPU tests pin to the exact Ising derivatives.
"""
import pytest

from paper_2004_08669_gb300 import workloads as W
from tests import exact as E

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_08669_gb300 import build
    build.build()
    from paper_2004_08669_gb300 import ctm as C
    return C


def test_ising_specific_heat_and_magnetisation_slope(ctm):
    from paper_2004_08669_gb300 import thermo
    dT = 1e-4
    temps = [1.8, 3.0]  # ordered (K = 0.556) and disordered (K = 0.333)
    rows = thermo.central_derivatives(W.ising(), 16, temps, dT=dT, workers=6)
    for r in rows:
        T = r["T"]
        assert r["converged"]
        u_ex = lambda t: E.onsager_u(1.0 / t)  # noqa: E731
        m_ex = lambda t: E.yang_m(1.0 / t)  # noqa: E731
        C_ex = (u_ex(T + dT) - u_ex(T - dT)) / (2 * dT)
        dM_ex = (m_ex(T + dT) - m_ex(T - dT)) / (2 * dT)
        print(f"\nT = {T}: C = {r['C']:.10f} (exact {C_ex:.10f}), dM/dT = {r['dM_dT']:.10f} (exact {dM_ex:.10f})")
        assert r["u"] == pytest.approx(E.onsager_u(1.0 / T), rel=1e-11)
        assert r["u_fd"] == pytest.approx(r["u"], rel=1e-7)
        assert r["C"] == pytest.approx(C_ex, rel=1e-6)
        assert r["dM_dT"] == pytest.approx(dM_ex, rel=1e-6, abs=1e-7)


def test_dodecahedron_derivatives_match_the_oracle_tangent(ctm):
    """q = 20, m = 8 at T = 0.44 and 0.6: C and dM/dT from the GPU scan's
    central differences (dT = 1e-4, each temperature converged to delta <
    1e-12) against the oracle's exact tangent.  The difference is the
    O(dT^2) error plus the convergence floor over 2 dT; the C oracle's own
    central differences with the same dT and stopping rule differ from the
    tangent by 1e-7 (C) and 7e-7 (dM/dT) relative."""
    from oracle import tangent as TG
    from paper_2004_08669_gb300 import thermo
    temps = [0.44, 0.6]
    rows = thermo.central_derivatives(W.dodecahedron(), 8, temps, dT=1e-4, workers=6)
    for r in rows:
        t = TG.TangentCTMRG(W.dodecahedron(), 8, 1.0 / r["T"])
        hist = t.run(3000, 1e-13, 1e-11)
        assert hist[-1]["delta_tangent"] < 1e-10
        ob = t.observables()
        print(f"\nT = {r['T']}: C = {r['C']:.10f} (tangent {ob['C']:.10f}), "
              f"dM/dT = {r['dM_dT']:.10f} (tangent {ob['dM_dT']:.10f})")
        assert r["converged"]
        assert r["u"] == pytest.approx(ob["u"], rel=1e-9)
        assert r["C"] == pytest.approx(ob["C"], rel=1e-5)
        assert r["dM_dT"] == pytest.approx(ob["dM_dT"], rel=1e-5)
        assert r["u_fd"] == pytest.approx(ob["d_beta_f_dbeta"], rel=1e-6)
