"""Temperature derivatives through the scan (paper_2004_08669_gb300.thermo)
against the exact Ising ones.

q = 2 is the Ising model at K = 1/T; Onsager's energy u(K) and Yang's
magnetisation M(K) are closed forms, so their central differences with the
same dT are what the scan's central differences must give: the specific
heat C = du/dT and dM/dT agree up to the CTMRG error of u and M (about
1e-11) divided by 2 dT.  The GPU's bond-expectation energy must also equal
its own d(beta f)/d beta.
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
