"""Parity of the GPU tangent step (ctm_tangent_step, FP64 form) with the
oracle's forward-mode step (oracle/tangent.py, pinned on the CPU to the exact
Ising derivatives, the beta = 0 energy and central differences).

The state and its input tangent come from the oracle's unrolled tangent run
(so the input respects the lattice symmetry, as every beta-tangent does).
The two sides pick their own bases for the new renormalised leg (signs, and
rotations inside exact multiplets), so the comparison is on what the basis
does not change: kappa, its tangent, the spectrum omega and its tangent, and
the traces of powers of P'^t diag(omega'^2) P' with their tangents.  The GPU
takes the eigen tangent from its Ritz block and a deflated iteration, the
oracle from the whole live spectrum; the two agree to rounding."""
import numpy as np
import pytest

from oracle import tangent as TG
from paper_2004_08669_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODELS = {"cube": W.cube, "dodecahedron": W.dodecahedron}


@pytest.fixture(scope="module")
def ctm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2004_08669_gb300 import build
    build.build()
    from paper_2004_08669_gb300 import ctm as C
    return C


def invariants(P, om, P_dot, om_dot):
    """tr G^k and d tr G^k (k = 1..3) for G = P'^t diag(omega'^2) P': both
    block legs of P' carry the new basis, so G changes by a conjugation and
    its traces do not."""
    om, om_dot = np.asarray(om), np.asarray(om_dot)
    w, wd = om ** 2, 2.0 * om * om_dot
    G = P.T @ (w[:, None] * P)
    Gd = P_dot.T @ (w[:, None] * P) + P.T @ (w[:, None] * P_dot) + P.T @ (wd[:, None] * P)
    t, dt, Gk = [], [], np.eye(len(G))
    for k in (1, 2, 3):
        dt.append(k * np.trace(Gk @ Gd))
        Gk = Gk @ G
        t.append(np.trace(Gk))
    return np.array(t), np.array(dt)


@pytest.mark.parametrize("model,m,T,steps", [("dodecahedron", 8, 0.44, 20), ("dodecahedron", 6, 0.5, 15),
                                             ("cube", 8, 0.5, 10)])
def test_tangent_step_matches_the_oracle(ctm, model, m, T, steps):
    spins = MODELS[model]()
    t = TG.TangentCTMRG(spins, m, 1.0 / T)
    for _ in range(steps):
        t.step()
    pr = t._primal(t.P, t.omega, t.live)
    Pd_o, od_o, kd_o = t._tangent(pr, t.P_dot, t.omega_dot, True)
    g = ctm.CTMRG(spins, m, 1.0 / T, device="cuda:0")
    try:
        g.set_state(t.P, t.omega[:m], t.live)
        r = g.tangent_step(t.P_dot, t.omega_dot[:m], True)
    finally:
        g.close()
    print(f"\n{model} m={m} T={T}: m_eff {r['m_eff']}, Ritz pairs {r['ritz_pairs']}, deflated iterations "
          f"{r['deflate_iterations']}, kappa_dot {r['kappa_dot']:.12e} (oracle {kd_o:.12e})")
    assert r["m_eff"] == pr["meff"]
    assert r["kappa"] == pytest.approx(pr["nrm"], rel=1e-12)
    np.testing.assert_allclose(r["omega_new"], pr["omega_new"][:m], atol=1e-12)
    assert r["kappa_dot"] == pytest.approx(kd_o, rel=1e-9)
    np.testing.assert_allclose(r["omega_dot_new"], od_o[:m], atol=1e-9 * np.abs(od_o).max())
    t_g, dt_g = invariants(r["P_new"], r["omega_new"], r["P_dot_new"], r["omega_dot_new"])
    t_o, dt_o = invariants(pr["P_new"], pr["omega_new"][:m], Pd_o, od_o[:m])
    print(f"tr G^k {t_g} (oracle {t_o}), d tr G^k {dt_g} (oracle {dt_o})")
    np.testing.assert_allclose(t_g, t_o, rtol=1e-11)
    np.testing.assert_allclose(dt_g, dt_o, rtol=1e-8)


def test_unrolled_gpu_tangent_gives_the_oracle_derivative(ctm):
    """Stepping the GPU tangent from the initial state (each output fed back
    through ctm_set_state) reproduces the oracle's d ln kappa / d beta and
    the derivative of the spectrum after the fixed point has converged."""
    spins, m, beta, steps = W.cube(), 8, 1 / 0.5, 40
    t = TG.TangentCTMRG(spins, m, beta)
    for _ in range(steps):
        t.step()
    g = ctm.CTMRG(spins, m, beta, device="cuda:0")
    try:
        N = m * spins.shape[0]
        P = np.zeros((m, N), order="F")
        P[0, 0] = 1.0  # boundary spin 0 (Algorithm 3's initial state)
        om = np.zeros(m)
        om[0] = 1.0
        P_dot, om_dot, live = np.zeros((m, N), order="F"), np.zeros(m), 1
        for _ in range(steps):
            g.set_state(P, om, live)
            r = g.tangent_step(P_dot, om_dot, True)
            P, om, P_dot, om_dot, live = r["P_new"], r["omega_new"], r["P_dot_new"], r["omega_dot_new"], r["m_eff"]
    finally:
        g.close()
    assert live == t.live
    assert r["kappa"] == pytest.approx(t.kappa, rel=1e-11)
    assert r["kappa_dot"] / r["kappa"] == pytest.approx(t.kappa_dot / t.kappa, rel=1e-9)
    np.testing.assert_allclose(om_dot, t.omega_dot[:m], atol=1e-9 * np.abs(t.omega_dot).max())


def test_tangent_step_rejects_other_forms_and_bad_arguments(ctm):
    spins = W.dodecahedron()
    g = ctm.CTMRG(spins, 8, 1 / 0.44, prec="tf32", device="cuda:0")
    try:
        with pytest.raises(ctm.CtmError) as e:
            g.tangent_step(np.zeros((8, 160)), np.zeros(8))
        assert e.value.status == ctm.CTM_EUNSUPPORTED
    finally:
        g.close()
    g = ctm.CTMRG(spins, 8, 1 / 0.44, device="cuda:0")
    try:
        with pytest.raises(ValueError):
            g.tangent_step(np.zeros((8, 159)), np.zeros(8))
    finally:
        g.close()


@pytest.mark.parametrize("T", [0.44, 0.6])
def test_backward_free_energy_derivative_matches_the_oracle(ctm, T):
    """ctm_step_backward at the converged q = 20, m = 8 fixed point: df/dbeta
    by GMRES on (I - J) x = d(step)/dbeta with the GPU tangent step equals
    the oracle's fixed-point derivative, and f + beta df/dbeta equals the
    bond-expectation energy u (thermodynamics)."""
    spins, m, beta = W.dodecahedron(), 8, 1.0 / T
    t = TG.TangentCTMRG(spins, m, beta)
    assert t.run_primal(3000, 1e-13)[-1]["delta"] < 1e-13
    assert t.fixed_point_derivative()["residual"] <= 1e-12
    ob = t.observables()
    g = ctm.CTMRG(spins, m, beta, device="cuda:0")
    try:
        g.run(5000)
        o = g.observables()
        df = g.df_dbeta()
    finally:
        g.close()
    print(f"\nT = {T}: df/dbeta GPU {df:.12e}, oracle {ob['df_dbeta']:.12e}; f + beta df/dbeta "
          f"{o['f'] + beta * df:.12f}, u {o['u']:.12f}")
    assert df == pytest.approx(ob["df_dbeta"], rel=1e-8)
    assert o["f"] + beta * df == pytest.approx(o["u"], rel=1e-9)


def test_free_energy_autograd_function(ctm):
    """torch.autograd through the library: f(beta) at the converged q = 20,
    m = 8 fixed point and its gradient from ctm_step_backward, against the
    oracle's fixed point and implicit derivative."""
    import torch

    from paper_2004_08669_gb300 import autograd as AG
    spins, m, T = W.dodecahedron(), 8, 0.44
    t = TG.TangentCTMRG(spins, m, 1.0 / T)
    assert t.run_primal(3000, 1e-13)[-1]["delta"] < 1e-13
    t.fixed_point_derivative()
    ob = t.observables()
    beta = torch.tensor(1.0 / T, dtype=torch.float64, requires_grad=True)
    f = AG.free_energy(beta, spins, m)
    f.backward()
    assert f.item() == pytest.approx(ob["f"], rel=1e-12)
    assert beta.grad.item() == pytest.approx(ob["df_dbeta"], rel=1e-8)


def test_backward_observable_derivatives_match_the_oracle(ctm):
    """ctm_step_backward with the gradient of M, u or S_E: the observables'
    tangents at the fixed point along the implicit solution (the eigen
    tangent's dz and dlambda, and C~_h with its own beta-derivative) against
    the oracle's fixed-point derivative, at q = 20, m = 8, T = 0.44."""
    spins, m, T = W.dodecahedron(), 8, 0.44
    beta = 1.0 / T
    t = TG.TangentCTMRG(spins, m, beta)
    assert t.run_primal(3000, 1e-13)[-1]["delta"] < 1e-13
    t.fixed_point_derivative()
    ob = t.observables()
    g = ctm.CTMRG(spins, m, beta, device="cuda:0")
    try:
        g.run(5000)
        got = {}
        for name in ("M", "u", "S_E"):
            go = ctm.ctm_obs()
            setattr(go, name, 1.0)
            got[name] = ctm.ctm_step_backward(g.h, go)
    finally:
        g.close()
    print(f"\ndM/dbeta {got['M']:.12e} (oracle {ob['dM_dbeta']:.12e}), du/dbeta {got['u']:.12e} "
          f"(oracle {ob['du_dbeta']:.12e}), dS/dbeta {got['S_E']:.12e} (oracle {ob['dS_dbeta']:.12e})")
    assert got["M"] == pytest.approx(ob["dM_dbeta"], rel=1e-7)
    assert got["u"] == pytest.approx(ob["du_dbeta"], rel=1e-7)
    assert got["S_E"] == pytest.approx(ob["dS_dbeta"], rel=1e-7)
