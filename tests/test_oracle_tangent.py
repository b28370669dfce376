"""Pins of the forward-mode beta derivative of the CTMRG fixed point
(oracle/tangent.py) to what the mathematics fixes:
- the weight's derivative against central differences of the oracle's own W;
- first-order eigen-perturbation against central differences of LAPACK's
  eigh on a matrix with exact doublets (simple pairs and the doublets'
  projectors);
- q = 2: the specific heat C = du/dT and dM/dT against the exact derivatives
  of Onsager's u and Yang's M, and df/dT = (f - u)/T;
- beta = 0: the first-order energy du/dbeta = -2/dim (a bond's own weight is
  the only first-order correlation; the vertex vectors of every model here
  form a spherical 2-design), dM/dbeta = 0 and d ln kappa/dbeta = 0;
- u = d(beta f)/dbeta with u from the bond expectation and d(beta f)/dbeta
  from the tangent of the growth factor;
- central differences (Richardson-extrapolated) of the converged C oracle for
  models without a closed form;
- planted mistakes (the coupling to discarded states dropped, the weight's
  derivative dropped) fail these pins."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from oracle import tangent as TG
from paper_2004_08669_gb300 import workloads as W
from tests import exact as E

MODELS = {"ising": W.ising, "clock3": lambda: W.clock(3), "cube": W.cube, "dodecahedron": W.dodecahedron}


def converged(spins, m, beta, max_steps=3000):
    t = TG.TangentCTMRG(spins, m, beta)
    hist = t.run(max_steps, 1e-13, 1e-11)
    assert hist[-1]["delta"] < 1e-12 and hist[-1]["delta_tangent"] < 1e-10, hist[-1]
    return t.observables()


# --- pieces --------------------------------------------------------------------

@pytest.mark.parametrize("model", sorted(MODELS))
def test_weight_exponent_is_the_log_derivative_of_w(model):
    spins = MODELS[model]()
    e = TG.weight_exponent(spins)
    b, h = 0.7, 1e-5
    for bond in (False, True):
        w = O.weight_matrix(spins, b, bond)
        fd = (O.weight_matrix(spins, b + h, bond) - O.weight_matrix(spins, b - h, bond)) / (2 * h)
        np.testing.assert_allclose(w * e, fd, rtol=1e-8, atol=1e-9 * np.abs(fd).max())


def test_eig_tangent_matches_central_differences_of_lapack():
    rng = np.random.default_rng(5)
    n = 12
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.array([5.0, -4.0, 3.0, 3.0, 2.5, 2.0, -1.5, 1.0, 0.5, 0.5, 0.2, 0.1])
    A = Q @ np.diag(lam) @ Q.T
    B = rng.standard_normal((n, n))
    A_dot = B + B.T
    ev, Z = O.eigh(A)
    ld, Zd = TG._eig_tangent(ev, Z, A_dot, n, 1e-10)
    h = 1e-6

    def lapack(eps):
        w, V = np.linalg.eigh(A + eps * A_dot)
        o = np.argsort(-np.abs(w), kind="stable")
        return w[o], V[:, o]

    (wp, Vp), (wm, Vm) = lapack(h), lapack(-h)
    simple = [0, 1, 4, 5, 6, 7, 10, 11]
    for i in simple:
        assert ld[i] == pytest.approx((wp[i] - wm[i]) / (2 * h), abs=1e-7)
        vp = Vp[:, i] * np.sign(Vp[:, i] @ Z[:, i])
        vm = Vm[:, i] * np.sign(Vm[:, i] @ Z[:, i])
        np.testing.assert_allclose(Zd[:, i], (vp - vm) / (2 * h), atol=1e-7)
    for c in ((2, 3), (8, 9)):
        c = list(c)
        # the doublet's projector and the sum of its eigenvalues are smooth
        Pd = Zd[:, c] @ Z[:, c].T + Z[:, c] @ Zd[:, c].T
        fdP = (Vp[:, c] @ Vp[:, c].T - Vm[:, c] @ Vm[:, c].T) / (2 * h)
        np.testing.assert_allclose(Pd, fdP, atol=1e-7)
        assert ld[c].sum() == pytest.approx((wp[c].sum() - wm[c].sum()) / (2 * h), abs=1e-7)


def test_primal_follows_the_c_oracle():
    """The tangent run takes the C oracle's primal steps."""
    t = TG.TangentCTMRG(W.dodecahedron(), 4, 1 / 0.5)
    c = O.CTMRG(W.dodecahedron(), 4, 1 / 0.5)
    for _ in range(25):
        a, b = t.step(), c.step()
        assert a["kappa"] == pytest.approx(b["kappa"], rel=1e-12)
        assert a["m_eff"] == b["m_eff"]
    P, om, live = c.get_state()
    assert live == t.live
    np.testing.assert_allclose(np.abs(t.omega), np.abs(om), atol=1e-12)


# --- exact values ----------------------------------------------------------------

@pytest.mark.parametrize("T", [1.8, 3.0])
def test_ising_specific_heat_and_dm_dt_are_exact(T):
    """q = 2 is the Ising model at K = beta; off-critical at m = 16 the CTMRG
    is exact to ~1e-13, and so are its derivatives: C = -K^2 du/dK,
    dM/dT = -K^2 dM/dK, df/dT = -s = (f - u)/T."""
    K = 1.0 / T
    ob = converged(W.ising(), 16, K)
    assert ob["C"] == pytest.approx(-K * K * E.onsager_du_dK(K), rel=1e-9)
    assert ob["dM_dT"] == pytest.approx(-K * K * E.yang_dm_dK(K), abs=1e-9)
    assert ob["df_dT"] == pytest.approx((E.onsager_f(K) - E.onsager_u(K)) / T, rel=1e-10)
    assert ob["d_beta_f_dbeta"] == pytest.approx(E.onsager_u(K), rel=1e-11)


@pytest.mark.parametrize("model", sorted(MODELS))
def test_beta_zero_first_order_energy(model):
    spins = MODELS[model]()
    t = TG.TangentCTMRG(spins, 6, 0.0)
    for _ in range(4):
        t.step()
    ob = t.observables()
    dim = spins.shape[1]
    assert ob["du_dbeta"] == pytest.approx(-2.0 / dim, abs=1e-12)
    assert abs(ob["dM_dbeta"]) < 1e-12
    assert abs(ob["dlnkappa_dbeta"]) < 1e-12
    assert ob["kappa"] == pytest.approx(spins.shape[0] ** 2, rel=1e-13)


# --- thermodynamic identity and finite differences --------------------------------

FD_CASES = [("clock3", 12, 0.5), ("cube", 8, 1 / 0.5), ("dodecahedron", 6, 1 / 0.5)]


def oracle_obs(spins, m, beta):
    c = O.CTMRG(spins, m, beta)
    hist = c.run(5000, 1e-13)
    assert hist[-1]["delta"] < 1e-12
    return c.observables()


@pytest.mark.parametrize("model,m,beta", FD_CASES)
def test_tangent_matches_central_differences_of_the_c_oracle(model, m, beta):
    """Richardson-extrapolated central differences of the converged C oracle
    at beta +- h and beta +- h/2 (error O(h^4) plus the convergence floor
    ~1e-13 / h) against the tangent; and u = d(beta f)/dbeta."""
    spins = MODELS[model]()
    ob = converged(spins, m, beta)
    h = 2e-4 * beta
    g = {s: oracle_obs(spins, m, beta + s) for s in (-h, -h / 2, h / 2, h)}
    keys = {"df_dbeta": "f", "du_dbeta": "u_kept", "dM_dbeta": "M_kept", "dS_dbeta": "S_E_kept"}
    for k, ok in keys.items():
        d1 = (g[h][ok] - g[-h][ok]) / (2 * h)
        d2 = (g[h / 2][ok] - g[-h / 2][ok]) / h
        rich = (4.0 * d2 - d1) / 3.0
        assert ob[k] == pytest.approx(rich, rel=1e-7, abs=1e-8), (k, ob[k], rich)
    assert ob["d_beta_f_dbeta"] == pytest.approx(ob["u"], rel=1e-10)


# --- planted mistakes ----------------------------------------------------------------

def test_planted_kept_only_eigen_coupling_fails(monkeypatch):
    """Dropping the kept states' coupling to the discarded ones (j over the
    kept block only) moves dM/dbeta and du/dbeta (by 3e-4 and 1e-3 here) far
    beyond the finite-difference pin's tolerance (1e-7 relative).  (The growth factor's derivative, and with it
    u = d(beta f)/dbeta, does not notice: at the fixed point kappa is
    stationary under a rotation of the kept subspace.)"""
    spins, m, beta = W.cube(), 8, 1 / 0.5
    good = converged(spins, m, beta)
    real = TG._eig_tangent

    def kept_only(ev, Z, A_dot, n, tol_c):
        H = Z.T @ A_dot @ Z
        lam_dot, _ = real(ev, Z, A_dot, n, tol_c)
        gap = ev[None, :n] - ev[:n, None]
        tiny = np.abs(gap) <= tol_c * abs(ev[0])
        Fm = np.where(tiny, 0.0, H[:n, :n] / np.where(tiny, 1.0, gap))
        return lam_dot, Z[:, :n] @ Fm

    monkeypatch.setattr(TG, "_eig_tangent", kept_only)
    t = TG.TangentCTMRG(spins, m, beta)
    t.run(3000, 1e-13, 1e-11)
    bad = t.observables()
    for k in ("dM_dbeta", "du_dbeta"):
        assert abs(bad[k] - good[k]) > 1e-5 * abs(good[k]), k


def test_planted_missing_weight_derivative_fails():
    K = 1 / 1.8
    t = TG.TangentCTMRG(W.ising(), 16, K)
    t.w_dot = np.zeros_like(t.w_dot)
    t.run(3000, 1e-13, 1e-11)
    ob = t.observables()
    assert abs(ob["C"] + K * K * E.onsager_du_dK(K)) > 1e-3
    assert not math.isclose(ob["d_beta_f_dbeta"], E.onsager_u(K), rel_tol=1e-6)


# --- implicit fixed-point derivative ------------------------------------------------

def test_gmres_solves_a_nonsymmetric_system():
    rng = np.random.default_rng(11)
    n = 40
    A = np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)
    b = rng.standard_normal(n)
    x, iters, res = TG._gmres(lambda v: A @ v, b, 1e-13, n)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11, atol=1e-11)
    assert res <= 1e-13 and iters <= n


def test_procrustes_alignment_undoes_cluster_rotations_and_signs():
    rng = np.random.default_rng(12)
    Z_ref, _ = np.linalg.qr(rng.standard_normal((10, 5)))
    ev = np.array([4.0, 2.0, 2.0, 2.0, -1.0])
    G, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    Z = Z_ref.copy()
    Z[:, 1:4] = Z_ref[:, 1:4] @ G
    Z[:, 0] *= -1.0
    Z[:, 4] *= -1.0
    Za, rot = TG._align(Z, Z_ref, ev, 1e-10)
    np.testing.assert_allclose(Za, Z_ref, atol=1e-14)
    assert [c for c, _ in rot] == [[0], [1, 2, 3], [4]]


@pytest.mark.parametrize("model,m,beta", [("cube", 8, 1 / 0.5), ("ising", 16, 1 / 1.8)])
def test_implicit_derivative_equals_the_unrolled_one(model, m, beta):
    spins = MODELS[model]()
    unrolled = converged(spins, m, beta)
    t = TG.TangentCTMRG(spins, m, beta)
    t.run_primal(3000, 1e-13)
    info = t.fixed_point_derivative()
    assert info["residual"] <= 1e-12
    implicit = t.observables()
    for k in ("df_dbeta", "du_dbeta", "dM_dbeta", "dS_dbeta"):
        assert implicit[k] == pytest.approx(unrolled[k], rel=1e-8, abs=1e-12), k


def test_implicit_derivative_at_an_unstable_fixed_point():
    """q = 20, m = 8, T = 0.5: the converged state is unstable (continued
    iteration amplifies the rounding noise), so the unrolled tangent cannot
    converge; the implicit solve gives the derivative of that branch, which
    Richardson differences of primal runs stopped on the branch (delta <
    1e-12, reached before the drift) reproduce."""
    spins, m, beta = W.dodecahedron(), 8, 1 / 0.5
    t = TG.TangentCTMRG(spins, m, beta)
    hist = t.run_primal(3000, 1e-12)
    assert hist[-1]["delta"] < 1e-12
    probe = TG.TangentCTMRG(spins, m, beta)
    probe.run_primal(3000, 1e-12)
    drift = probe.run_primal(150, 0.0)
    assert max(r["delta"] for r in drift[-10:]) > 1e3 * hist[-1]["delta"]
    t.fixed_point_derivative()
    ob = t.observables()
    assert ob["d_beta_f_dbeta"] == pytest.approx(ob["u"], rel=1e-10)

    def on_branch(b):
        c = TG.TangentCTMRG(spins, m, b)
        assert c.run_primal(3000, 1e-12)[-1]["delta"] < 1e-12
        return c.observables()

    h = 2e-4 * beta
    g = {s: on_branch(beta + s) for s in (-h, -h / 2, h / 2, h)}
    for k, ok in (("df_dbeta", "f"), ("du_dbeta", "u"), ("dM_dbeta", "M"), ("dS_dbeta", "S_E")):
        d1 = (g[h][ok] - g[-h][ok]) / (2 * h)
        d2 = (g[h / 2][ok] - g[-h / 2][ok]) / h
        assert ob[k] == pytest.approx((4.0 * d2 - d1) / 3.0, rel=1e-7), k
