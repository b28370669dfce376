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


# --- reverse mode -------------------------------------------------------------------

def test_pindex2_adjoint_is_the_transpose():
    rng = np.random.default_rng(13)
    a, b, c = 3, 4, 5
    A = np.asfortranarray(rng.standard_normal((a * b, c)))
    B_bar = np.asfortranarray(rng.standard_normal((a, c * b)))
    assert (B_bar * O.pindex2(A, a, b, c)).sum() == pytest.approx((TG._pindex2_adjoint(B_bar, a, b, c) * A).sum(),
                                                                 rel=1e-14)


def test_eig_vjp_is_the_transpose_of_eig_tangent():
    rng = np.random.default_rng(14)
    n = 10
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev_in = np.array([4.0, -3.0, 2.0, 2.0, 1.5, 1.0, 0.7, 0.7, 0.3, 0.1])
    ev, Z = O.eigh(Q @ np.diag(ev_in) @ Q.T)
    B = rng.standard_normal((n, n))
    A_dot = B + B.T
    k = 6
    lam_dot, Z_dot = TG._eig_tangent(ev, Z, A_dot, k, 1e-10)
    lam_bar, Z_bar = rng.standard_normal(k), rng.standard_normal((n, k))
    lhs = lam_bar @ lam_dot + (Z_bar * Z_dot).sum()
    rhs = (TG._eig_vjp(ev, Z, lam_bar, Z_bar, k, 1e-10) * A_dot).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def twisted_reference(t, pr0, angle=0.7):
    """pr0's kept basis with every multiplet's columns turned by a fixed
    angle (pairs) or orthogonal matrix, so that aligning onto it takes a
    rotation that is not symmetric."""
    U = pr0["U"].copy()
    idx, meff = pr0["idx"], pr0["meff"]
    rng = np.random.default_rng(17)
    for c in TG._clusters(pr0["ev"][:meff], t.tol_c):
        if len(c) > 1:
            G, _ = np.linalg.qr(rng.standard_normal((len(c), len(c))))
            if len(c) == 2:
                G = np.array([[np.cos(angle), -np.sin(angle)], [np.sin(angle), np.cos(angle)]])
            sub = U[np.ix_(idx, c)] @ G
            U[np.ix_(idx, c)] = sub
    return U


REVERSE_CASES = [("clock3", 6, 0.5, 5), ("dodecahedron", 4, 1 / 0.5, 8), ("cube", 8, 1 / 0.5, 12),
                 ("ising", 16, 1 / 1.8, 30)]


@pytest.mark.parametrize("model,m,beta,steps", REVERSE_CASES)
@pytest.mark.parametrize("rotated", [False, True])
def test_reverse_step_is_the_transpose_of_the_tangent_step(model, m, beta, steps, rotated):
    """<y_bar, J x_dot> = <J^t y_bar, x_dot> for one step, J with W's beta
    dependence as a third input, with and without the gauge rotation onto a
    reference basis."""
    spins = MODELS[model]()
    t = TG.TangentCTMRG(spins, m, beta)
    t.run_primal(steps, 0.0)
    pr0 = t._primal(t.P, t.omega, t.live)
    pr = t._primal(pr0["P_new"], pr0["omega_new"], pr0["meff"], twisted_reference(t, pr0) if rotated else None)
    assert (pr["rot"] is not None) == rotated
    rng = np.random.default_rng(15)
    N = t.N
    P_dot = np.asfortranarray(rng.standard_normal((m, N)))
    om_dot = np.zeros(N)
    om_dot[:m] = rng.standard_normal(m)
    Pn_dot, on_dot, k_dot = t._tangent(pr, P_dot, om_dot, True)
    P_bar = np.asfortranarray(rng.standard_normal((m, N)))
    om_bar = np.zeros(N)
    om_bar[: pr["meff"]] = rng.standard_normal(pr["meff"])
    k_bar = float(rng.standard_normal())
    Pb, ob, bb = t._vjp(pr, P_bar, om_bar, k_bar, True)
    lhs = (P_bar * Pn_dot).sum() + om_bar @ on_dot + k_bar * k_dot
    rhs = (Pb * P_dot).sum() + ob @ om_dot + bb
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("model,m,beta", [("cube", 8, 1 / 0.5), ("ising", 16, 1 / 1.8)])
def test_adjoint_fixed_point_equals_forward(model, m, beta):
    """d ln kappa / d beta through the adjoint equation (I - J^t) x_bar = g
    equals the forward implicit derivative; for Ising it is -2 u (ln kappa =
    -2 beta f) with Onsager's u."""
    spins = MODELS[model]()
    t = TG.TangentCTMRG(spins, m, beta)
    t.run_primal(3000, 1e-13)
    rev = t.adjoint_dlnkappa_dbeta()
    assert rev["residual"] <= 1e-12
    t.fixed_point_derivative()
    assert rev["dlnkappa_dbeta"] == pytest.approx(t.kappa_dot / t.kappa, rel=1e-9)
    if model == "ising":
        assert rev["dlnkappa_dbeta"] == pytest.approx(-2.0 * E.onsager_u(beta), rel=1e-10)


def test_planted_untransposed_gauge_rotation_fails_the_transpose_test(monkeypatch):
    """Rotating the eigenvector cotangent by R instead of R^t breaks the
    transpose identity wherever a cluster's rotation is not symmetric (a
    C3v doublet of the q = 20 corner, turned against a twisted reference)."""
    spins, m, beta = W.dodecahedron(), 4, 1 / 0.5
    t = TG.TangentCTMRG(spins, m, beta)
    t.run_primal(8, 0.0)
    pr0 = t._primal(t.P, t.omega, t.live)
    # a 2 x 2 reflection is symmetric: pick the twist that makes the
    # doublet's alignment a proper rotation
    for flip in (False, True):
        U_ref = twisted_reference(t, pr0)
        if flip:
            c = next(c for c in TG._clusters(pr0["ev"][: pr0["meff"]], t.tol_c) if len(c) == 2)
            U_ref[pr0["idx"], c[1]] *= -1.0
        pr = t._primal(pr0["P_new"], pr0["omega_new"], pr0["meff"], U_ref)
        if any(len(c) == 2 and abs(Rc[0, 1] - Rc[1, 0]) > 0.1 for c, Rc in pr["rot"]):
            break
    else:
        raise AssertionError("no doublet rotation that is not symmetric")
    real_rotate = TG._rotate

    def wrong_rotate(Z_dot, rot):
        return real_rotate(Z_dot, [(c, Rc.T) for c, Rc in rot])

    rng = np.random.default_rng(16)
    N = t.N
    P_dot = np.asfortranarray(rng.standard_normal((m, N)))
    om_dot = np.zeros(N)
    Pn_dot, on_dot, k_dot = t._tangent(pr, P_dot, om_dot, False)
    P_bar = np.asfortranarray(rng.standard_normal((m, N)))
    om_bar = np.zeros(N)
    monkeypatch.setattr(TG, "_rotate", wrong_rotate)
    Pb, ob, _ = t._vjp(pr, P_bar, om_bar, 0.0, False)
    lhs = (P_bar * Pn_dot).sum()
    rhs = (Pb * P_dot).sum()
    assert abs(lhs - rhs) > 1e-6 * abs(lhs)


# --- the eigen tangent from a Ritz block (what the GPU's subspace iteration has) --

def q20_corner(m=8, T=0.44, steps=40):
    t = TG.TangentCTMRG(W.dodecahedron(), m, 1.0 / T, ritz_block=m + max(8, m // 8))
    t.run_primal(steps, 0.0)
    pr0 = t._primal(t.P, t.omega, t.live)
    return t, t._primal(pr0["P_new"], pr0["omega_new"], pr0["meff"], pr0["U"])


def test_block_eigen_tangent_equals_the_full_spectrum_one():
    """From the leading b = m + 8 eigenpairs and the deflated iteration
    (rate |lambda_b / lambda_m|, 0.40 here) the kept pairs' tangent equals
    the one coupled to the whole live spectrum, on a q = 20 corner."""
    t, pr = q20_corner()
    rng = np.random.default_rng(18)
    L = len(pr["ev"])
    B = rng.standard_normal((L, L))
    A_dot = B + B.T
    n, b = pr["meff"], t.ritz_block
    ld, Zd = TG._eig_tangent(pr["ev"], pr["Z"], A_dot, n, t.tol_c)
    ld_b, Zd_b, it = TG._eig_tangent_block(pr["A"], pr["ev"], pr["Z"], A_dot, n, b, t.tol_c)
    rate = abs(pr["ev"][b] / pr["ev"][n - 1])
    assert rate < 0.5 and it <= int(np.log(1e-14) / np.log(rate)) + 8
    np.testing.assert_allclose(ld_b, ld, rtol=1e-12, atol=1e-12 * np.abs(ld).max())
    np.testing.assert_allclose(Zd_b, Zd, atol=1e-12 * np.abs(Zd).max())
    lam_bar, Z_bar = rng.standard_normal(n), rng.standard_normal((L, n))
    lhs = lam_bar @ ld_b + (Z_bar * Zd_b).sum()
    rhs = (TG._eig_vjp_block(pr["A"], pr["ev"], pr["Z"], lam_bar, Z_bar, n, b, t.tol_c) * A_dot).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_block_step_is_transposed_and_equals_the_full_step():
    t, pr = q20_corner(m=6, T=0.5)
    full = TG.TangentCTMRG(W.dodecahedron(), 6, 1 / 0.5)
    rng = np.random.default_rng(19)
    N = t.N
    P_dot = np.asfortranarray(rng.standard_normal((6, N)))
    om_dot = np.zeros(N)
    om_dot[:6] = rng.standard_normal(6)
    Pn, on, kd = t._tangent(pr, P_dot, om_dot, True)
    Pn_f, on_f, kd_f = full._tangent(pr, P_dot, om_dot, True)
    np.testing.assert_allclose(Pn, Pn_f, atol=1e-12 * np.abs(Pn_f).max())
    assert kd == pytest.approx(kd_f, rel=1e-12)
    P_bar = np.asfortranarray(rng.standard_normal((6, N)))
    om_bar = np.zeros(N)
    om_bar[: pr["meff"]] = rng.standard_normal(pr["meff"])
    Pb, ob, bb = t._vjp(pr, P_bar, om_bar, 0.3, True)
    lhs = (P_bar * Pn).sum() + om_bar @ on + 0.3 * kd
    rhs = (Pb * P_dot).sum() + ob @ om_dot + bb
    assert lhs == pytest.approx(rhs, rel=1e-12)


@pytest.mark.parametrize("model,m,beta", [("cube", 8, 1 / 0.5), ("ising", 16, 1 / 1.8)])
def test_ritz_block_run_gives_the_same_derivatives(model, m, beta):
    spins = MODELS[model]()
    full = converged(spins, m, beta)
    t = TG.TangentCTMRG(spins, m, beta, ritz_block=m + max(8, m // 8))
    t.run(3000, 1e-13, 1e-11)
    blk = t.observables()
    assert t.block_iterations > 0
    for k in ("df_dbeta", "du_dbeta", "dM_dbeta", "dS_dbeta"):
        assert blk[k] == pytest.approx(full[k], rel=1e-11, abs=1e-13), k


@pytest.mark.parametrize("model,m,beta", [("cube", 8, 1 / 0.5), ("dodecahedron", 6, 1 / 0.5), ("ising", 16, 1 / 1.8)])
def test_adjoint_observables_equal_forward(model, m, beta):
    """Reverse mode of M, u and S_E (their cotangents at the fixed point and
    the adjoint equation) gives the forward implicit derivatives; for Ising
    they are Yang's dM/dK and Onsager's du/dK."""
    spins = MODELS[model]()
    fw = TG.TangentCTMRG(spins, m, beta)
    fw.run_primal(3000, 1e-13)
    fw.fixed_point_derivative()
    ob = fw.observables()
    t = TG.TangentCTMRG(spins, m, beta)
    t.run_primal(3000, 1e-13)
    rev = {"dM_dbeta": t.adjoint_observables(M_bar=1.0)["derivative"],
           "du_dbeta": t.adjoint_observables(u_bar=1.0)["derivative"],
           "dS_dbeta": t.adjoint_observables(S_bar=1.0)["derivative"]}
    for k, v in rev.items():
        assert v == pytest.approx(ob[k], rel=1e-9, abs=1e-13), k
    if model == "ising":
        assert rev["dM_dbeta"] == pytest.approx(E.yang_dm_dK(beta), rel=1e-9)
        assert rev["du_dbeta"] == pytest.approx(E.onsager_du_dK(beta), rel=1e-9)


def test_cube_derivatives_are_three_isings():
    """q = 8 is three Ising models at K = beta / 3: M = M_Yang(K) and u =
    u_Onsager(K) per spin, so dM/dbeta = Yang'(K) / 3 and du/dbeta =
    Onsager's du/dK / 3.  At T = 0.5 the tangent's error falls from ~1e-5 at
    m = 8 to ~1e-12 at m = 24 (the truncation of the product spectrum)."""
    beta = 1 / 0.5
    K = beta / 3
    dM_ex, du_ex = E.yang_dm_dK(K) / 3, E.onsager_du_dK(K) / 3
    errs = []
    for m in (8, 24):
        ob = converged(W.cube(), m, beta)
        errs.append((abs(ob["dM_dbeta"] / dM_ex - 1), abs(ob["du_dbeta"] / du_ex - 1)))
    assert errs[1][0] < 1e-10 and errs[1][1] < 1e-10
    assert errs[0][0] > 100 * errs[1][0] and errs[0][1] > 100 * errs[1][1]
