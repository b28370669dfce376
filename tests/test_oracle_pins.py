"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these compares the oracle with itself: each checks a closed form,
a library routine, a brute-force enumeration, an exact special case or an
invariant, chosen so that a dropped term, a wrong index or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_08669_gb300 import workloads as W
from tests import exact as E


# --- model tables (Sec. I, Fig. 1) -------------------------------------------

def test_dodecahedron_dot_product_multiset():
    """From every vertex the 20 dot products are {1, 3 x sqrt5/3, 6 x 1/3,
    6 x -1/3, 3 x -sqrt5/3, -1}: the dodecahedron's vertex-distance shells."""
    v = W.dodecahedron()
    assert v.shape == (20, 3)
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    want = np.sort([1.0] + [math.sqrt(5) / 3] * 3 + [1 / 3] * 6 + [-1 / 3] * 6
                   + [-math.sqrt(5) / 3] * 3 + [-1.0])
    for s in range(20):
        np.testing.assert_allclose(np.sort(v @ v[s]), want, atol=1e-14)
    np.testing.assert_allclose(v.sum(axis=0), 0.0, atol=1e-14)
    np.testing.assert_allclose(v[0], np.ones(3) / math.sqrt(3), atol=1e-16)


def test_cube_dot_product_multiset():
    v = W.cube()
    want = np.sort([1.0, 1 / 3, 1 / 3, 1 / 3, -1 / 3, -1 / 3, -1 / 3, -1.0])
    for s in range(8):
        np.testing.assert_allclose(np.sort(v @ v[s]), want, atol=1e-15)


def test_weight_matrix_symmetries():
    """W is invariant under the plaquette's rotations and reflections, so its
    q^2 x q^2 matrix form is symmetric; a spin relabelling that preserves all
    dot products (an element of the point group) leaves it invariant."""
    v = W.dodecahedron()
    beta = 1 / 0.44
    w = O.weight_matrix(v, beta)
    np.testing.assert_allclose(w, w.T, rtol=1e-14)
    # 3-fold rotation about (1,1,1): (x,y,z) -> (y,z,x) permutes the vertices
    rot = v[:, [1, 2, 0]]
    perm = np.array([np.argmin(np.linalg.norm(v - r, axis=1)) for r in rot])
    assert sorted(perm.tolist()) == list(range(20))
    q = 20
    idx = (perm[:, None] + q * perm[None, :]).reshape(-1, order="F")
    np.testing.assert_allclose(w[np.ix_(idx, idx)], w, rtol=1e-13)
    # beta = 0: every weight is 1
    np.testing.assert_array_equal(O.weight_matrix(v, 0.0), np.ones((400, 400)))


def test_weight_matrix_ising_values():
    """Ising plaquette at coupling K: all four spins equal -> e^{4K}; one
    spin flipped -> 1; two opposite corners flipped -> e^{-4K}."""
    K = 0.37
    w = O.weight_matrix(W.ising(), K)
    # index (a + 2 b, c + 2 d), corners in cyclic order a, b, d, c; spin 0 = +1
    assert w[0, 0] == pytest.approx(math.exp(4 * K), rel=1e-15)
    assert w[1 + 0, 0] == pytest.approx(1.0, rel=1e-15)        # a flipped
    # a and d flipped (opposite corners of the cycle a,b,d,c): every bond broken
    assert w[1 + 0, 0 + 2 * 1] == pytest.approx(math.exp(-4 * K), rel=1e-15)
    # a and b flipped (neighbours): two bonds broken
    assert w[1 + 2 * 1, 0] == pytest.approx(1.0, rel=1e-15)


# --- index permutations (Algorithms 1 and 2) ---------------------------------

def test_pindex_against_tensor_transpose():
    rng = np.random.default_rng(1)
    a, b, c, d = 2, 3, 4, 5
    T = rng.standard_normal((a, b, c, d))
    A = T.reshape((a * b, c * d), order="F")
    B = O.pindex(A, a, b, c, d)
    # element by element on the 4-leg tensor: B_{(p,r),(q,s)} = A_{(p,q),(r,s)}
    for p in range(a):
        for qq in range(b):
            for r in range(c):
                for s in range(d):
                    assert B[p + a * r, qq + b * s] == T[p, qq, r, s]
    # applying the inverse permutation restores A
    np.testing.assert_array_equal(O.pindex(B, a, c, b, d), A)


def test_pindex2_against_tensor_transpose():
    rng = np.random.default_rng(2)
    a, b, c = 3, 4, 5
    T = rng.standard_normal((a, b, c))
    A = T.reshape((a * b, c), order="F")
    B = O.pindex2(A, a, b, c)
    for p in range(a):
        for qq in range(b):
            for r in range(c):
                assert B[p, r + c * qq] == T[p, qq, r]


# --- dense eigensolver --------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 17, 160, 400])
def test_eigh_against_lapack(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((n, n))
    A = A + A.T
    ev, Z = O.eigh(A)
    ref = np.linalg.eigvalsh(A)
    ref = ref[np.argsort(-np.abs(ref))]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(np.sort(ev), np.sort(ref), atol=1e-13 * n * scale)
    assert np.all(np.diff(np.abs(ev)) <= 1e-15 * scale)
    assert np.abs(A @ Z - Z * ev).max() <= 1e-13 * n * scale
    assert np.abs(Z.T @ Z - np.eye(n)).max() <= 1e-13 * n


def test_eigh_degenerate_clusters():
    rng = np.random.default_rng(7)
    Q, _ = np.linalg.qr(rng.standard_normal((60, 60)))
    d = np.repeat([5.0, 3.0, -3.0, 2.0, 1e-3, 0.0], 10)
    A = (Q * d) @ Q.T
    ev, Z = O.eigh(A)
    np.testing.assert_allclose(np.abs(ev[:10]), 5.0, rtol=1e-13)
    np.testing.assert_allclose(np.abs(ev[10:30]), 3.0, rtol=1e-13)
    assert np.abs(A @ Z - Z * ev).max() <= 1e-12
    assert np.abs(Z.T @ Z - np.eye(60)).max() <= 1e-12
    # projector onto the 5-cluster matches the planted one
    Pi = Z[:, :10] @ Z[:, :10].T
    Pi0 = Q[:, :10] @ Q[:, :10].T
    assert np.linalg.norm(Pi - Pi0, 2) <= 1e-12


# --- brute force: untruncated corners are exact CTMs ---------------------------

@pytest.mark.parametrize("model,kmax,m", [("ising", 4, 8), ("clock3", 3, 9), ("dodecahedron", 2, 20)])
def test_untruncated_corner_matches_brute_force(model, kmax, m):
    """While q^k <= m q nothing is truncated, and the extended corner after
    k-1 steps is the exact CTM of a k x k quadrant with fixed boundary."""
    spins = W.clock(3) if model == "clock3" else W.spins_for(model)
    q = spins.shape[0]
    beta = 0.7
    c = O.CTMRG(spins, m, beta, tol_cluster=0.0, tol_zero=0.0)
    for k in range(1, kmax + 1):
        Ct = c.extend()
        np.testing.assert_allclose(Ct, Ct.T, rtol=0, atol=1e-15 * np.abs(Ct).max())
        a = E.normalised_abs_spectrum(Ct, q ** k)
        b = E.normalised_abs_spectrum(E.brute_force_corner(spins, beta, k), q ** k)
        np.testing.assert_allclose(a, b, atol=1e-14)
        c.step()


def test_cube_untruncated_spectrum_is_three_isings():
    """v.v' for the cube is (s1 s1' + s2 s2' + s3 s3')/3, so the cube corner is
    the tensor product of three Ising corners at coupling beta/3."""
    beta = 1.1
    cc = O.CTMRG(W.cube(), 64, beta, tol_cluster=0.0, tol_zero=0.0)
    ci = O.CTMRG(W.ising(), 4, beta / 3, tol_cluster=0.0, tol_zero=0.0)
    for k in range(1, 3):
        a = E.normalised_abs_spectrum(cc.extend(), 8 ** k)
        e = E.normalised_abs_spectrum(ci.extend(), 2 ** k)
        prod = np.sort(np.abs(np.einsum("i,j,k->ijk", e, e, e).ravel()))[::-1]
        np.testing.assert_allclose(np.abs(a), prod, atol=1e-14)
        cc.step()
        ci.step()


# --- the whole iteration: Onsager, Yang ---------------------------------------

@pytest.mark.parametrize("beta", [0.3, 0.6])
def test_ising_free_energy_magnetisation_energy(beta):
    """q = 2 is the Ising model at K = beta (reading R2): Onsager's f and u,
    Yang's M; off-critical at m = 16 the CTMRG is exact to ~1e-13."""
    c = O.CTMRG(W.ising(), 16, beta)
    hist = c.run(2000, 1e-13)
    assert hist[-1]["delta"] < 1e-13
    ob = c.observables()
    assert ob["f"] == pytest.approx(E.onsager_f(beta), rel=1e-12)
    assert ob["M_kept"] == pytest.approx(E.yang_m(beta), abs=1e-12)
    assert ob["u_kept"] == pytest.approx(E.onsager_u(beta), rel=1e-11)
    assert ob["S_E_kept"] >= 0.0


@pytest.mark.parametrize("T", [1.2])
def test_cube_converged_close_to_three_isings(T):
    """f_cube(T) = f_Ising(K = 1/(3T)) per spin, M_cube = M_Yang(1/(3T));
    finite m limits the agreement, which must improve with m."""
    beta = 1.0 / T
    errs = []
    for m in (16, 32):
        c = O.CTMRG(W.cube(), m, beta)
        c.run(400, 1e-12)
        ob = c.observables()
        f_exact = -3.0 * E.onsager_minus_beta_f(beta / 3) / beta
        errs.append(abs(ob["f"] - f_exact) / abs(f_exact))
        assert ob["M_kept"] == pytest.approx(E.yang_m(beta / 3), abs=1e-3)
    assert errs[1] < errs[0] < 1e-4


# --- special cases --------------------------------------------------------------

def test_beta_zero_is_exact():
    """beta = 0: W = 1, every spin free: kappa = q^2 (f = -T ln q), the
    vertex vectors sum to zero so M = 0, and C~ has rank one (S_E = 0)."""
    c = O.CTMRG(W.dodecahedron(), 8, 0.0)
    for _ in range(4):
        r = c.step()
    assert r["kappa"] == pytest.approx(400.0, rel=1e-14)
    assert r["m_eff"] == 1
    ob = c.observables()
    assert abs(ob["M_kept"]) < 1e-14
    assert abs(ob["S_E_kept"]) < 1e-14


def test_low_temperature_limit():
    """T -> 0: all spins aligned with the boundary, two bonds of -1 per spin:
    f -> -2, u -> -2, M -> 1.  The lowest excitation costs about 1.02 (one
    spin moved to a neighbouring vertex breaks four bonds by 1 - sqrt5/3), so
    corrections at T = 0.05 are below 1e-8."""
    c = O.CTMRG(W.dodecahedron(), 8, 1 / 0.05)
    c.run(200, 1e-12)
    ob = c.observables()
    assert ob["f"] == pytest.approx(-2.0, abs=1e-8)
    assert ob["u_kept"] == pytest.approx(-2.0, abs=1e-6)
    assert ob["M_kept"] == pytest.approx(1.0, abs=1e-6)


# --- symmetry -------------------------------------------------------------------

def test_boundary_choice_invariance_and_exact_multiplets():
    """The point group acts transitively on the vertices: every boundary spin
    gives the same f, M and spectrum.  With the boundary fixed the residual
    symmetry is the vertex stabiliser C3v, whose irreps have dimension 1 or 2,
    so the converged spectrum consists of exact singlets and doublets."""
    v = W.dodecahedron()
    res = []
    for b in (0, 7, 13):
        c = O.CTMRG(v, 8, 1 / 0.5, boundary_spin=b)
        c.run(400, 1e-12)
        ob = c.observables()
        _, om, live = c.get_state()
        res.append((ob["f"], ob["M_kept"], np.abs(om[:live])))
    for f, M, om in res[1:]:
        assert f == pytest.approx(res[0][0], rel=1e-12)
        assert M == pytest.approx(res[0][1], rel=1e-10)
        np.testing.assert_allclose(om, res[0][2], atol=1e-10)
    om = res[0][2] / res[0][2][0]
    i, groups = 0, []
    while i < len(om):
        j = i + 1
        while j < len(om) and abs(om[j] - om[i]) < 1e-11:
            j += 1
        groups.append(j - i)
        i = j
    assert set(groups) <= {1, 2} and 2 in groups


def test_entropy_bounds():
    c = O.CTMRG(W.dodecahedron(), 8, 1 / 0.44)
    for _ in range(30):
        r = c.step()
        assert 0.0 <= r["S_E_kept"] <= math.log(r["m_eff"]) + 1e-12
        assert r["S_E_kept"] <= r["S_E_paper"] + 1e-12 or r["m_eff"] == r["live_dim"]
        assert r["S_E_paper"] <= math.log(r["live_dim"]) + 1e-12


# --- Baxter's exact corner spectrum (off-critical Ising) -----------------------

@pytest.mark.parametrize("T,m,tol_w", [(1.5, 32, 1e-11), (1.8, 32, 1e-9), (3.0, 32, 1e-9), (4.0, 32, 1e-11)])
def test_ising_kept_spectrum_and_entropy_match_baxter(T, m, tol_w):
    """The converged Ising corner on both sides of T_c = 2.269 against
    Baxter's exact corner transfer matrix spectrum: the normalised kept
    spectrum |w_i| / |w_1| = (rho_i / rho_1)^(1/4) (rho = C^4, Eq. 4), and
    S_E of Eq. (6) against the free-fermion entropy of the same levels.  Away
    from T_c the spectrum decays fast enough that m = 32 holds all of rho's
    weight above 1e-30, so S_E is exact to rounding."""
    K = 1.0 / T
    c = O.CTMRG(W.ising(), m, K)
    c.run(5000, 1e-13)
    _, om, _ = c.get_state()
    w = np.sort(np.abs(om[:m]))[::-1]
    w = w[w > 0]
    rho = E.baxter_rho_spectrum(K, len(w))
    np.testing.assert_allclose(w / w[0], (rho / rho[0]) ** 0.25, rtol=0, atol=tol_w)
    S = c.observables()["S_E_kept"]
    assert S == pytest.approx(E.baxter_entropy(K), abs=1e-13)
    assert S > 1e-4  # a non-trivial spectrum


def test_planted_entropy_power_fails_baxter():
    """The entropy with weights w^2 (or w^8) instead of w^4 = eigenvalues of
    rho~ = C~^4 misses Baxter's exact entropy by far more than the tolerance
    above, on both sides of T_c."""
    for T in (1.8, 3.0):
        K = 1.0 / T
        c = O.CTMRG(W.ising(), 32, K)
        c.run(5000, 1e-13)
        _, om, _ = c.get_state()
        exact = E.baxter_entropy(K)
        assert O.entropy(om[:32], 4) == pytest.approx(exact, abs=1e-13)
        for power in (2, 8):
            assert abs(O.entropy(om[:32], power) - exact) > 1e-3


# --- planted mistakes: each must fail a pin ------------------------------------

def _twisted_weight(spins, beta):
    """The literal reading of the matrix form of W (open legs exchanged)."""
    q = spins.shape[0]
    w = O.weight_matrix(spins, beta)
    cols = np.array([d + q * c for d in range(q) for c in range(q)]).reshape(q, q).T.ravel(order="F")
    return w[:, cols]


def test_planted_twisted_weight_fails_onsager():
    beta = 0.3
    c = O.CTMRG(W.ising(), 16, beta)
    c.set_weights(_twisted_weight(W.ising(), beta))
    c.run(2000, 1e-13)
    rel = abs(c.observables()["f"] - E.onsager_f(beta)) / abs(E.onsager_f(beta))
    assert rel > 1e-4


def test_planted_twisted_weight_fails_brute_force():
    spins, beta = W.clock(3), 0.7
    c = O.CTMRG(spins, 9, beta, tol_cluster=0.0, tol_zero=0.0)
    c.set_weights(_twisted_weight(spins, beta))
    c.step()
    a = E.normalised_abs_spectrum(c.extend(), 9)
    b = E.normalised_abs_spectrum(E.brute_force_corner(spins, beta, 2), 9)
    assert np.abs(a - b).max() > 1e-3


def test_planted_half_temperature_fails_onsager():
    """The every-plaquette convention beta/2 per bond would halve K."""
    beta = 0.6
    c = O.CTMRG(W.ising(), 16, beta)
    c.set_weights(O.weight_matrix(W.ising(), beta / 2))
    c.run(2000, 1e-13)
    assert abs(c.observables()["M_kept"] - E.yang_m(beta)) > 0.1


def test_ctilde_entries_match_full_extension():
    """The one-by-one entry routine and the full Sub-CTMRG agree (both are
    pinned to brute force through the extension test above)."""
    P, om = W.random_state(6, 3, 4, seed=3)
    w = O.weight_matrix(W.clock(3), 0.8)
    full = O.sub_ctmrg(P, om[:6, None] * P, w, 6, 3)
    rng = np.random.default_rng(0)
    r = rng.integers(0, 18, 50)
    c = rng.integers(0, 18, 50)
    np.testing.assert_allclose(O.ctilde_entries(P, om[:6], w, 6, 3, r, c), full[r, c], rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("model,m,beta", [("clock3", 12, 0.5), ("cube", 24, 0.8), ("dodecahedron", 8, 1 / 0.6)])
def test_energy_is_the_beta_derivative_of_beta_f(model, m, beta):
    """Thermodynamics fixes u = d(beta f)/d beta: the internal energy from the
    bond expectation (reading R7: 2 <h> with one bond energy in the tip
    vertex) must equal the central difference of beta f from the growth
    factor (reading R5) at beta +- 1e-4, for models without a closed form
    (measured 2e-8, 3e-9, 1.5e-9; the difference is the O(delta^2) error)."""
    spins = W.clock(3) if model == "clock3" else W.spins_for(model)

    def run(b):
        c = O.CTMRG(spins, m, b)
        hist = c.run(5000, 1e-13)
        assert hist[-1]["delta"] < 1e-12
        return c.observables()

    d = 1e-4
    fd = ((beta + d) * run(beta + d)["f"] - (beta - d) * run(beta - d)["f"]) / (2 * d)
    u = run(beta)["u_kept"]
    assert abs(fd - u) <= 1e-7 * abs(u)
