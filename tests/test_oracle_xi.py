"""Pins of the oracle's effective correlation length (Sec. II): the
renormalised row-to-row transfer matrix T built from P and W (reading R10).

- Brute force: while nothing is truncated (q^k <= m), the half-row P after
  k steps is the exact half row of k vertices in an orthonormal basis, so T
  has the spectrum of the row transfer matrix of 2k + 1 vertices with the
  fixed boundary spin at both ends, enumerated here directly from W.  This
  fixes which legs of P are the upper and lower block legs, where the
  centre vertex sits and the cyclic order of its legs.
- Ising, m -> infinity: the eigenvalue ratio of the transfer matrix along
  the lattice diagonal is known exactly (one-particle gap above T_c:
  l1/l0 = sinh^2 2K; two-particle gap below T_c in the broken phase:
  sinh^-4 2K).  At finite m the ratio approaches it from below.
- beta = 0: T has rank one (l1 = 0 exactly); T and P are symmetric under the
  reflection of the row.
- A planted mistake (the half rows joined to adjacent corners of the centre
  vertex) fails the brute force.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2004_08669_gb300 import workloads as W


def brute_row_transfer(spins, beta, L, b=0):
    """Row transfer matrix of L vertices, the outer side legs fixed to spin b:
    T[(t_1..t_L), (u_1..u_L)] = sum_h prod_i W(h_{i-1}, t_i, h_i, u_i), with
    W(a, b, c, d) the plaquette weight of Eq. (1) in cyclic corner order,
    computed here from the spin vectors alone."""
    q = spins.shape[0]
    B = np.exp(beta * spins @ spins.T)
    Wc = np.einsum("ab,bc,cd,da->abcd", B, B, B, B)
    R = np.zeros((q, 1, 1))
    R[b, 0, 0] = 1.0
    for _ in range(L):
        new = np.einsum("hxy,htgu->gxtyu", R, Wc)
        n1 = R.shape[1] * q
        R = new.reshape(q, n1, n1)
    return R[b]


def top_ratios(ev, k):
    ev = np.asarray(ev)
    ev = ev[np.argsort(-np.abs(ev))]
    return np.abs(ev[1:k] / ev[0])


@pytest.mark.parametrize("model,beta,kmax", [("ising", 0.4, 3), ("ising", 0.7, 3), ("clock3", 0.9, 2),
                                             ("cube", 1.0, 1)])
def test_untruncated_row_transfer_matches_brute_force(model, beta, kmax):
    spins = W.clock(3) if model == "clock3" else W.spins_for(model)
    q = spins.shape[0]
    m = q ** kmax
    o = O.CTMRG(spins, m, beta)
    for k in range(1, kmax + 1):
        o.step()
        lam = o.row_transfer_spectrum(5)
        Tb = brute_row_transfer(spins, beta, 2 * k + 1)
        assert np.abs(Tb - Tb.T).max() <= 1e-14 * np.abs(Tb).max()
        nk = min(5, Tb.shape[0])
        want = top_ratios(np.linalg.eigvalsh(Tb), nk)
        got = top_ratios(lam[:nk], nk)
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-13)


def test_planted_leg_swap_fails_brute_force():
    """Build T with the two half rows joined to adjacent corners of the
    centre vertex instead of opposite ones, T = sum P W(s, s', t, u) P (the
    matrix rows of w read as the two side legs): the spectrum no longer
    matches the enumerated row (Ising, k = 2, beta = 0.4)."""
    spins, beta, m, q = W.ising(), 0.4, 4, 2
    o = O.CTMRG(spins, m, beta)
    o.step()
    o.step()
    P, _, _ = o.get_state()
    w = O.weight_matrix(spins, beta)
    Wc = w.reshape(q, q, q, q, order="F").transpose(0, 1, 3, 2)  # Wc[a,b,c,d] = W(a,b,c,d)
    Wbad = Wc.transpose(0, 2, 1, 3)                              # Wbad(s, t, s', u) = W(s, s', t, u)
    wbad = Wbad.transpose(0, 1, 3, 2).reshape(q * q, q * q, order="F")
    T_bad = O.row_transfer(P, wbad, m, q)
    T_ok = O.row_transfer(P, w, m, q)
    want = top_ratios(np.linalg.eigvalsh(brute_row_transfer(spins, beta, 5)), 4)
    np.testing.assert_allclose(top_ratios(np.linalg.eigvals(T_ok), 4), want, rtol=1e-11)
    assert np.abs(top_ratios(np.linalg.eigvals(T_bad), 4) - want).max() > 1e-3


def test_reflection_symmetry_and_beta_zero():
    spins = W.dodecahedron()
    m, q = 4, 20
    o = O.CTMRG(spins, m, 1 / 0.44)
    o.run(400, 1e-12)
    P, _, _ = o.get_state()
    P3 = P.reshape(m, m, q, order="F")
    assert np.abs(P3 - P3.transpose(1, 0, 2)).max() <= 1e-14 * np.abs(P3).max()
    T = O.row_transfer(P, O.weight_matrix(spins, 1 / 0.44), m, q)
    assert np.abs(T - T.T).max() <= 1e-14 * np.abs(T).max()
    o0 = O.CTMRG(spins, m, 0.0)
    o0.run(50, 1e-12)
    lam = o0.row_transfer_spectrum(2)
    assert abs(lam[1]) <= 1e-13 * abs(lam[0])


@pytest.mark.parametrize("K,phase", [(0.3, "disordered"), (0.6, "ordered")])
def test_ising_ratio_approaches_exact_diagonal_gap(K, phase):
    exact = np.sinh(2 * K) ** 2 if phase == "disordered" else np.sinh(2 * K) ** -4
    errs = []
    for m in (8, 16, 32):
        o = O.CTMRG(W.ising(), m, K)
        o.run(5000, 1e-13)
        lam = o.row_transfer_spectrum(2)
        r = abs(lam[1] / lam[0])
        errs.append((exact - r) / exact)
        xi = o.xi()
        assert xi == pytest.approx(-1.0 / np.log(r), rel=1e-14)
    # from below, shrinking with m; measured 2.5 / 1.2 / 0.74 % (T > T_c) and
    # 10 / 5.4 / 3.3 % (T < T_c)
    assert all(e > 0 for e in errs)
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < (0.01 if phase == "disordered" else 0.04)
