"""Forward-mode derivative of the Symmetric-CTMRG fixed point with respect to
beta, on the host, in FP64.

TEST INFRASTRUCTURE ONLY: tests/ may use this module; the GPU product path
never imports it.

What it computes.  Algorithm 3 of arXiv:2004.08669 maps the half-row tensor
P and the corner spectrum omega of one step to those of the next; the
observables of Eq. (4)-(6) (and f, u from the growth factor and the bond
expectation) are functions of the state it converges to.  Every operation of
the step is differentiable away from eigenvalue crossings at the cut, so each
step is run twice over: the primal step exactly as the C oracle takes it
(through the oracle's own Sub-CTMRG, P-Index2 and eigensolver), and its
first-order tangent (P_dot, omega_dot) = d(P, omega)/d beta by the product
rule:

  * Sub-CTMRG(P, P', W) is bilinear in (P, P') and linear in W, so its
    tangent is Sub(P_dot, P', W) + Sub(P, P'_dot, W) + Sub(P, P', W_dot);
  * W = exp(beta * sum of the plaquette's four dot products) (Eq. 1-2), so
    W_dot = W * (that sum), entry by entry; the bond-impurity weight
    h W likewise;
  * the eigenpairs of the live block A of C~ follow first-order perturbation
    theory of a symmetric matrix: lambda_i_dot = z_i^t A_dot z_i and
    z_i_dot = sum_{j != i} z_j (z_j^t A_dot z_i) / (lambda_i - lambda_j),
    j over the whole live spectrum (the kept states' derivative has
    components along the discarded ones);
  * P-Index2 is a permutation, the projection P = U^t X a product, the
    Frobenius normalisation (kappa = ||P||) and the omega normalisation
    (sum omega^4 = 1) quotients.

Reading R11 (the paper does not differentiate the method): within a cluster
of eigenvalues that the kept-state rule treats as one multiplet
(|lambda_i - lambda_j| <= tol_cluster |lambda_1|) the coupling term is set to
zero.  The basis inside an exact multiplet is arbitrary; zero coupling is the
parallel-transported choice, a smooth gauge, so every gauge-invariant
observable has the right derivative while the basis itself may rotate from
step to step (as it does in the primal).

The iteration starts from the beta-independent initial state of Algorithm 3
(P_dot = 0, omega_dot = 0) and runs primal and tangent together; once the
primal has converged the tangents of the gauge-invariant quantities converge
at the same rate, and their limits are the derivatives of the fixed point.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def weight_exponent(spins: np.ndarray) -> np.ndarray:
    """The plaquette's sum of four dot products in the q^2 x q^2 layout of the
    weight matrix (reading R1: element (a + q b, c + q d) is the plaquette
    with corners a, b, d, c in cyclic order), so that dW/dbeta = W * this."""
    v = np.asarray(spins, dtype=np.float64)
    q = v.shape[0]
    G = v @ v.T
    a, b, c, d = np.meshgrid(np.arange(q), np.arange(q), np.arange(q), np.arange(q), indexing="ij")
    e4 = G[a, b] + G[b, d] + G[d, c] + G[c, a]
    return np.reshape(e4, (q * q, q * q), order="F")


def _kept_count(ev: np.ndarray, m: int, tol_c: float, tol_z: float) -> int:
    """Reading R4, as the C oracle applies it."""
    L = len(ev)
    if L == 0:
        return 0
    a1 = abs(ev[0])
    meff = min(m, L)
    while 0 < meff < L and abs(abs(ev[meff - 1]) - abs(ev[meff])) <= tol_c * a1:
        meff -= 1
    while meff > 0 and abs(ev[meff - 1]) <= tol_z * a1:
        meff -= 1
    return meff


def _eig_tangent(ev: np.ndarray, Z: np.ndarray, A_dot: np.ndarray, n: int, tol_c: float):
    """First-order perturbation of the eigenpairs (ev, Z) of a symmetric
    matrix along A_dot, for the first n pairs: (lambda_dot[:n], Z_dot[:, :n]).
    Couplings inside a cluster (reading R11) are dropped."""
    H = Z.T @ A_dot @ Z
    H = 0.5 * (H + H.T)
    lam_dot = np.diag(H)[:n].copy()
    gap = ev[None, :n] - ev[:, None]          # gap[j, i] = lambda_i - lambda_j
    tiny = np.abs(gap) <= tol_c * abs(ev[0])
    Fm = np.where(tiny, 0.0, H[:, :n] / np.where(tiny, 1.0, gap))
    return lam_dot, Z @ Fm


def _entropy4_and_tangent(ev: np.ndarray, ev_dot: np.ndarray):
    """S = -sum p ln p with p = ev^4 / sum ev^4, and dS."""
    w4 = ev ** 4
    z = w4.sum()
    p = w4 / z
    z_dot = (4.0 * ev ** 3 * ev_dot).sum()
    p_dot = (4.0 * ev ** 3 * ev_dot) / z - w4 * z_dot / z ** 2
    nz = p > 0.0
    S = -float((p[nz] * np.log(p[nz])).sum())
    S_dot = -float((p_dot[nz] * np.log(p[nz])).sum())
    return S, S_dot


class TangentCTMRG:
    """Symmetric-CTMRG (Algorithm 3) with the forward-mode beta tangent
    carried beside every step."""

    def __init__(self, spins, m: int, beta: float, boundary_spin: int = 0,
                 tol_cluster: float = 1e-10, tol_zero: float = 1e-10):
        self.spins = np.ascontiguousarray(spins, dtype=np.float64)
        self.q, self.dim = self.spins.shape
        if m < 1 or not 0 <= boundary_spin < self.q:
            raise ValueError("invalid configuration")
        self.m, self.N = m, m * self.q
        self.beta = float(beta)
        self.bspin = boundary_spin
        self.tol_c, self.tol_z = tol_cluster, tol_zero
        self.w = O.weight_matrix(self.spins, beta)
        self.wh = O.weight_matrix(self.spins, beta, bond=True)
        e = weight_exponent(self.spins)
        self.w_dot = np.asfortranarray(self.w * e)
        self.wh_dot = np.asfortranarray(self.wh * e)
        # initial state of Algorithm 3 (independent of beta)
        self.P = np.zeros((m, self.N), order="F")
        self.P[0, self.m * boundary_spin] = 1.0
        self.omega = np.zeros(self.N)
        self.omega[0] = 1.0
        self.P_dot = np.zeros((m, self.N), order="F")
        self.omega_dot = np.zeros(self.N)
        self.live = 1
        self.kappa = 0.0
        self.kappa_dot = 0.0
        self.steps = 0
        self._prev = None

    # -- pieces ---------------------------------------------------------------
    def _live_idx(self) -> np.ndarray:
        return np.array([g + self.m * s for s in range(self.q) for g in range(self.live)], dtype=np.int64)

    def _sub(self, P, Pp, w):
        return O.sub_ctmrg(P, Pp, w, self.m, self.q)

    def _extension(self, w, w_dot):
        """C~ = Sub(P, Omega P, w) and its tangent."""
        Pp = np.asfortranarray(self.omega[: self.m, None] * self.P)
        Pp_dot = np.asfortranarray(self.omega_dot[: self.m, None] * self.P + self.omega[: self.m, None] * self.P_dot)
        C = self._sub(self.P, Pp, w)
        C_dot = self._sub(self.P_dot, Pp, w) + self._sub(self.P, Pp_dot, w) + self._sub(self.P, Pp, w_dot)
        return C, C_dot

    def _live_eig(self, C, C_dot):
        idx = self._live_idx()
        A = C[np.ix_(idx, idx)]
        A = 0.5 * (A + A.T)
        ev, Z = O.eigh(A)
        A_dot = C_dot[np.ix_(idx, idx)]
        return idx, ev, Z, A_dot

    # -- one step -------------------------------------------------------------
    def step(self) -> dict:
        m, q, N = self.m, self.q, self.N
        C, C_dot = self._extension(self.w, self.w_dot)
        idx, ev, Z, A_dot = self._live_eig(C, C_dot)
        meff = _kept_count(ev, m, self.tol_c, self.tol_z)
        lam_dot, Z_dot = _eig_tangent(ev, Z, 0.5 * (A_dot + A_dot.T), meff, self.tol_c)

        U = np.zeros((N, m), order="F")
        U_dot = np.zeros((N, m), order="F")
        U[idx, :meff] = Z[:, :meff]
        U_dot[idx, :meff] = Z_dot
        Up = O.pindex2(U, m, q, m)
        Up_dot = O.pindex2(U_dot, m, q, m)
        X = self._sub(self.P, Up, self.w)
        X_dot = self._sub(self.P_dot, Up, self.w) + self._sub(self.P, Up_dot, self.w) + self._sub(self.P, Up, self.w_dot)
        R = U.T @ X
        R_dot = U_dot.T @ X + U.T @ X_dot
        nrm = float(np.sqrt((R * R).sum()))
        nrm_dot = float((R * R_dot).sum()) / nrm
        self.P = np.asfortranarray(R / nrm)
        self.P_dot = np.asfortranarray(R_dot / nrm - R * (nrm_dot / nrm ** 2))
        self.kappa, self.kappa_dot = nrm, nrm_dot

        evk, evk_dot = ev[:meff], lam_dot
        z4 = float((evk ** 4).sum())
        z4_dot = float((4.0 * evk ** 3 * evk_dot).sum())
        sc = z4 ** -0.25
        sc_dot = -0.25 * z4 ** -1.25 * z4_dot
        self.omega = np.zeros(N)
        self.omega_dot = np.zeros(N)
        self.omega[:meff] = evk * sc
        self.omega_dot[:meff] = evk_dot * sc + evk * sc_dot
        self.live = meff
        self.steps += 1

        # convergence of the primal (reading R6) and of the tangent: the
        # normalised spectrum |omega_i| / |omega_1|, kappa, and their
        # derivatives
        a1 = abs(self.omega[0])
        ratio = np.abs(self.omega[:m]) / a1
        sgn = np.sign(self.omega[:m])
        ratio_dot = sgn * self.omega_dot[:m] / a1 - ratio * np.sign(self.omega[0]) * self.omega_dot[0] / a1
        cur = (ratio, ratio_dot, nrm, nrm_dot)
        if self._prev is None:
            delta = delta_t = np.inf
        else:
            pr, prd, pk, pkd = self._prev
            delta = max(float(np.max(np.abs(ratio - pr))), abs(nrm / pk - 1.0))
            delta_t = max(float(np.max(np.abs(ratio_dot - prd))), abs(nrm_dot - pkd) / nrm)
        self._prev = cur
        return {"kappa": nrm, "kappa_dot": nrm_dot, "delta": delta, "delta_tangent": delta_t, "m_eff": meff}

    def run(self, max_steps: int, tol: float = 1e-12, tol_tangent: float = 1e-10) -> list:
        hist = []
        for _ in range(max_steps):
            r = self.step()
            hist.append(r)
            if r["delta"] < tol and r["delta_tangent"] < tol_tangent:
                break
        return hist

    # -- observables and their derivatives -----------------------------------
    def observables(self) -> dict:
        """f, M, u, S_E over the kept states (as the C oracle's "kept"
        values) and their derivatives with respect to beta and to T."""
        m = self.m
        C, C_dot = self._extension(self.w, self.w_dot)
        Ch, Ch_dot = self._extension(self.wh, self.wh_dot)
        idx, ev, Z, A_dot = self._live_eig(C, C_dot)
        meff = _kept_count(ev, m, self.tol_c, self.tol_z)
        lam_dot, Z_dot = _eig_tangent(ev, Z, 0.5 * (A_dot + A_dot.T), meff, self.tol_c)
        evk, Zk = ev[:meff], Z[:, :meff]
        Hh = Ch[np.ix_(idx, idx)]
        Hh_dot = Ch_dot[np.ix_(idx, idx)]

        vb = self.spins[self.bspin]
        mag = np.array([vb @ self.spins[t // m] for t in idx])
        mi = (Zk * Zk * mag[:, None]).sum(axis=0)
        mi_dot = 2.0 * (Zk * Z_dot * mag[:, None]).sum(axis=0)
        hi = np.einsum("ti,tu,ui->i", Zk, Hh, Zk)
        hi_dot = (np.einsum("ti,tu,ui->i", Z_dot, Hh, Zk) + np.einsum("ti,tu,ui->i", Zk, Hh, Z_dot)
                  + np.einsum("ti,tu,ui->i", Zk, Hh_dot, Zk))
        w4, w3 = evk ** 4, evk ** 3
        w4_dot, w3_dot = 4.0 * evk ** 3 * lam_dot, 3.0 * evk ** 2 * lam_dot
        z4, z4_dot = w4.sum(), w4_dot.sum()
        M = float((w4 * mi).sum() / z4)
        M_dot = float(((w4_dot * mi + w4 * mi_dot).sum() - M * z4_dot) / z4)
        hb = float((w3 * hi).sum() / z4)
        hb_dot = float(((w3_dot * hi + w3 * hi_dot).sum() - hb * z4_dot) / z4)
        S, S_dot = _entropy4_and_tangent(evk, lam_dot)
        b = self.beta
        if b > 0.0:
            f = -0.5 / b * np.log(self.kappa)
            f_dot = 0.5 / b ** 2 * np.log(self.kappa) - 0.5 / b * self.kappa_dot / self.kappa
            bf_dot = f + b * f_dot
        else:  # f = -T ln q diverges at T = infinity; beta f stays finite
            f = f_dot = float("nan")
            bf_dot = -0.5 * self.kappa_dot / self.kappa
        u, u_dot = 2.0 * hb, 2.0 * hb_dot
        dT = -b * b  # d beta / dT
        return {
            "f": float(f), "M": M, "u": u, "S_E": S, "kappa": self.kappa,
            "df_dbeta": float(f_dot), "dM_dbeta": M_dot, "du_dbeta": u_dot, "dS_dbeta": S_dot,
            "d_beta_f_dbeta": float(bf_dot), "dlnkappa_dbeta": self.kappa_dot / self.kappa,
            "C": dT * u_dot, "dM_dT": dT * M_dot, "df_dT": dT * float(f_dot), "dS_dT": dT * S_dot,
        }
