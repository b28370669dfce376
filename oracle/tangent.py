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
At a gauge-fixed fixed point the same derivative comes from the implicit
equation (I - J) x = dF/dbeta (fixed_point_derivative), and in reverse mode
from the adjoint equation (I - J^t) x_bar = g with J^t applied as the
transpose of one step (_vjp: transposed contractions, inverse permutations,
the symmetric-eigen adjoint; adjoint_dlnkappa_dbeta for the free energy,
adjoint_observables for M, u and S_E, whose cotangents come from
_observables_vjp).
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


def _deflated_solve(A: np.ndarray, Zb: np.ndarray, lam: np.ndarray, Rhs: np.ndarray, tol: float = 1e-14,
                    max_iter: int = 2000):
    """Y with lambda_i y_i - A y_i = r_i on the complement of span(Zb) (Zb
    eigenvectors of the symmetric A, so A leaves the complement invariant),
    column by column, for right sides in that complement: the fixed-point
    iteration Y <- (R + (I - Zb Zb^t) A Y) diag(lambda)^-1, which converges at
    the rate max_i |lambda_b| / |lambda_i| (lambda_b the largest eigenvalue
    left outside the block).  Returns (Y, iterations)."""
    def deflate(Y):
        return Y - Zb @ (Zb.T @ Y)

    inv = 1.0 / lam
    Y = Rhs * inv
    scale = max(float(np.abs(Y).max()), 1e-300)
    for it in range(1, max_iter + 1):
        Y_new = (Rhs + deflate(A @ Y)) * inv
        change = float(np.abs(Y_new - Y).max())
        Y = Y_new
        if change <= tol * scale:
            return Y, it
    raise RuntimeError("deflated iteration did not converge")


def _block_coupling(ev: np.ndarray, b: int, n: int, tol_c: float) -> np.ndarray:
    gap = ev[None, :n] - ev[:b, None]
    tiny = np.abs(gap) <= tol_c * abs(ev[0])
    return np.where(tiny, 0.0, 1.0 / np.where(tiny, 1.0, gap))


def _eig_tangent_block(A: np.ndarray, ev: np.ndarray, Z: np.ndarray, A_dot: np.ndarray, n: int, b: int,
                       tol_c: float):
    """_eig_tangent from the leading b eigenpairs only (what a block
    subspace iteration provides), for the first n <= b pairs.  Inside the
    block the coupling is the same sum over j < b; the part outside it,
    y_i = (lambda_i - A)^-1 (I - Z_b Z_b^t) A_dot z_i, comes from the deflated
    iteration (_deflated_solve).  Returns (lambda_dot, Z_dot, iterations)."""
    Zb = Z[:, :b]
    H = Zb.T @ A_dot @ Zb
    H = 0.5 * (H + H.T)
    lam_dot = np.diag(H)[:n].copy()
    Z_in = Zb @ (H[:, :n] * _block_coupling(ev, b, n, tol_c))
    Rhs = A_dot @ Z[:, :n]
    Y, it = _deflated_solve(A, Zb, ev[:n], Rhs - Zb @ (Zb.T @ Rhs))
    return lam_dot, Z_in + Y, it


def _eig_vjp_block(A: np.ndarray, ev: np.ndarray, Z: np.ndarray, lam_bar: np.ndarray, Z_bar: np.ndarray, n: int,
                   b: int, tol_c: float):
    """Transpose of _eig_tangent_block.  The deflated solve is symmetric
    column by column, so the outside part's cotangent is the same solve
    applied to the deflated Z_bar, paired with the kept vectors."""
    Zb = Z[:, :b]
    K = (Zb.T @ Z_bar) * _block_coupling(ev, b, n, tol_c)
    K[np.arange(n), np.arange(n)] += lam_bar
    A_bar = Zb[:, :] @ np.hstack([K, np.zeros((b, b - n))]) @ Zb.T
    Xb, _ = _deflated_solve(A, Zb, ev[:n], Z_bar - Zb @ (Zb.T @ Z_bar))
    Xb = Xb - Zb @ (Zb.T @ Xb)
    A_bar = A_bar + Xb @ Z[:, :n].T
    return 0.5 * (A_bar + A_bar.T)


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



def _clusters(ev: np.ndarray, tol_c: float):
    """Runs of consecutive eigenvalues (sorted by modulus) closer than
    tol_c |lambda_1|: the multiplets whose basis is arbitrary."""
    out, cur = [], [0]
    for i in range(1, len(ev)):
        if abs(ev[i] - ev[i - 1]) <= tol_c * abs(ev[0]):
            cur.append(i)
        else:
            out.append(cur)
            cur = [i]
    if len(ev):
        out.append(cur)
    return out


def _align(Z: np.ndarray, Z_ref: np.ndarray, ev: np.ndarray, tol_c: float):
    """Rotate each cluster's columns of Z onto Z_ref's (the orthogonal
    factor of the polar decomposition of Z_c^t Z_ref,c; a sign for a single
    state).  Returns the rotated copy and the rotations."""
    Z = Z.copy()
    rot = []
    for c in _clusters(ev, tol_c):
        M = Z[:, c].T @ Z_ref[:, c]
        a, _, bt = np.linalg.svd(M)
        Rc = a @ bt
        Z[:, c] = Z[:, c] @ Rc
        rot.append((c, Rc))
    return Z, rot


def _rotate(Z_dot: np.ndarray, rot) -> np.ndarray:
    Z_dot = Z_dot.copy()
    for c, Rc in rot:
        Z_dot[:, c] = Z_dot[:, c] @ Rc
    return Z_dot



def _pindex2_adjoint(B_bar: np.ndarray, a: int, b: int, c: int) -> np.ndarray:
    """Transpose (= inverse) of the permutation P-Index2 (Algorithm 2),
    (a b) x c -> a x (c b): the oracle's own P-Index2 applied to the entry
    numbers says where every entry goes."""
    n = a * b * c
    where = O.pindex2(np.arange(n, dtype=np.float64).reshape((a * b, c), order="F"), a, b, c)
    src = where.ravel(order="F").astype(np.int64)
    out = np.zeros(n)
    out[src] = np.asarray(B_bar).ravel(order="F")
    return np.asfortranarray(out.reshape((a * b, c), order="F"))


def _eig_vjp(ev: np.ndarray, Z: np.ndarray, lam_bar: np.ndarray, Z_bar: np.ndarray, n: int, tol_c: float):
    """Transpose of _eig_tangent: the cotangent of the (symmetrised) matrix
    from those of the first n eigenvalues and eigenvectors."""
    L = len(ev)
    gap = ev[None, :n] - ev[:, None]
    tiny = np.abs(gap) <= tol_c * abs(ev[0])
    Fm = np.where(tiny, 0.0, 1.0 / np.where(tiny, 1.0, gap))
    K = np.zeros((L, L))
    K[:, :n] = (Z.T @ Z_bar) * Fm
    K[np.arange(n), np.arange(n)] += lam_bar
    A_bar = Z @ K @ Z.T
    return 0.5 * (A_bar + A_bar.T)


def _gmres(apply, b: np.ndarray, tol: float, max_iter: int):
    """Solve apply(x) = b by GMRES without restarts (Arnoldi with modified
    Gram-Schmidt, applied twice; the small least-squares problem by lstsq).
    Returns (x, iterations, relative residual)."""
    b0 = float(np.linalg.norm(b))
    if b0 == 0.0:
        return np.zeros_like(b), 0, 0.0
    V = [b / b0]
    H = np.zeros((max_iter + 1, max_iter))
    res = 1.0
    for k in range(max_iter):
        w = apply(V[k])
        for _ in range(2):
            for j in range(k + 1):
                h = float(V[j] @ w)
                H[j, k] += h
                w = w - h * V[j]
        H[k + 1, k] = float(np.linalg.norm(w))
        e1 = np.zeros(k + 2)
        e1[0] = b0
        y = np.linalg.lstsq(H[: k + 2, : k + 1], e1, rcond=None)[0]
        res = float(np.linalg.norm(H[: k + 2, : k + 1] @ y - e1)) / b0
        if res <= tol or H[k + 1, k] <= 1e-300:
            return sum(yj * vj for yj, vj in zip(y, V)), k + 1, res
        V.append(w / H[k + 1, k])
    raise RuntimeError(f"GMRES did not reach {tol} in {max_iter} iterations (residual {res:.2e})")


class TangentCTMRG:
    """Symmetric-CTMRG (Algorithm 3) with the forward-mode beta tangent
    carried beside every step."""

    def __init__(self, spins, m: int, beta: float, boundary_spin: int = 0,
                 tol_cluster: float = 1e-10, tol_zero: float = 1e-10, ritz_block: int | None = None):
        """ritz_block: take the eigen tangent (and its transpose) from the
        leading ritz_block eigenpairs and a deflated iteration, as a block
        subspace iteration would, instead of from the whole live spectrum."""
        self.ritz_block = ritz_block
        self.block_iterations = 0
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
        """C~ = Sub(P, Omega P, w) and its tangent at the current state."""
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

    def _eig_t(self, A, ev, Z, A_dot, n):
        if self.ritz_block is None:
            return _eig_tangent(ev, Z, A_dot, n, self.tol_c)
        b = min(len(ev), max(self.ritz_block, n))
        if b == len(ev):
            return _eig_tangent(ev, Z, A_dot, n, self.tol_c)
        lam_dot, Z_dot, it = _eig_tangent_block(A, ev, Z, A_dot, n, b, self.tol_c)
        self.block_iterations = max(self.block_iterations, it)
        return lam_dot, Z_dot

    def _eig_v(self, A, ev, Z, lam_bar, Z_bar, n):
        if self.ritz_block is None:
            return _eig_vjp(ev, Z, lam_bar, Z_bar, n, self.tol_c)
        b = min(len(ev), max(self.ritz_block, n))
        if b == len(ev):
            return _eig_vjp(ev, Z, lam_bar, Z_bar, n, self.tol_c)
        return _eig_vjp_block(A, ev, Z, lam_bar, Z_bar, n, b, self.tol_c)

    # -- one step, primal and tangent ----------------------------------------
    def _primal(self, P, omega, live, U_ref=None) -> dict:
        """The primal pieces of one step of Algorithm 3 from (P, omega).
        With U_ref the kept eigenvectors are rotated, cluster by cluster,
        onto U_ref's columns (orthogonal Procrustes; signs for single
        states), which fixes the gauge of the step's output."""
        m, q, N = self.m, self.q, self.N
        Pp = np.asfortranarray(omega[:m, None] * P)
        C = self._sub(P, Pp, self.w)
        idx = np.array([g + m * s for s in range(q) for g in range(live)], dtype=np.int64)
        A = C[np.ix_(idx, idx)]
        A = 0.5 * (A + A.T)
        ev, Z = O.eigh(A)
        meff = _kept_count(ev, m, self.tol_c, self.tol_z)
        Zk = Z[:, :meff].copy()
        rot = None
        if U_ref is not None:
            Zk, rot = _align(Zk, U_ref[idx, :meff], ev[:meff], self.tol_c)
        U = np.zeros((N, m), order="F")
        U[idx, :meff] = Zk
        Up = O.pindex2(U, m, q, m)
        X = self._sub(P, Up, self.w)
        R = U.T @ X
        nrm = float(np.sqrt((R * R).sum()))
        z4 = float((ev[:meff] ** 4).sum())
        omega_new = np.zeros(N)
        omega_new[:meff] = ev[:meff] * z4 ** -0.25
        return {"P": P, "omega": omega, "Pp": Pp, "idx": idx, "A": A, "ev": ev, "Z": Z, "meff": meff, "rot": rot,
                "U": U, "Up": Up, "X": X, "R": R, "nrm": nrm, "z4": z4,
                "P_new": np.asfortranarray(R / nrm), "omega_new": omega_new}

    def _tangent(self, pr: dict, P_dot, omega_dot, source: bool = True):
        """Tangent of the step whose primal pieces are pr, along the input
        tangent (P_dot, omega_dot), with (source) or without W's own beta
        dependence.  Returns (P_new_dot, omega_new_dot, kappa_dot)."""
        m, q, N = self.m, self.q, self.N
        P, omega, Pp, idx, ev, Z, meff = pr["P"], pr["omega"], pr["Pp"], pr["idx"], pr["ev"], pr["Z"], pr["meff"]
        Pp_dot = np.asfortranarray(omega_dot[:m, None] * P + omega[:m, None] * P_dot)
        C_dot = self._sub(P_dot, Pp, self.w) + self._sub(P, Pp_dot, self.w)
        if source:
            C_dot += self._sub(P, Pp, self.w_dot)
        A_dot = C_dot[np.ix_(idx, idx)]
        lam_dot, Z_dot = self._eig_t(pr["A"], ev, Z, 0.5 * (A_dot + A_dot.T), meff)
        if pr["rot"] is not None:
            Z_dot = _rotate(Z_dot, pr["rot"])
        U_dot = np.zeros((N, m), order="F")
        U_dot[idx, :meff] = Z_dot
        Up_dot = O.pindex2(U_dot, m, q, m)
        X_dot = self._sub(P_dot, pr["Up"], self.w) + self._sub(P, Up_dot, self.w)
        if source:
            X_dot += self._sub(P, pr["Up"], self.w_dot)
        R, nrm = pr["R"], pr["nrm"]
        R_dot = U_dot.T @ pr["X"] + pr["U"].T @ X_dot
        nrm_dot = float((R * R_dot).sum()) / nrm
        P_new_dot = np.asfortranarray(R_dot / nrm - R * (nrm_dot / nrm ** 2))
        evk = ev[:meff]
        z4 = pr["z4"]
        z4_dot = float((4.0 * evk ** 3 * lam_dot).sum())
        sc = z4 ** -0.25
        sc_dot = -0.25 * z4 ** -1.25 * z4_dot
        omega_new_dot = np.zeros(N)
        omega_new_dot[:meff] = lam_dot * sc + evk * sc_dot
        return P_new_dot, omega_new_dot, nrm_dot

    def _measure(self, with_tangent: bool):
        """Convergence of the primal (reading R6: the normalised spectrum
        |omega_i| / |omega_1| and kappa) and of their derivatives."""
        m = self.m
        a1 = abs(self.omega[0])
        ratio = np.abs(self.omega[:m]) / a1
        sgn = np.sign(self.omega[:m])
        ratio_dot = sgn * self.omega_dot[:m] / a1 - ratio * np.sign(self.omega[0]) * self.omega_dot[0] / a1
        cur = (ratio, ratio_dot, self.kappa, self.kappa_dot)
        if self._prev is None:
            delta = delta_t = np.inf
        else:
            pr, prd, pk, pkd = self._prev
            delta = max(float(np.max(np.abs(ratio - pr))), abs(self.kappa / pk - 1.0))
            delta_t = (max(float(np.max(np.abs(ratio_dot - prd))), abs(self.kappa_dot - pkd) / self.kappa)
                       if with_tangent else np.inf)
        self._prev = cur
        return delta, delta_t

    def step(self) -> dict:
        """One primal step with its tangent (no gauge fixing: the tangent
        follows whatever basis the eigensolver returns, reading R11)."""
        pr = self._primal(self.P, self.omega, self.live)
        P_dot, omega_dot, nrm_dot = self._tangent(pr, self.P_dot, self.omega_dot, True)
        self.P, self.omega, self.live = pr["P_new"], pr["omega_new"], pr["meff"]
        self.P_dot, self.omega_dot = P_dot, omega_dot
        self.kappa, self.kappa_dot = pr["nrm"], nrm_dot
        self.steps += 1
        delta, delta_t = self._measure(True)
        return {"kappa": self.kappa, "kappa_dot": nrm_dot, "delta": delta, "delta_tangent": delta_t,
                "m_eff": pr["meff"]}

    def run_primal(self, max_steps: int, tol: float = 1e-12) -> list:
        """Primal steps only (the tangent is left untouched) until the
        spectrum change falls below tol."""
        hist = []
        for _ in range(max_steps):
            pr = self._primal(self.P, self.omega, self.live)
            self.P, self.omega, self.live, self.kappa = pr["P_new"], pr["omega_new"], pr["meff"], pr["nrm"]
            self.steps += 1
            delta, _ = self._measure(False)
            hist.append({"kappa": self.kappa, "delta": delta, "m_eff": pr["meff"]})
            if delta < tol:
                break
        return hist

    def gauge_fixed_point(self, tol_fixed: float = 1e-10) -> dict:
        """From a converged state, a few primal steps with each step's kept
        eigenvectors rotated onto the previous step's (Procrustes per
        cluster) until P repeats entry by entry: a fixed point P* = F(P*) of
        the gauge-fixed step.  Returns that step's primal pieces, whose
        rotation reference is held fixed from then on."""
        m, q = self.m, self.q
        U_ref = None
        for _ in range(24):
            pr = self._primal(self.P, self.omega, self.live, U_ref)
            change = np.inf
            if U_ref is not None:
                # entries weighted by |omega| of both block legs: states far
                # down the spectrum with nearly equal eigenvalues are fixed
                # only to rounding / gap, and weigh nothing in any observable
                a = np.abs(self.omega[:m]) / abs(self.omega[0])
                wgt = a[:, None] * np.tile(a, q)[None, :]
                change = float(np.max(wgt * np.abs(pr["P_new"] - self.P)))
            self.P, self.omega, self.live, self.kappa = pr["P_new"], pr["omega_new"], pr["meff"], pr["nrm"]
            U_ref = pr["U"]
            if change < tol_fixed:
                break
        else:
            raise RuntimeError("the gauge-fixed step does not repeat: not at a fixed point")
        pr = self._primal(self.P, self.omega, self.live, U_ref)
        pr["fixed_point_change"] = change
        return pr

    def _packing(self, meff: int):
        """The state vector of the fixed-point equations: P (m x N) and the
        kept entries of omega."""
        m, N = self.m, self.N
        nP = m * N

        def unpack(x):
            om = np.zeros(N)
            om[:meff] = x[nP:]
            return np.asfortranarray(x[:nP].reshape((m, N), order="F")), om

        def pack(P_part, om_part):
            return np.concatenate([np.asarray(P_part).ravel(order="F"), om_part[:meff]])

        return pack, unpack

    def fixed_point_derivative(self, tol: float = 1e-12, max_iter: int = 500, tol_fixed: float = 1e-10) -> dict:
        """Derivative of a converged fixed point by the implicit function
        theorem instead of the unrolled iteration.

        At the gauge-fixed fixed point (gauge_fixed_point), with the
        reference basis held fixed, d P*/d beta solves
          (I - J) x = dF/dbeta,   J = dF/d(P, omega) at the fixed point,
        where J is one tangent step without W's own beta dependence and the
        right side one tangent step from a zero input with it; the rotation
        onto the reference does not move to first order there (the
        parallel-transported tangent is orthogonal to its cluster).  The
        linear system is solved by GMRES.  This works at unstable fixed
        points too, where the unrolled tangent diverges (J has an eigenvalue
        outside the unit circle but none equal to one)."""
        m, N = self.m, self.N
        pr = self.gauge_fixed_point(tol_fixed)
        pack, unpack = self._packing(pr["meff"])

        def one_minus_J(x):
            P_dot, om_dot, _ = self._tangent(pr, *unpack(x), source=False)
            return x - pack(P_dot, om_dot)

        rhs_P, rhs_om, _ = self._tangent(pr, np.zeros((m, N), order="F"), np.zeros(N), source=True)
        x, iters, res = _gmres(one_minus_J, pack(rhs_P, rhs_om), tol, max_iter)
        self.P_dot, self.omega_dot = unpack(x)
        _, _, self.kappa_dot = self._tangent(pr, self.P_dot, self.omega_dot, source=True)
        return {"iterations": iters, "residual": res, "fixed_point_change": pr["fixed_point_change"]}

    # -- reverse mode ----------------------------------------------------------
    def _sub_vjp(self, P, Pp, w, X_bar):
        """Adjoint of out = Sub-CTMRG(P, P', w) (Algorithm 3: X1 = P^t P',
        P-Index, the product with w, P-Index), linear in each argument: the
        cotangents (P_bar, P'_bar, w_bar) of an output cotangent X_bar.  The
        transposes of the two P-Index permutations are P-Index with the
        middle legs exchanged (Algorithm 1 swaps the second and third legs)."""
        m, q = self.m, self.q
        X2 = O.pindex(P.T @ Pp, m, q, m, q)
        X3_bar = O.pindex(X_bar, m, q, m, q)
        X2_bar = X3_bar @ w.T
        w_bar = X2.T @ X3_bar
        X1_bar = O.pindex(X2_bar, m, m, q, q)
        return Pp @ X1_bar.T, P @ X1_bar, w_bar

    def _vjp(self, pr: dict, P_bar, omega_bar, kappa_bar: float, source: bool = True):
        """Reverse mode of one step: the transpose of _tangent.  Given the
        cotangents of the step's outputs (P_new, omega_new, kappa), returns
        those of its inputs (P, omega) and, with source, of beta through W.
        Each stage is the transpose of its forward counterpart: the
        normalisations, U^t X, the Sub-CTMRG contractions (transposed
        products and inverse permutations), P-Index2 (an inverse
        permutation), the gauge rotation, and the symmetric-eigen adjoint
        A_bar = Z (diag(lambda_bar) + F o (Z^t Z_bar)) Z^t (symmetrised) with
        F_ji = 1 / (lambda_i - lambda_j), set to zero inside a cluster
        (reading R11) and coupling the kept columns to the whole live
        spectrum."""
        m, q, N = self.m, self.q, self.N
        P, omega, Pp, idx, ev, Z, meff = pr["P"], pr["omega"], pr["Pp"], pr["idx"], pr["ev"], pr["Z"], pr["meff"]
        R, nrm, U, X = pr["R"], pr["nrm"], pr["U"], pr["X"]
        # P_new = R / kappa, kappa = ||R||
        R_bar = P_bar / nrm + (kappa_bar - float((P_bar * R).sum()) / nrm ** 2) * R / nrm
        # R = U^t X
        U_bar = X @ R_bar.T
        X_bar = U @ R_bar
        # X = Sub(P, U', w)
        P_in_bar, Up_bar, wX_bar = self._sub_vjp(P, pr["Up"], self.w, X_bar)
        U_bar = U_bar + _pindex2_adjoint(Up_bar, m, q, m)
        Z_bar = U_bar[idx, :meff]
        if pr["rot"] is not None:
            Z_bar = _rotate(Z_bar, [(c, Rc.T) for c, Rc in pr["rot"]])
        # omega_new = lambda (sum lambda^4)^(-1/4) on the kept states
        evk = ev[:meff]
        z4 = pr["z4"]
        ob = omega_bar[:meff]
        lam_bar = ob * z4 ** -0.25 - float((ob * evk).sum()) * z4 ** -1.25 * evk ** 3
        A_bar = self._eig_v(pr["A"], ev, Z, lam_bar, Z_bar, meff)
        C_bar = np.zeros((N, N), order="F")
        C_bar[np.ix_(idx, idx)] = A_bar
        # C~ = Sub(P, Omega P, w)
        P_a, Pp_bar, wC_bar = self._sub_vjp(P, Pp, self.w, C_bar)
        P_in_bar = P_in_bar + P_a + omega[:m, None] * Pp_bar
        omega_in_bar = np.zeros(N)
        omega_in_bar[:m] = (P * Pp_bar).sum(axis=1)
        beta_bar = float(((wX_bar + wC_bar) * self.w_dot).sum()) if source else 0.0
        return np.asfortranarray(P_in_bar), omega_in_bar, beta_bar

    def adjoint_dlnkappa_dbeta(self, tol: float = 1e-12, max_iter: int = 500, tol_fixed: float = 1e-10) -> dict:
        """d ln kappa / d beta of the fixed point in reverse mode: the
        cotangent of ln kappa through one gauge-fixed step gives its partial
        derivatives (g_x, g_beta); the adjoint fixed-point equation
          (I - J^t) x_bar = g_x
        is solved by GMRES with J^t applied as one reverse step, and the
        total derivative is g_beta + x_bar . dF/dbeta, the last term again
        one reverse step (its beta cotangent).  f = -ln kappa / (2 beta)."""
        pr = self.gauge_fixed_point(tol_fixed)
        meff = pr["meff"]
        pack, unpack = self._packing(meff)
        zP, zo = np.zeros((self.m, self.N), order="F"), np.zeros(self.N)
        gP, go, g_beta = self._vjp(pr, zP, zo, 1.0 / pr["nrm"], source=True)

        def one_minus_Jt(y):
            P_b, om_b, _ = self._vjp(pr, *unpack(y), 0.0, source=False)
            return y - pack(P_b, om_b)

        x_bar, iters, res = _gmres(one_minus_Jt, pack(gP, go), tol, max_iter)
        _, _, b_beta = self._vjp(pr, *unpack(x_bar), 0.0, source=True)
        return {"dlnkappa_dbeta": g_beta + b_beta, "iterations": iters, "residual": res}

    def _observables_vjp(self, M_bar: float, u_bar: float, S_bar: float):
        """Reverse mode of the observables at the current state: the
        cotangents of (P, omega) and the explicit beta cotangent (through W
        and the bond-impurity weight) of M_bar M + u_bar u + S_bar S_E, with
        M = sum w^4 m_i / sum w^4, u = 2 sum w^3 h_i / sum w^4, S_E = -sum p
        ln p over the kept states (as observables())."""
        m, N = self.m, self.N
        P, omega = self.P, self.omega
        Pp = np.asfortranarray(omega[:m, None] * P)
        C = self._sub(P, Pp, self.w)
        Ch = self._sub(P, Pp, self.wh)
        idx = self._live_idx()
        A = C[np.ix_(idx, idx)]
        A = 0.5 * (A + A.T)
        ev, Z = O.eigh(A)
        meff = _kept_count(ev, m, self.tol_c, self.tol_z)
        w, Zk = ev[:meff], Z[:, :meff]
        Hh = Ch[np.ix_(idx, idx)]
        vb = self.spins[self.bspin]
        mag = np.array([vb @ self.spins[t // m] for t in idx])
        mi = (Zk * Zk * mag[:, None]).sum(axis=0)
        hi = np.einsum("ti,tu,ui->i", Zk, Hh, Zk)
        w3, w4 = w ** 3, w ** 4
        z4 = w4.sum()
        M = (w4 * mi).sum() / z4
        u = 2.0 * (w3 * hi).sum() / z4
        p = w4 / z4
        lp = np.where(p > 0.0, np.log(np.where(p > 0.0, p, 1.0)), 0.0)
        S = -(p * lp).sum()
        # cotangents of the eigenvalues, of m_i and h_i
        w_bar = (M_bar * 4.0 * w3 * (mi - M) + u_bar * (6.0 * w * w * hi - 4.0 * u * w3)
                 - S_bar * 4.0 * w3 * (lp + S)) / z4
        m_bar = M_bar * w4 / z4
        h_bar = u_bar * 2.0 * w3 / z4
        Z_bar = np.zeros_like(Z)
        Z_bar[:, :meff] = 2.0 * Zk * mag[:, None] * m_bar + ((Hh + Hh.T) @ Zk) * h_bar
        A_bar = self._eig_v(A, ev, Z, w_bar, Z_bar[:, :meff], meff)
        Hh_bar = (Zk * h_bar) @ Zk.T
        C_bar = np.zeros((N, N), order="F")
        Ch_bar = np.zeros((N, N), order="F")
        C_bar[np.ix_(idx, idx)] = A_bar
        Ch_bar[np.ix_(idx, idx)] = Hh_bar
        Pa, Ppa, wa = self._sub_vjp(P, Pp, self.w, C_bar)
        Pb, Ppb, wb = self._sub_vjp(P, Pp, self.wh, Ch_bar)
        Pp_bar = Ppa + Ppb
        P_bar = Pa + Pb + omega[:m, None] * Pp_bar
        omega_bar = np.zeros(N)
        omega_bar[:m] = (P * Pp_bar).sum(axis=1)
        beta_bar = float((wa * self.w_dot).sum() + (wb * self.wh_dot).sum())
        return np.asfortranarray(P_bar), omega_bar, beta_bar

    def adjoint_observables(self, M_bar: float = 0.0, u_bar: float = 0.0, S_bar: float = 0.0,
                            tol: float = 1e-12, max_iter: int = 500, tol_fixed: float = 1e-10) -> dict:
        """d(M_bar M + u_bar u + S_bar S_E)/d beta of the fixed point in
        reverse mode: the observables' cotangent g = (g_x, g_beta) at the
        gauge-fixed fixed point, the adjoint equation (I - J^t) x_bar = g_x by
        GMRES, and g_beta + x_bar . dF/dbeta (one reverse step's beta
        cotangent)."""
        pr = self.gauge_fixed_point(tol_fixed)
        pack, unpack = self._packing(pr["meff"])
        gP, go, g_beta = self._observables_vjp(M_bar, u_bar, S_bar)

        def one_minus_Jt(y):
            P_b, om_b, _ = self._vjp(pr, *unpack(y), 0.0, source=False)
            return y - pack(P_b, om_b)

        x_bar, iters, res = _gmres(one_minus_Jt, pack(gP, go), tol, max_iter)
        _, _, b_beta = self._vjp(pr, *unpack(x_bar), 0.0, source=True)
        return {"derivative": g_beta + b_beta, "iterations": iters, "residual": res}

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
        A = C[np.ix_(idx, idx)]
        meff = _kept_count(ev, m, self.tol_c, self.tol_z)
        lam_dot, Z_dot = self._eig_t(0.5 * (A + A.T), ev, Z, 0.5 * (A_dot + A_dot.T), meff)
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
