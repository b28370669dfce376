"""Closed forms and brute-force references used to pin the oracle.

Nothing here shares code with the oracle or with the CUDA path.
- Onsager's free energy of the square-lattice Ising model (Onsager 1944),
  evaluated by Gauss-Legendre quadrature.
- Onsager's internal energy (closed form with the complete elliptic integral
  of the first kind, scipy.special.ellipk).
- Yang's spontaneous magnetisation (Yang 1952).
- Their exact derivatives in K: d u/dK from the closed form of u with the
  derivative of the complete elliptic integral,
  dK(k)/dk = E(k) / (k (1 - k^2)) - K(k) / k, and d M/dK of Yang's formula.
- Baxter's corner transfer matrix spectrum of the off-critical Ising model
  (R. J. Baxter, J. Stat. Phys. 15, 485 (1976) and 17, 1 (1977); in the
  free-fermion form of I. Peschel, M. Kaulke and O. Legeza, Ann. Phys.
  (Leipzig) 8, 153 (1999)): the density matrix of a half-infinite cut is
  rho ~ exp(-sum_j eps_j n_j), n_j in {0, 1}, with single-particle levels
  eps_j linear in j and spacing set by the elliptic modulus of the model.
- Exact corner transfer matrices of a k x k quadrant of vertex tensors by
  direct contraction of the network drawn from its geometry.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

K_CRIT = 0.5 * math.log(1.0 + math.sqrt(2.0))


def onsager_minus_beta_f(K: float, n: int = 400) -> float:
    """-beta f per spin = ln 2 + 1/(2 pi^2) int_0^pi int_0^pi ln[cosh^2 2K - sinh 2K (cos a + cos b)]."""
    x, w = np.polynomial.legendre.leggauss(n)
    t = 0.5 * math.pi * (x + 1.0)
    wt = 0.5 * math.pi * w
    c = np.cos(t)
    arg = math.cosh(2 * K) ** 2 - math.sinh(2 * K) * (c[:, None] + c[None, :])
    integral = float(wt @ np.log(arg) @ wt)
    return math.log(2.0) + integral / (2.0 * math.pi ** 2)


def onsager_f(beta: float, K: float | None = None) -> float:
    """Free energy per spin at inverse temperature beta and coupling K (default beta)."""
    K = beta if K is None else K
    return -onsager_minus_beta_f(K) / beta


def onsager_u(K: float) -> float:
    """Energy per spin (J = 1): -coth 2K [1 + (2/pi)(2 tanh^2 2K - 1) K1(k)], k = 2 sinh 2K / cosh^2 2K."""
    k = 2.0 * math.sinh(2 * K) / math.cosh(2 * K) ** 2
    K1 = special.ellipk(k * k)
    return -1.0 / math.tanh(2 * K) * (1.0 + 2.0 / math.pi * (2.0 * math.tanh(2 * K) ** 2 - 1.0) * K1)


def onsager_du_dK(K: float) -> float:
    """d u / d K of onsager_u, differentiated by hand: u = -A B with
    A = coth 2K and B = 1 + (2/pi)(2 t^2 - 1) K1(k), t = tanh 2K."""
    s, c = math.sinh(2 * K), math.cosh(2 * K)
    t = s / c
    k = 2.0 * s / c ** 2
    K1, E1 = special.ellipk(k * k), special.ellipe(k * k)
    dK1_dk = E1 / (k * (1.0 - k * k)) - K1 / k
    dk_dK = 4.0 / c - 8.0 * s * s / c ** 3
    A, dA = c / s, -2.0 / s ** 2
    B = 1.0 + 2.0 / math.pi * (2.0 * t * t - 1.0) * K1
    dB = 2.0 / math.pi * (8.0 * t * (1.0 - t * t) * K1 + (2.0 * t * t - 1.0) * dK1_dk * dk_dK)
    return -(dA * B + A * dB)


def yang_dm_dK(K: float) -> float:
    """d M / d K of Yang's M = (1 - sinh^-4 2K)^(1/8): cosh 2K sinh^-5 2K (1 - sinh^-4 2K)^(-7/8)."""
    if K <= K_CRIT:
        return 0.0
    s = math.sinh(2 * K)
    return math.cosh(2 * K) * s ** -5 * (1.0 - s ** -4) ** -0.875


def yang_m(K: float) -> float:
    if K <= K_CRIT:
        return 0.0
    return (1.0 - math.sinh(2 * K) ** -4) ** 0.125


def vertex_tensor(spins: np.ndarray, beta: float) -> np.ndarray:
    """V[r, u, l, d]: one vertex (black plaquette) whose corner spins, in cyclic
    order around the plaquette, are the right, up, left and down legs."""
    B = np.exp(beta * spins @ spins.T)
    return np.einsum("ru,ul,ld,dr->ruld", B, B, B, B)


def brute_force_corner(spins: np.ndarray, beta: float, k: int, boundary: int = 0) -> np.ndarray:
    """Exact corner transfer matrix of a k x k quadrant of vertices.

    Vertex (i, j), 0 <= i, j < k, sits at column i, row j; its right leg
    meets the left leg of (i+1, j) and its up leg the down leg of (i, j+1).
    The right legs of column k-1 and the up legs of row k-1 are fixed to the
    boundary spin.  Row index: the down legs of row 0 (i = 0..k-1); column
    index: the left legs of column 0 (j = 0..k-1).  Contracted directly with
    einsum over the whole network."""
    q = spins.shape[0]
    V = vertex_tensor(spins, beta)
    letters = iter("abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ")
    # bond labels
    h = {}  # horizontal bond between (i,j) and (i+1,j)
    v = {}  # vertical bond between (i,j) and (i,j+1)
    for j in range(k):
        for i in range(k - 1):
            h[(i, j)] = next(letters)
    for i in range(k):
        for j in range(k - 1):
            v[(i, j)] = next(letters)
    row = [next(letters) for _ in range(k)]
    col = [next(letters) for _ in range(k)]
    ops, subs = [], []
    e = np.zeros(q)
    e[boundary] = 1.0
    for j in range(k):
        for i in range(k):
            r = h[(i, j)] if i < k - 1 else None
            u = v[(i, j)] if j < k - 1 else None
            l = h[(i - 1, j)] if i > 0 else col[j]
            d = v[(i, j - 1)] if j > 0 else row[i]
            T = V
            idx = ""
            # fix boundary legs by contracting with the unit vector
            if r is None:
                T = np.einsum("ruld,r->uld", T, e)
            else:
                idx += r
            if u is None:
                T = np.einsum(("uld,u->ld" if r is None else "ruld,u->rld"), T, e)
            else:
                idx += u
            idx += l + d
            ops.append(T)
            subs.append(idx)
    out = "".join(row) + "".join(col)
    expr = ",".join(subs) + "->" + out
    C = np.einsum(expr, *ops, optimize="greedy")
    return C.reshape(q ** k, q ** k, order="F")


def normalised_abs_spectrum(C: np.ndarray, n: int) -> np.ndarray:
    ev = np.linalg.eigvalsh(0.5 * (C + C.T))
    ev = ev[np.argsort(-np.abs(ev))][:n]
    return ev / ev[0]


def baxter_ctm_levels(K: float, nmax: int = 80) -> list:
    """Single-particle levels eps_j of the isotropic square-lattice Ising
    model's corner transfer matrix (rho = A^4 in the thermodynamic limit), at
    coupling K != K_CRIT, with the boundary spins fixed:
      eps = pi K(k') / K(k), K() the complete elliptic integral of the first
      kind, k' = sqrt(1 - k^2);
      ordered phase (sinh 2K > 1):    k = sinh^-2 2K, eps_j = 2 j eps, j = 1, 2, ...
        (the fixed boundary selects one of the two ordered states, which
        removes the zero mode j = 0 of the symmetric corner);
      disordered phase (sinh 2K < 1): k = sinh^2 2K,  eps_j = (2 j + 1) eps, j = 0, 1, ...
    Levels above 700 (weights below 1e-304) are dropped."""
    s = math.sinh(2.0 * K)
    k = 1.0 / (s * s) if s > 1.0 else s * s
    eps = math.pi * special.ellipk(1.0 - k * k) / special.ellipk(k * k)
    js = range(1, nmax + 1) if s > 1.0 else range(nmax)
    lev = [(2 * j if s > 1.0 else 2 * j + 1) * eps for j in js]
    return [e for e in lev if e < 700.0]


def baxter_rho_spectrum(K: float, n: int) -> np.ndarray:
    """The n largest eigenvalues of rho (normalised to trace 1 over all
    states) as sums of distinct levels: every subset {j} gives exp(-sum eps_j)."""
    lev = baxter_ctm_levels(K)
    sums = [0.0]
    for e in lev:
        sums = sorted(sums + [x + e for x in sums])[:max(4 * n, 64)]
    sums = np.array(sums)
    logZ = sum(math.log1p(math.exp(-e)) for e in lev)
    return np.exp(-sums[:n] - logZ)


def baxter_entropy(K: float) -> float:
    """Von Neumann entropy of rho from the free-fermion levels:
    S = sum_j [ln(1 + e^-eps_j) + eps_j / (e^eps_j + 1)]."""
    return float(sum(math.log1p(math.exp(-e)) + e / (math.exp(e) + 1.0) for e in baxter_ctm_levels(K)))
