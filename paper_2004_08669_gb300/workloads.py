"""Seeded, synthetic inputs shared by the GPU path's tests/bench and the oracle.

This module holds NO arithmetic of the method: only the model definitions
(vertex tables of the polyhedron spins, Sec. I of arXiv:2004.08669 and
Fig. 1) and the named workloads (sizes, temperatures).  Both the CUDA path
and the CPU oracle receive their inputs from here.

Vertex order of the dodecahedron: the four families (+-1,+-1,+-1),
(0,+-1/phi,+-phi), (+-1/phi,+-phi,0), (+-phi,0,+-1/phi), in that order, signs
enumerated + before -, first component slowest; every vector divided by
sqrt(3) to unit length.  Spin 0 = (1,1,1)/sqrt(3) is the boundary spin
"s = 1" of the paper's fixed ferromagnetic boundary condition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PHI = (1.0 + math.sqrt(5.0)) / 2.0


def dodecahedron() -> np.ndarray:
    """q = 20 unit vectors (20 x 3, row-major)."""
    v = []
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            for c in (1.0, -1.0):
                v.append((a, b, c))
    for b in (1.0, -1.0):
        for c in (1.0, -1.0):
            v.append((0.0, b / PHI, c * PHI))
    for a in (1.0, -1.0):
        for b in (1.0, -1.0):
            v.append((a / PHI, b * PHI, 0.0))
    for a in (1.0, -1.0):
        for c in (1.0, -1.0):
            v.append((a * PHI, 0.0, c / PHI))
    return np.array(v, dtype=np.float64) / math.sqrt(3.0)


def cube() -> np.ndarray:
    """q = 8 unit vectors (+-1,+-1,+-1)/sqrt(3), first component slowest."""
    v = [(a, b, c) for a in (1.0, -1.0) for b in (1.0, -1.0) for c in (1.0, -1.0)]
    return np.array(v, dtype=np.float64) / math.sqrt(3.0)


def ising() -> np.ndarray:
    """q = 2 'unit vectors' +1, -1 in one dimension (the Ising model)."""
    return np.array([[1.0], [-1.0]], dtype=np.float64)


def clock(q: int) -> np.ndarray:
    """q planar unit vectors at angles 2 pi k / q (small test models)."""
    t = 2.0 * np.pi * np.arange(q) / q
    return np.stack([np.cos(t), np.sin(t)], axis=1)


def spins_for(name: str) -> np.ndarray:
    return {"dodecahedron": dodecahedron, "cube": cube, "ising": ising}[name]()


@dataclass(frozen=True)
class Workload:
    """A named CTMRG workload: model, cutoff m, temperatures."""
    name: str
    model: str
    m: int
    temperatures: tuple
    max_steps: int = 5000
    tol_spectrum: float = 1e-12
    extra: dict = field(default_factory=dict)

    @property
    def spins(self) -> np.ndarray:
        return spins_for(self.model)

    @property
    def q(self) -> int:
        return self.spins.shape[0]

    @property
    def betas(self) -> np.ndarray:
        return 1.0 / np.asarray(self.temperatures, dtype=np.float64)


WORKLOADS = {
    "dodeca_m8": Workload("dodeca_m8", "dodecahedron", 8, (0.44,)),
    "dodeca_m64": Workload("dodeca_m64", "dodecahedron", 64, (0.4398,)),
    "cube_m64": Workload("cube_m64", "cube", 64, (0.5, 0.8, 1.2)),
    "dodeca_m256": Workload("dodeca_m256", "dodecahedron", 256, (0.4398,)),
    "dodeca_m128_scan": Workload("dodeca_m128_scan", "dodecahedron", 128,
                                 tuple(np.linspace(0.40, 0.48, 32).tolist())),
    "dodeca_m1024": Workload("dodeca_m1024", "dodecahedron", 1024, (0.4398,)),
}


def random_state(m: int, q: int, live: int, seed: int):
    """Seeded random half-row tensor P (m x m q, rows >= live zero) and a
    sorted positive omega, in the paper's storage order (column index
    gamma + m s).  P is made symmetric in its two renormalised legs, as the
    fixed point of the method is."""
    rng = np.random.default_rng(seed)
    N = m * q
    T = rng.standard_normal((m, m, q))
    T = 0.5 * (T + T.transpose(1, 0, 2))
    T[live:, :, :] = 0.0
    T[:, live:, :] = 0.0
    P = np.asfortranarray(T.reshape(m, N, order="F"))
    om = np.zeros(N)
    om[:live] = np.sort(rng.uniform(0.05, 1.0, live))[::-1]
    om[0] = 1.0
    return P, om
