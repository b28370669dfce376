"""Temperature derivatives of the observables by central differences through
one temperature scan on the GPU.

For every temperature T of a list the scan runs T - dT, T and T + dT
together (each beta to its own convergence) and returns, beside the
observables at T,
  u_fd  = d(beta f) / d beta  (to compare with the bond-expectation energy u),
  C     = du / dT             (specific heat per spin),
  dM_dT = dM / dT.
These are the finite-difference values that derivatives of the converged
fixed point are checked against; every observable comes from the library's
kernels (ctm_scan_*), only the differences are taken here.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def central_derivatives(spins, m: int, temps: Sequence[float], dT: float = 1e-4, prec: str = "fp64",
                        workers: int = 8, max_steps: int = 5000, device: str = "cuda:0", **kw) -> List[dict]:
    from paper_2004_08669_gb300 import ctm
    temps = [float(t) for t in temps]
    if dT <= 0 or any(t - dT <= 0 for t in temps):
        raise ValueError("need 0 < dT < T for every T")
    grid = []
    for t in temps:
        grid += [t - dT, t, t + dT]
    betas = 1.0 / np.asarray(grid)
    sc = ctm.Scan(spins, m, betas, workers=workers, prec=prec, device=device, **kw)
    try:
        done, conv = sc.run(max_steps)
        obs = sc.observables()
    finally:
        sc.close()
    out = []
    for i, t in enumerate(temps):
        lo, mid, hi = obs[3 * i], obs[3 * i + 1], obs[3 * i + 2]
        b_lo, b_hi = betas[3 * i], betas[3 * i + 2]
        out.append({
            "T": t, "f": mid["f"], "u": mid["u"], "M": mid["M"], "S_E": mid["S_E"],
            "u_fd": (b_hi * hi["f"] - b_lo * lo["f"]) / (b_hi - b_lo),
            "C": (hi["u"] - lo["u"]) / (2.0 * dT),
            "dM_dT": (hi["M"] - lo["M"]) / (2.0 * dT),
            "converged": bool(conv[3 * i] and conv[3 * i + 1] and conv[3 * i + 2]),
            "steps": [int(done[3 * i]), int(done[3 * i + 1]), int(done[3 * i + 2])],
        })
    return out
