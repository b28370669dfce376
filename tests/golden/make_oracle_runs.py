"""Write the stored oracle runs used by the GPU parity tests.

Calls only the CPU oracle (oracle/): Algorithm 3 of arXiv:2004.08669 from the
fixed-boundary initial state of the q = 20 dodecahedron model, with the
oracle's full dense diagonalisation every step.  Each run records, per step,
the growth factor kappa (f = -(T/2) ln kappa, reading R5), the kept-state S_E
(Eq. 6), m_eff and the convergence measure, and at the end the observables
(f, M of Eq. 5, u, S_E) of the last state.

  python tests/golden/make_oracle_runs.py traj    # m = 256, T = 0.4398, 20 steps
  python tests/golden/make_oracle_runs.py traj64  # m = 256, T = 0.4398, 64 steps
  python tests/golden/make_oracle_runs.py fixed   # m = 32 and 64, T = 0.4398, to delta < 1e-12
  python tests/golden/make_oracle_runs.py m1024   # m = 1024, T = 0.4398, 3 steps (live block <= 8000)

The m = 256 trajectory takes about 15 minutes on 8 host cores (64 steps: about
an hour), the fixed points a few minutes.
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2004_08669_gb300 import workloads as W  # noqa: E402


def run(m: int, T: float, max_steps: int, tol: float, name: str):
    t0 = time.time()
    c = O.CTMRG(W.dodecahedron(), m, 1.0 / T)
    steps = []
    for _ in range(max_steps):
        r = c.step()
        steps.append({k: r[k] for k in ("kappa", "delta", "S_E_kept", "m_eff")})
        if r["delta"] < tol:
            break
    ob = c.observables()
    out = {"_source": "oracle/ctm_oracle.c via oracle/oracle.py (tests/golden/make_oracle_runs.py): Algorithm 3 "
                      "of arXiv:2004.08669 from the fixed-boundary state, dense diagonalisation each step",
           "model": "dodecahedron", "q": 20, "m": m, "T": T, "beta": 1.0 / T, "boundary_spin": 0,
           "tol_cluster": 1e-10, "tol_zero": 1e-10, "steps_run": len(steps), "stop_tol": tol,
           "steps": steps,
           "observables": {"f": ob["f"], "M": ob["M_kept"], "u": ob["u_kept"], "S_E": ob["S_E_kept"],
                           "kappa": ob["kappa"]},
           "host_seconds": round(time.time() - t0, 1), "host_threads": O.num_threads()}
    with open(os.path.join(HERE, name), "w") as fh:
        json.dump(out, fh, indent=1)
    print(name, len(steps), out["observables"], flush=True)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "fixed"
    if what == "traj":
        run(256, 0.4398, 20, 0.0, "oracle_q20_m256_T0.4398_20steps.json")
    elif what == "m1024":
        run(1024, 0.4398, 3, 0.0, "oracle_q20_m1024_T0.4398_3steps.json")
    elif what == "traj64":
        run(256, 0.4398, 64, 0.0, "oracle_q20_m256_T0.4398_64steps.json")
    else:
        for m in (32, 64):
            run(m, 0.4398, 5000, 1e-12, f"oracle_q20_m{m}_T0.4398_fixed_point.json")
