"""Writes the stored expected values under tests/golden/ from the FP64 oracle.

Calls only oracle/ (and synth/ for the seeded inputs).  Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import accord_ref as R  # noqa: E402
from synth import workload  # noqa: E402


def chain_summary():
    """Oracle trajectory summary for the AR(1) p=200, n=100, lambda=0.2 chain
    (tau0 = 1, beta = 1/2, KKT tolerance 1e-8)."""
    w = workload("ar1")
    r = R.fit(w.X, w.lam, kkt_tol=1e-8, max_iter=500)
    return {
        "source": "tests/golden/make_golden.py, calling oracle/accord_ref.py only",
        "citation": "Algorithm 1 with the update of Eq. 3.5 and the KKT residual of Eq. 3.3",
        "workload": w.name, "recipe": w.recipe, "lam": w.lam, "kkt_tol": 1e-8,
        "status": r.status, "iters": r.iters, "trials": r.trials, "L": r.L,
        "tau": r.tau, "ntrials": r.ntrials, "f": r.f, "kkt": r.kkt, "nnz": r.nnz,
        "omega_fro": float(np.linalg.norm(r.Omega)), "omega_diag_sum": float(np.trace(r.Omega)),
        "omega_row0": r.Omega[0, :8].tolist(),
    }


def tiny_brute_force():
    """Exact p = 3 minimiser by sign enumeration for a seeded 6 x 3 design."""
    X = np.random.Generator(np.random.PCG64(31)).standard_normal((6, 3))
    S = X.T @ X / 6
    return {"source": "tests/golden/make_golden.py, calling oracle/accord_ref.py only",
            "citation": "Eq. 3.3 restricted to each sign pattern of each row (f separates over rows, "
                        "proof of Thm 3.2); the minimiser of Eq. 3.2 is unique (Thm 3.2)",
            "X": X.tolist(), "lam": 0.25, "Omega": R.brute_force(S, 0.25, 0.25).tolist()}


if __name__ == "__main__":
    with open(os.path.join(HERE, "chain_p200_n100.json"), "w") as fh:
        json.dump(chain_summary(), fh, indent=1)
    with open(os.path.join(HERE, "brute_p3.json"), "w") as fh:
        json.dump(tiny_brute_force(), fh, indent=1)
