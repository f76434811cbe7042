"""The stored oracle fixtures still match the oracle (a change to the
oracle's arithmetic shows up here), and the p = 3 fixture is the limit of the
iterative solver."""
import json
import os

import numpy as np

from oracle import accord_ref as R
from synth import workload

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_chain_fixture_reproduces():
    ref = json.load(open(os.path.join(GOLD, "chain_p200_n100.json")))
    w = workload("ar1")
    r = R.fit(w.X, w.lam, kkt_tol=ref["kkt_tol"], max_iter=500)
    assert r.status == ref["status"] == R.OK
    assert r.iters == ref["iters"] and r.ntrials == ref["ntrials"]
    np.testing.assert_allclose(r.f, ref["f"], rtol=1e-12)
    np.testing.assert_allclose(r.tau, ref["tau"], rtol=0)
    assert abs(np.linalg.norm(r.Omega) - ref["omega_fro"]) <= 1e-10


def test_brute_force_fixture_is_solver_limit():
    ref = json.load(open(os.path.join(GOLD, "brute_p3.json")))
    X = np.array(ref["X"])
    r = R.fit(X, ref["lam"], kkt_tol=1e-13, max_iter=20000)
    assert r.status == R.OK
    assert np.max(np.abs(r.Omega - np.array(ref["Omega"]))) <= 1e-9
