"""Refresh of Y = Omega X^T in the mixed modes.

Algorithm 1 needs Y = Omega^t X^T for the gradient G = Y X / n and for
g = ||Y||^2 / (2n) (Eq. 3.4).  The mixed modes carry Y from step to step as
Y + Delta X^T in FP32, so rounding accumulates over the steps of a fit and
over the penalties of a path chain.  The library forms Y afresh from the
iterate every opts.y_refresh steps, ahead of a step whose KKT test is
predicted to pass, and before a passing KKT test may end a fit, and reports
the largest drift ||Y_carried - Omega X^T||_F / ||Omega X^T||_F it found.
These tests bound that drift, check the bookkeeping, and check against the
FP64 oracle that the returned estimate's objective and KKT residual are those
of Y = Omega X^T formed from it.
"""
import numpy as np
import pytest
import torch

from oracle import accord_ref as R
from synth import workload

pytestmark = pytest.mark.gpu


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def long_fit_case():
    # a hub-and-block graph: about 70 accepted steps (the oracle takes 71)
    return workload("hubblock", p=1000, n=300), 2e-5


def test_refresh_bounds_the_drift_of_y(A):
    w, tol = long_fit_case()
    X = dev(w.X)
    Om, st = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=tol, max_iter=5000)
    print(f"iters {st.iters} trials {st.trials} refreshes {st.y_refreshes} drift {st.y_drift:.2e}")
    assert st.status == 0 and st.iters > 40, st
    # every 32 steps at least, and once more before the stop
    assert st.y_refreshes >= st.iters // 32 + 1
    assert 0.0 < st.y_drift <= 1e-6
    O = Om.double().cpu().numpy()
    Xd = np.asarray(w.X, dtype=np.float64)
    # f and g of the returned estimate are those of Y = Omega X^T formed afresh
    f_ref = R.objective(O, Xd, w.lam)
    assert abs(st.f - f_ref) <= 1e-6 * abs(f_ref), (st.f, f_ref)
    assert abs(st.g - R.smooth_g(O, Xd)) <= 1e-6 * abs(st.g)
    # its FP64 KKT residual: the tolerance, plus what the mixed gradient
    # product itself gets wrong at this estimate
    err_g = float((A.accord_grad(X, Om).double() - A.accord_grad(X, Om.double())).abs().max())
    assert R.kkt_residual(O, R.grad_g(O, Xd), w.lam, w.lam) <= tol + 2 * err_g


def test_refresh_walks_many_chunk_groups(A):
    """p = 2400 has 75 32-column chunks a row.  The group walk splits them
    into eight slices of ten chunks (the last one five), read sixteen chunks
    at a time; the row walk (forced by the testing hook, with lists of at
    most 32 entries) reads a row's words in three groups (32, 32 and 11
    chunks).  Both give the same estimate and the same f, and f of the
    returned estimate, taken from the last Y formed afresh, is the oracle's
    objective at it; a word read twice or missed would be far off.  The
    drift stays at the level of one update's error (the early trials of this
    fit overflow the Delta buckets and take the dense split-BF16 update,
    ~2e-6 of Y; see the full-size path test)."""
    from paper_2412_11554_gb300 import accord
    w = workload("hubblock", p=2400, n=300)
    X = dev(w.X)
    Om, st = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=5000, y_refresh=4)
    try:
        assert accord.accord_test_refresh(32, 1) == 0
        Or, sr = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=5000, y_refresh=4)
    finally:
        assert accord.accord_test_refresh(0, 0) == 0
    assert st.status == 0 and st.y_refreshes >= 2, st
    assert st.y_drift <= 1e-5, st.y_drift
    assert torch.equal(Om, Or) and st.f == sr.f and st.y_drift == sr.y_drift
    O = Om.double().cpu().numpy()
    f_ref = R.objective(O, np.asarray(w.X, dtype=np.float64), w.lam)
    assert abs(st.f - f_ref) <= 1e-6 * abs(f_ref), (st.f, f_ref)


def test_refresh_interval_and_off(A):
    """y_refresh = 0 carries Y through the whole fit (no refresh, no drift
    measured); y_refresh = 1 forms it afresh before every step; a huge interval
    leaves only the refreshes near the stop.  All reach the same estimate."""
    w, tol = long_fit_case()
    X = dev(w.X)
    O32, s32 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=tol, max_iter=5000)
    O0, s0 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=tol, max_iter=5000, y_refresh=0)
    O1, s1 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=tol, max_iter=5000, y_refresh=1)
    Oh, sh = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=tol, max_iter=5000, y_refresh=1 << 30)
    print(f"drift: every 32 {s32.y_drift:.2e}, every step {s1.y_drift:.2e}, only near the stop {sh.y_drift:.2e}")
    for s in (s0, s1, sh):
        assert s.status == 0, s
    assert s0.y_refreshes == 0 and s0.y_drift == 0.0
    assert s1.y_refreshes >= s1.iters and s1.y_drift <= 1e-6
    assert 1 <= sh.y_refreshes <= 8
    ref = O32.double().cpu().numpy()
    for O in (O0, O1, Oh):
        assert rel_fro(O.double().cpu().numpy(), ref) <= 1e-4
    # the per-step drift is the smallest: one update's rounding
    assert s1.y_drift <= s32.y_drift <= max(sh.y_drift, s32.y_drift)


def test_tf32_refresh(A):
    w = workload("scalefree", p=600, n=400)
    Om, st = A.accord_fit(dev(w.X), w.lam, precision="tf32x3", kkt_tol=1e-6, max_iter=5000, y_refresh=4)
    assert st.status == 0 and st.y_refreshes >= 1 and st.y_drift <= 1e-6
    O = Om.double().cpu().numpy()
    f_ref = R.objective(O, np.asarray(w.X, dtype=np.float64), w.lam)
    assert abs(st.f - f_ref) <= 1e-6 * abs(f_ref)


def test_fp64_mode_forms_y_every_trial(A):
    """FP64 mode forms Y+ = Omega+ X^T in every trial: nothing to refresh."""
    w = workload("ar1", p=120, n=90)
    _, st = A.accord_fit(dev(w.X), w.lam, precision="fp64", kkt_tol=1e-9)
    assert st.status == 0 and st.y_refreshes == 0 and st.y_drift == 0.0


def test_path_chain_drift(A):
    """A path of 12 penalties on three subsamples, warm-started along each
    chain: the drift every refresh found stays under 1e-6 at every penalty,
    and every penalty that took a step ended on a Y formed afresh."""
    w = workload("scalefree", p=600, n=300)
    rng = np.random.Generator(np.random.PCG64(71))
    subs = [rng.integers(0, 300, size=m) for m in (150, 220, 300)]
    lams = list(np.geomspace(0.5, 0.08, 12))
    out = A.accord_path(dev(w.X), subs, lams, precision="mixed", kkt_tol=2e-5, max_iter=5000)
    assert out.status == 0 and np.all(out.entry_status == 0), out.entry_status
    steps = out.iters.sum(axis=0)
    longest = int(np.argmax(steps))
    print(f"chain steps {steps.tolist()}, refreshes {out.y_refreshes.sum(axis=0).tolist()}, "
          f"max drift {out.y_drift.max():.2e}")
    assert np.all(out.y_drift <= 1e-6)
    assert np.all(out.y_refreshes[out.iters > 0] >= 1)
    assert out.y_refreshes[:, longest].sum() >= steps[longest] // 32
    assert out.stats.y_drift == out.y_drift.max()
    # the estimates at the chain's best penalty: FP64 KKT against the oracle
    Xd = np.asarray(w.X, dtype=np.float64)
    kb = int(out.best_index[longest])
    O = out.omega_best[longest].double().cpu().numpy()
    assert R.kkt_residual(O, R.grad_g(O, Xd[subs[longest]]), lams[kb], lams[kb]) <= 1e-4


def test_refresh_forms_give_the_same_bits(A):
    """The walk over Omega's nonzeros and the blocked product form the same Y
    bit for bit (ascending column order; a zero term adds exactly 0).  At
    lambda = 0.065 the estimate has 35 to 95 nonzeros a row, so the walk
    lists most 32-row groups together (up to 4096 entries), while the walk
    made to go row by row with lists of at most 32 entries works each row in
    several segments; n = 700 takes two passes of output columns (512 + 188),
    the second listing a segmented row again.  The three fits must return
    the same estimate in the same steps; the two walks also give the same
    sums (f, drift), the blocked form the same f up to the order of its FP32
    partial sums, and f is the oracle's objective at the estimate."""
    from paper_2412_11554_gb300 import accord
    w = workload("hubblock", p=1000, n=700)
    X = dev(w.X)
    lam = 0.065
    runs = {}
    try:
        for key in ((0, 1), (32, 1), (0, 2)):
            assert accord.accord_test_refresh(*key) == 0
            runs[key] = A.accord_fit(X, lam, precision="mixed", kkt_tol=2e-5, max_iter=5000, y_refresh=4)
    finally:
        assert accord.accord_test_refresh(0, 0) == 0
    (Ow, sw), (Os, ss), (Ob, sb) = runs[(0, 1)], runs[(32, 1)], runs[(0, 2)]
    print(f"iters {sw.iters} refreshes {sw.y_refreshes} nnz_offdiag {sw.nnz_offdiag} "
          f"drift walk {sw.y_drift:.3e} blocked {sb.y_drift:.3e}")
    for s in (sw, ss, sb):
        assert s.status == 0 and s.y_refreshes >= 4, s
    assert sw.nnz_offdiag >= 40 * 1000
    assert torch.equal(Ow, Os) and (sw.iters, sw.trials) == (ss.iters, ss.trials)
    assert sw.f == ss.f and sw.y_drift == ss.y_drift
    assert torch.equal(Ow, Ob) and (sw.iters, sw.trials) == (sb.iters, sb.trials)
    # ||Y||^2 (hence g and f) is summed in FP32 partials, over a row's columns
    # in the walk and over the group's rows in the blocked form
    assert abs(sw.f - sb.f) <= 1e-6 * abs(sw.f)
    assert sw.y_drift <= 1e-5 and sb.y_drift <= 1e-5
    f_ref = R.objective(Ow.double().cpu().numpy(), np.asarray(w.X, dtype=np.float64), lam)
    assert abs(sw.f - f_ref) <= 1e-6 * abs(f_ref), (sw.f, f_ref)


def test_refresh_hook_rejects_bad_arguments(A):
    from paper_2412_11554_gb300 import accord
    assert accord.accord_test_refresh(31, 0) == accord.EINVAL
    assert accord.accord_test_refresh(513, 0) == accord.EINVAL
    assert accord.accord_test_refresh(0, 3) == accord.EINVAL
    assert accord.accord_test_refresh(0, -1) == accord.EINVAL
    assert accord.accord_test_refresh(0, 0) == 0
