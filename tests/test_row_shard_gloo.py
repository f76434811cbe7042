"""Row-sharded ACCORD-FBS across ranks (world size 2, gloo on CPU).

The objective separates over the rows of Omega (vectorised form in the proof
of Thm 3.2), so rank r can own a block of rows of Omega, Y = Omega X^T and
G = Y X / n with X replicated.  Algorithm 1 then needs one exchange per trial:
the sums ||Delta||^2, ||Y+ - Y||^2 (and the objective's parts) and the max of
the KKT residual.  This test runs that scheme with the FP64 oracle's row-block
functions and checks it reproduces the single-process oracle trajectory.  A
second scheme gives every row block its own line search and stopping test,
with no exchange until the end, and reaches the same estimate.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import accord_ref as R
from synth import workload


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def sharded_fit(rank, world, X, lam, kkt_tol, max_iter, tau0=1.0, beta=0.5):
    """Algorithm 1 on rows [r0, r1) of Omega with an all-reduce of the trial
    scalars; returns (Omega rows, trace of (tau, trials) and f)."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    bounds = np.linspace(0, p, world + 1).astype(int)
    r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
    lam_d = lam
    L = R.lipschitz(X)  # n x n eigenproblem, replicated
    Om = np.zeros((r1 - r0, p))
    Om[np.arange(r1 - r0), r0 + np.arange(r1 - r0)] = 1.0
    Y = Om @ X.T
    G = Y @ X / n

    def allsum(*vals):
        t = torch.tensor(vals, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return t.tolist()

    def allmax(v):
        t = torch.tensor([v], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t[0])

    taus, ntr, fs = [], [], []
    t = 0
    while True:
        d = R.diag_entries(Om, r0)
        g_loc = float(np.sum(Y * Y)) / (2.0 * n)
        l1 = float(np.abs(Om).sum() - np.abs(d).sum())
        g, logd, l1, dsum = allsum(g_loc, float(np.sum(np.log(d))), l1, float(d.sum()))
        fs.append(g - logd + lam * l1 + lam_d * dsum)
        r = allmax(R.kkt_residual(Om, G, lam, lam_d, row0=r0))
        if r <= kkt_tol or t >= max_iter:
            break
        tau = tau0
        for k in range(61):
            Op, Yp, d2, dy2, gp, dG = R.fbs_trial(Om, Y, G, X, tau, lam, lam_d, row0=r0)
            d2, dy2 = allsum(d2, dy2)
            if dy2 / n <= d2 / tau or tau <= 1.0 / L:
                break
            tau *= beta
        taus.append(tau)
        ntr.append(k + 1)
        Om, Y = Op, Yp
        G = Y @ X / n
        t += 1
    return Om, taus, ntr, fs


def _worker(rank, world, port, q, p=90):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workload("ar1", p=p, n=60)
    Om, taus, ntr, fs = sharded_fit(rank, world, w.X, w.lam, 1e-9, 2000)
    rows = [None] * world
    dist.all_gather_object(rows, Om)
    if rank == 0:
        q.put((np.vstack(rows), taus, ntr, fs))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,p", [(2, 90), (3, 91)])
def test_row_sharded_fit_matches_single_process_oracle(world, p):
    """The shared line search on row blocks reproduces the single-process
    oracle's steps, trial counts and objective values, with equal blocks
    (2 ranks, p = 90) and ragged ones (3 ranks, p = 91: 30, 30, 31 rows)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q, p)) for r in range(world)]
    for pr in procs:
        pr.start()
    Om, taus, ntr, fs = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    w = workload("ar1", p=p, n=60)
    ref = R.fit(w.X, w.lam, kkt_tol=1e-9, max_iter=2000)
    assert ref.status == R.OK
    assert taus == ref.tau and ntr == ref.ntrials
    np.testing.assert_allclose(fs, ref.f, rtol=1e-12)
    assert np.linalg.norm(Om - ref.Omega) <= 1e-11 * np.linalg.norm(ref.Omega)


def block_fit(rank, world, X, lam, kkt_tol, max_iter, tau0=1.0, beta=0.5):
    """The per-row-block variant: rank r runs Algorithm 1 on its rows alone,
    with its own step size, line search and stopping test, and no exchange at
    all until the end.  Because f is a sum of one term per row of Omega
    (vectorised form in the proof of Thm 3.2), each block minimises its own
    part of f, so the blocks together reach the same minimiser by a different
    sequence of steps.  Returns (Omega rows, block objective per iteration,
    steps)."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    bounds = np.linspace(0, p, world + 1).astype(int)
    r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
    lam_d = lam
    L = R.lipschitz(X)
    Om = np.zeros((r1 - r0, p))
    Om[np.arange(r1 - r0), r0 + np.arange(r1 - r0)] = 1.0
    Y = Om @ X.T
    G = Y @ X / n
    fs, taus = [], []
    for t in range(max_iter + 1):
        d = R.diag_entries(Om, r0)
        fs.append(float(np.sum(Y * Y)) / (2.0 * n) - float(np.sum(np.log(d)))
                  + lam * float(np.abs(Om).sum() - np.abs(d).sum()) + lam_d * float(d.sum()))
        if R.kkt_residual(Om, G, lam, lam_d, row0=r0) <= kkt_tol or t == max_iter:
            break
        tau = tau0
        for _ in range(61):
            Op, Yp, d2, dy2, gp, dG = R.fbs_trial(Om, Y, G, X, tau, lam, lam_d, row0=r0)
            if dy2 / n <= d2 / tau or tau <= 1.0 / L:
                break
            tau *= beta
        taus.append(tau)
        Om, Y = Op, Yp
        G = Y @ X / n
    return Om, fs, taus


def _block_worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = workload("er", p=120, n=80)
    Om, fs, taus = block_fit(rank, world, w.X, w.lam, 1e-11, 5000)
    out = [None] * world
    dist.all_gather_object(out, (Om, fs, taus))  # the only exchange
    if rank == 0:
        q.put(out)
    dist.barrier()
    dist.destroy_process_group()


def test_per_block_line_search_reaches_the_same_estimate():
    """Two ranks, each with its own line search: the gathered estimate equals
    the single-process oracle's (KKT 1e-11 on both sides), every block's own
    objective decreases at every step, and the blocks' step sequences differ
    from each other and from the global one."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_block_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = q.get(timeout=240)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    w = workload("er", p=120, n=80)
    ref = R.fit(w.X, w.lam, kkt_tol=1e-11, max_iter=5000)
    assert ref.status == R.OK
    Om = np.vstack([o[0] for o in out])
    assert np.linalg.norm(Om - ref.Omega) <= 1e-8 * np.linalg.norm(ref.Omega)
    for _, fs, _ in out:
        assert all(b <= a + 1e-13 * abs(a) for a, b in zip(fs, fs[1:]))
    steps = [o[2] for o in out]
    assert steps[0] != steps[1] and steps[0] != list(ref.tau)


def test_rank_failure_is_seen_by_the_survivor():
    """A rank that leaves between steps makes the next collective of the other
    rank fail with an error instead of hanging (host-side failure detection)."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dropout_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(2):
        r, v = q.get(timeout=120)
        res[r] = v
    for pr in procs:
        pr.join(timeout=60)
    assert res[1] == "left"
    assert res[0] == "error"


def _dropout_worker(rank, world, port, q):
    import datetime
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    t = torch.ones(4, dtype=torch.float64)
    dist.all_reduce(t)  # one healthy step
    if rank == 1:
        q.put((1, "left"))
        q.close()
        q.join_thread()
        os._exit(0)  # leaves between steps, with nothing in flight
    try:
        dist.all_reduce(t)
        q.put((0, "no error"))
    except Exception:
        q.put((0, "error"))
    q.close()
    q.join_thread()
    os._exit(0)


# ------------------------------------------------ the library's host entry ---
# accord_fit_rows (include/accord.h) over gloo ranks: the binding and its
# exchange helper (dist_exchange) run as shipped; the device side of the call is
# played on the host by the oracle, following the library's calling protocol
# (one exchange of the starting iterate's sums, then one per trial with the
# current iterate's KKT residual as the maximum), so the test needs no GPU.

SUMS = 9  # ||Delta||^2, sum log w+_ii, sum w+_ii, sum |w+_ij| (i != j), nnz, bad, ||Delta X^T||^2, ||Y+||^2, bad Y


class OracleRowsLib:
    """The two entry points accord_fit_rows needs, with the oracle's FP64
    arithmetic on one block of rows in place of the kernels."""

    def __init__(self):
        self.exchanges = 0

    def accord_default_opts(self, o_ref):
        o = o_ref._obj
        o.tau0, o.beta, o.max_iter, o.max_backtracks, o.kkt_tol, o.penalize_diag = 1.0, 0.5, 3000, 60, 1e-4, 1

    def accord_fit_rows(self, Xp, n, p, row0, rows, lam, o_ref, cb, ctx, Omp, ws, ws_bytes, st_ref):
        import ctypes
        o, st = o_ref._obj, st_ref._obj
        X = np.ctypeslib.as_array((ctypes.c_float * (n * p)).from_address(Xp)).reshape(n, p).astype(np.float64)
        out = np.ctypeslib.as_array((ctypes.c_double * (rows * p)).from_address(Omp)).reshape(rows, p)
        lam_d = lam if o.penalize_diag else 0.0
        diag = (np.arange(rows), row0 + np.arange(rows))
        sums, maxes = (ctypes.c_double * SUMS)(), (ctypes.c_double * 1)()

        def block_sums(Om, Y, D, dY):
            d = Om[diag]
            off = Om.copy()
            off[diag] = 0.0
            return [float(np.sum(D * D)), float(np.sum(np.log(d))), float(d.sum()), float(np.abs(off).sum()),
                    float(np.count_nonzero(off)), 0.0, float(np.sum(dY * dY)), float(np.sum(Y * Y)), 0.0]

        def exchange(vals, kkt):
            sums[:] = vals
            maxes[0] = kkt
            if cb(sums, SUMS, maxes, 1, ctx) != 0:
                return None
            self.exchanges += 1
            return list(sums), maxes[0]

        def objective(s):
            return s[7] / (2.0 * n) - s[1] + lam * s[3] + lam_d * s[2]

        L = R.lipschitz(X)
        Om = np.zeros((rows, p))
        Om[diag] = 1.0
        Y = Om @ X.T
        ex = exchange(block_sums(Om, Y, 0.0, 0.0), 0.0)
        if ex is None:
            return -6
        f, nnz = objective(ex[0]), ex[0][4]
        it = trials = 0
        status = 1
        while True:
            G = Y @ X / n
            kkt_loc = R.kkt_residual(Om, G, lam, lam_d, row0=row0)
            tau, accepted = o.tau0, False
            for k in range(o.max_backtracks + 1):
                Op, Yp, _, _, _, _ = R.fbs_trial(Om, Y, G, X, tau, lam, lam_d, row0=row0)
                ex = exchange(block_sums(Op, Yp, Op - Om, Yp - Y), kkt_loc)
                if ex is None:
                    return -6
                s, kkt = ex
                if k == 0 and (kkt <= o.kkt_tol or it >= o.max_iter):
                    status = 0 if kkt <= o.kkt_tol else 1
                    break
                trials += 1
                if s[6] / n <= s[0] / tau or tau <= 1.0 / L:
                    accepted = True
                    break
                tau *= o.beta
            if not accepted:
                break
            Om, Y = Op, Yp
            f, nnz = objective(s), s[4]
            it += 1
        out[:] = Om
        st.iters, st.trials, st.status, st.f, st.kkt, st.nnz_offdiag, st.L = it, trials, status, f, kkt, int(nnz), L
        return status


def _host_check(t, name, dtype, shape=None, ndim=None):
    dts = dtype if isinstance(dtype, tuple) else (dtype,)
    assert t.dtype in dts and (shape is None or tuple(t.shape) == tuple(shape)), name


class _HostStream:
    cuda_stream = 0


def _binding_worker(rank, world, port, q, p, bounds, fail_rank):
    import datetime

    from paper_2412_11554_gb300 import accord
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    fake = OracleRowsLib()
    accord.load_library = lambda path=None: fake
    accord._check_tensor = _host_check
    w = workload("ar1", p=p, n=60)
    X = torch.as_tensor(w.X, dtype=torch.float32)
    r0, r1 = bounds[rank]
    exchange = accord.dist_exchange()
    if rank == fail_rank:
        calls = [0]

        def exchange(sums, maxes, inner=exchange):
            calls[0] += 1
            if calls[0] == 5:
                raise RuntimeError("exchange lost")
            inner(sums, maxes)
    try:
        Om, st = accord.accord_fit_rows(X, w.lam, r0, r1 - r0, exchange, precision="fp64", kkt_tol=1e-9,
                                        stream=_HostStream())
        q.put((rank, "ok", Om.numpy(), (st.iters, st.trials, st.status, st.f, st.nnz_offdiag), fake.exchanges))
    except Exception as e:  # the fit ended on this rank: report why
        q.put((rank, "raised", type(e).__name__ + ": " + str(e), None, fake.exchanges))
    q.close()
    q.join_thread()
    os._exit(0)  # a rank whose peer failed may hold a broken group; leave without a collective


def _run_binding(world, p, bounds, fail_rank=-1):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_binding_worker, args=(r, world, port, q, p, bounds, fail_rank))
             for r in range(world)]
    for pr in procs:
        pr.start()
    res = {}
    for _ in range(world):
        r = q.get(timeout=240)
        res[r[0]] = r[1:]
    for pr in procs:
        pr.join(timeout=60)
    return res


@pytest.mark.parametrize("world,p,bounds", [(2, 90, [(0, 64), (64, 90)]),
                                            (3, 96, [(0, 32), (32, 64), (64, 96)])])
def test_binding_exchange_over_gloo_reproduces_the_single_fit(world, p, bounds):
    """accord_fit_rows on gloo ranks, one row block each (row0 a multiple of
    32, a ragged last block for p = 90), with dist_exchange as the exchange:
    every rank reports the global stats of the oracle's single fit, after the
    same number of exchanges, and the gathered rows equal its estimate."""
    res = _run_binding(world, p, bounds)
    ref = R.fit(workload("ar1", p=p, n=60).X, workload("ar1", p=p, n=60).lam, kkt_tol=1e-9, max_iter=3000)
    assert ref.status == R.OK
    assert all(v[0] == "ok" for v in res.values()), res
    Om = np.vstack([res[r][1] for r in range(world)])
    assert len({res[r][3] for r in range(world)}) == 1  # exchanges
    for r in range(world):
        iters, trials, status, f, nnz = res[r][2]
        assert status == 0 and iters == ref.iters and trials == ref.trials
        assert abs(f - ref.f[-1]) <= 1e-12 * abs(ref.f[-1])
        assert nnz == ref.nnz[-1]
    assert np.linalg.norm(Om - ref.Omega) <= 1e-11 * np.linalg.norm(ref.Omega)


def test_binding_exchange_failure_ends_every_rank():
    """One rank's exchange raises on its fifth call: that rank's
    accord_fit_rows re-raises it, and the other rank's next all-gather fails
    on the group's timeout, which its accord_fit_rows raises in turn, instead
    of hanging."""
    res = _run_binding(2, 90, [(0, 64), (64, 90)], fail_rank=1)
    assert res[1][0] == "raised" and "exchange lost" in res[1][1]
    assert res[0][0] == "raised"
    assert res[1][3] == 4 and res[0][3] == 4  # four exchanges completed on both ranks
