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
