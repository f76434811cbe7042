"""A fit split into row blocks (accord_fit_rows): the objective of Eq. 3.2
separates over the rows of Omega (the row-wise form in the proof of Thm
3.2), so blocks of rows that keep X whole and exchange only Algorithm 1's
scalars follow the iterate sequence of one fit.  Here the blocks run on one
GPU, one host thread each, and the exchange sums over the threads in block
order (the role an all-reduce plays between GPUs)."""
import threading

import numpy as np
import pytest
import torch

from oracle import accord_ref as R
from synth import workload

pytestmark = pytest.mark.gpu


class ThreadExchange:
    """Sum / max over k threads, in block order, behind a barrier."""

    def __init__(self, k):
        self.k = k
        self.bar = threading.Barrier(k, timeout=120)
        self.slots = [None] * k
        self.calls = [0] * k

    def fn(self, idx):
        def exchange(sums, maxes):
            self.slots[idx] = (sums.copy(), maxes.copy())
            self.calls[idx] += 1
            self.bar.wait()
            tot = self.slots[0][0].copy()
            for s, _ in self.slots[1:]:
                tot += s
            mx = np.max(np.stack([m for _, m in self.slots]), axis=0)
            self.bar.wait()  # every block has read the round before the next overwrites it
            sums[:] = tot
            maxes[:] = mx
        return exchange


def run_blocks(A, X, lam, bounds, **kw):
    ex = ThreadExchange(len(bounds))
    res = [None] * len(bounds)
    errs = []

    def work(i, r0, r1):
        try:
            res[i] = A.accord_fit_rows(X, lam, r0, r1 - r0, ex.fn(i), **kw)
        except Exception as e:  # surfaced below
            errs.append(e)
            ex.bar.abort()

    th = [threading.Thread(target=work, args=(i, r0, r1)) for i, (r0, r1) in enumerate(bounds)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    assert len(set(ex.calls)) == 1, ex.calls  # the same number of exchanges in every block
    return res


def rel_fro(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("bounds", [[(0, 64), (64, 120)], [(0, 32), (32, 96), (96, 120)]])
def test_fp64_row_blocks_follow_the_single_fit(A, bounds):
    w = workload("ar1", p=120, n=90)
    X = torch.as_tensor(w.X, device="cuda")
    O1, s1 = A.accord_fit(X, w.lam, precision="fp64", kkt_tol=1e-9, max_iter=3000, trace=True)
    res = run_blocks(A, X, w.lam, bounds, precision="fp64", kkt_tol=1e-9, max_iter=3000, trace=True)
    O = torch.cat([r[0] for r in res]).cpu().numpy()
    for _, st in res:
        assert st.status == 0
        assert st.iters == s1.iters and st.trials == s1.trials
        np.testing.assert_array_equal(st.trace[:, 2], s1.trace[:, 2])  # the same step sizes
        assert abs(st.f - s1.f) <= 1e-12 * abs(s1.f)
        assert st.nnz_offdiag == s1.nnz_offdiag
    assert rel_fro(O, O1.cpu().numpy()) <= 1e-12
    ref = R.fit(w.X, w.lam, kkt_tol=1e-9, max_iter=3000)
    assert res[0][1].iters == ref.iters and res[0][1].trials == ref.trials
    assert rel_fro(O, ref.Omega) <= 1e-9


def test_mixed_row_blocks_match_the_oracle(A):
    """BF16x3 blocks at p=600 (a ragged last block of 88 rows): the oracle's
    estimate to 1e-4 and the single mixed fit's iteration count."""
    w = workload("scalefree", p=600, n=400)
    X = torch.as_tensor(w.X, device="cuda")
    O1, s1 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=3000)
    res = run_blocks(A, X, w.lam, [(0, 256), (256, 512), (512, 600)], precision="mixed", kkt_tol=2e-5,
                     max_iter=3000)
    O = torch.cat([r[0] for r in res]).double().cpu().numpy()
    for _, st in res:
        assert st.status == 0
        assert st.iters == res[0][1].iters and st.trials == res[0][1].trials
    ref = R.fit(w.X, w.lam, kkt_tol=1e-7, max_iter=3000)
    assert rel_fro(O, ref.Omega) <= 1e-4
    assert rel_fro(O, O1.double().cpu().numpy()) <= 1e-4
    assert abs(res[0][1].iters - s1.iters) <= 2


def test_one_block_is_the_whole_fit(A):
    w = workload("er", p=90, n=60)
    X = torch.as_tensor(w.X, device="cuda")
    O1, s1 = A.accord_fit(X, w.lam, precision="fp64", kkt_tol=1e-9)
    O, st = A.accord_fit_rows(X, w.lam, 0, 90, lambda s, m: None, precision="fp64", kkt_tol=1e-9)
    assert st.iters == s1.iters and st.trials == s1.trials
    assert rel_fro(O.cpu().numpy(), O1.cpu().numpy()) <= 1e-13


def test_row_block_arguments_are_checked(A):
    from paper_2412_11554_gb300 import accord
    w = workload("ar1", p=64, n=40)
    X = torch.as_tensor(w.X, device="cuda")
    for r0, rows in ((16, 32), (0, 0), (32, 40), (-32, 32)):
        _, st = A.accord_fit_rows(X, w.lam, r0, rows, lambda s, m: None, precision="fp64", check=False)
        assert st.status == accord.EINVAL, (r0, rows)

    def failing(sums, maxes):
        raise RuntimeError("exchange lost")

    with pytest.raises(RuntimeError, match="exchange lost"):
        A.accord_fit_rows(X, w.lam, 0, 32, failing, precision="fp64")
