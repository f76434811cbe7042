"""Failure detection on the device without a GPU fault: every mbarrier wait
of the tensor-core kernels is bounded.  A testing hook shortens the limit to
1 ms and has the next prox GEMM's producers withhold their first stage's
copies, so the MMA issuer's first wait runs out (a barrier that nothing will
complete).  The kernel records the timeout bit, lets the copies it issued
land, frees its TMEM and returns; the fit reports ACCORD_ECUDA with the
timeout named in accord_last_error, and the same device then runs the same
fit to the oracle's answer."""
import numpy as np
import pytest
import torch

from oracle import accord_ref as R
from synth import workload

pytestmark = pytest.mark.gpu


def test_wait_timeout_reports_ecuda_and_the_device_stays_usable(A):
    from paper_2412_11554_gb300 import accord
    L = accord.load_library()
    w = workload("ar1", p=300, n=200)
    X = torch.as_tensor(w.X, device="cuda")
    try:
        assert L.accord_test_wait_limit(1_000_000, 1) == 0
        _, st = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=50, check=False)
        msg = L.accord_last_error().decode()
    finally:
        assert L.accord_test_wait_limit(0, 0) == 0
    assert st.status == accord.ECUDA, st
    assert "timed out" in msg and "0x1" in msg, msg
    torch.cuda.synchronize()
    ref = R.fit(w.X, w.lam, kkt_tol=1e-7, max_iter=3000)
    Om, st2 = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=3000)
    assert st2.status == 0, st2
    O = Om.double().cpu().numpy()
    assert np.linalg.norm(O - ref.Omega) / np.linalg.norm(ref.Omega) <= 1e-4


def test_wait_limit_hook_rejects_bad_arguments(A):
    from paper_2412_11554_gb300 import accord
    L = accord.load_library()
    assert L.accord_test_wait_limit(-1, 0) == accord.EINVAL
    assert L.accord_test_wait_limit(0, 2) == accord.EINVAL
    assert L.accord_test_wait_limit(0, 0) == 0
