"""accord_loss_f64_noalloc: the objective without any device allocation by
the library, for callers that must not allocate (allocator callbacks,
latency-bound loops, processes whose device memory another allocator has
reserved).  Called through the C ABI and compared with accord_loss on two
calls in a row that share the static scratch array.  Collected last on
purpose, so that a run that stops at the first failure has run everything
else first."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_11554_gb300 import build
    build.build()
    from paper_2412_11554_gb300 import accord
    L = accord.load_library()
    assert L.accord_device_check() == 0
    return L


def _case(n, p, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    X = rng.standard_normal((n, p)).astype(np.float32)
    Om = np.eye(p) + 0.03 * rng.standard_normal((p, p)) * (rng.random((p, p)) < 0.2)
    np.fill_diagonal(Om, 0.5 + rng.random(p))
    return X, Om


def _reference(lib, X32, Om, lam, pen):
    """accord_loss (FP64 mode), the existing entry point, through the C ABI."""
    from paper_2412_11554_gb300 import accord
    o = accord.accord_default_opts(precision="fp64", penalize_diag=int(pen))
    f, g = ctypes.c_double(), ctypes.c_double()
    n, p = X32.shape
    st = lib.accord_loss(X32.data_ptr(), n, p, Om.data_ptr(), lam, ctypes.byref(o), ctypes.byref(f), ctypes.byref(g))
    assert st == 0
    return f.value, g.value


def test_noalloc_loss_matches_accord_loss_twice(lib):
    stream = torch.cuda.current_stream()
    for (n, p, seed, lam, pen) in [(150, 300, 1, 0.2, True), (70, 130, 2, 0.35, False)]:
        X, Om = _case(n, p, seed)
        X32 = torch.as_tensor(X, device="cuda")
        X64 = X32.double().contiguous()
        O = torch.as_tensor(Om, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.accord_loss_f64_noalloc(X64.data_ptr(), n, p, O.data_ptr(), lam, int(pen),
                                         stream.cuda_stream or None, out.data_ptr())
        assert st == 0, lib.accord_last_error()
        torch.cuda.synchronize()
        f, g = out.tolist()
        f_ref, g_ref = _reference(lib, X32, O, lam, pen)
        assert abs(f - f_ref) <= 1e-12 * abs(f_ref)
        assert abs(g - g_ref) <= 1e-12 * abs(g_ref)


def test_noalloc_loss_matches_the_oracle(lib):
    """The same evaluation held directly against the oracle's objective and
    smooth part (Eq. 3.2), in FP64."""
    from oracle import accord_ref as R
    n, p, lam = 90, 210, 0.25
    X, Om = _case(n, p, 3)
    X64 = torch.as_tensor(X, device="cuda").double().contiguous()
    O = torch.as_tensor(Om, device="cuda")
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    for pen in (True, False):
        st = lib.accord_loss_f64_noalloc(X64.data_ptr(), n, p, O.data_ptr(), lam, int(pen), None, out.data_ptr())
        assert st == 0, lib.accord_last_error()
        torch.cuda.synchronize()
        f, g = out.tolist()
        Xd = X.astype(np.float64)
        assert abs(g - R.smooth_g(Om, Xd)) <= 1e-12 * abs(g)
        assert abs(f - R.objective(Om, Xd, lam, penalize_diag=pen)) <= 1e-12 * abs(f)


def test_noalloc_loss_on_a_side_stream(lib):
    """On a caller's own stream the call queues its work there and does not
    synchronise; the result is read once that stream has finished."""
    n, p, lam = 120, 260, 0.3
    X, Om = _case(n, p, 4)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        X32 = torch.as_tensor(X, device="cuda")
        X64 = X32.double().contiguous()
        O = torch.as_tensor(Om, device="cuda")
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.accord_loss_f64_noalloc(X64.data_ptr(), n, p, O.data_ptr(), lam, 1, side.cuda_stream,
                                         out.data_ptr())
        assert st == 0, lib.accord_last_error()
    side.synchronize()
    f, g = out.tolist()
    f_ref, g_ref = _reference(lib, X32, O, lam, True)
    assert abs(f - f_ref) <= 1e-12 * abs(f_ref)
    assert abs(g - g_ref) <= 1e-12 * abs(g_ref)


def test_noalloc_non_finite_inputs_give_the_documented_values(lib):
    """The status cannot report domain errors (nothing is read back): a
    non-finite X gives f = g = NaN and a non-positive diagonal gives
    f = +inf, with status ACCORD_OK."""
    n, p = 40, 70
    X, Om = _case(n, p, 5)
    X[3, 11] = np.nan
    X64 = torch.as_tensor(X, device="cuda").double().contiguous()
    O = torch.as_tensor(Om, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.accord_loss_f64_noalloc(X64.data_ptr(), n, p, O.data_ptr(), 0.2, 1, None, out.data_ptr())
    assert st == 0
    torch.cuda.synchronize()
    assert all(np.isnan(v) for v in out.tolist())
    X, Om = _case(n, p, 6)
    Om[5, 5] = -0.5
    X64 = torch.as_tensor(X, device="cuda").double().contiguous()
    O = torch.as_tensor(Om, device="cuda")
    st = lib.accord_loss_f64_noalloc(X64.data_ptr(), n, p, O.data_ptr(), 0.2, 1, None, out.data_ptr())
    assert st == 0
    torch.cuda.synchronize()
    f, g = out.tolist()
    assert f == float("inf") and np.isfinite(g)


def test_noalloc_rejects_extents_beyond_the_index_limit(lib):
    from paper_2412_11554_gb300 import accord
    X = torch.zeros((1, 8), dtype=torch.float64, device="cuda")  # never read: rejected first
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    for n, p in ((2 ** 31, 8), (1, 2 ** 40), (2 ** 62, 2 ** 62)):
        st = lib.accord_loss_f64_noalloc(X.data_ptr(), n, p, X.data_ptr(), 0.1, 1, None, out.data_ptr())
        assert st == accord.EINVAL, (n, p)


def test_noalloc_rejects_sizes_beyond_the_static_array(lib):
    from paper_2412_11554_gb300 import accord
    n, p = 1, 200000  # needs 72 * p > 8 MiB of scratch
    X = torch.zeros((n, 8), dtype=torch.float64, device="cuda")  # never read: rejected first
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = lib.accord_loss_f64_noalloc(X.data_ptr(), n, p, X.data_ptr(), 0.1, 1, None, out.data_ptr())
    assert st == accord.ENOMEM
    assert "scratch" in lib.accord_last_error().decode()
