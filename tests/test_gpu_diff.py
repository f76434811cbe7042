"""GPU parity of the differentiation entry points against the oracle:
the smooth loss and its gradients in Omega and X (through the autograd
Function as well), and the implicit derivative of a held-out loss in
log(lambda), which is also checked against central finite differences of
GPU fits (h = 1e-4) at the full differentiation workload (p = 2000,
300 training + 100 held-out rows, lambda = 0.2)."""
import math

import numpy as np
import pytest
import torch

from oracle import accord_ref as R
from synth import diff_workload

pytestmark = pytest.mark.gpu


def dev(x, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def rand_omega(p, seed, density=0.05):
    rng = np.random.Generator(np.random.PCG64(seed))
    O = 0.1 * rng.standard_normal((p, p)) * (rng.random((p, p)) < density)
    np.fill_diagonal(O, 1.0 + rng.random(p))
    return O


@pytest.mark.parametrize("n,p", [(15, 20), (37, 150), (300, 2000)])
def test_gradients_match_oracle_fp64(A, n, p):
    X = np.random.Generator(np.random.PCG64(n + p)).standard_normal((n, p)).astype(np.float32)
    O = rand_omega(p, 3 * p)
    Xd = X.astype(np.float64)
    GO = A.accord_grad(dev(X), dev(O, torch.float64), smooth=True).cpu().numpy()
    GX = A.accord_grad_x(dev(X), dev(O, torch.float64)).cpu().numpy()
    rO, rX = R.smooth_loss_grad_omega(O, Xd), R.smooth_loss_grad_x(O, Xd)
    assert np.max(np.abs(GO - rO)) <= 1e-12 * np.max(np.abs(rO))
    assert np.max(np.abs(GX - rX)) <= 1e-12 * np.max(np.abs(rX))


@pytest.mark.parametrize("n,p", [(37, 150), (300, 2000)])
def test_gradients_match_oracle_mixed(A, n, p):
    X = np.random.Generator(np.random.PCG64(n + p)).standard_normal((n, p)).astype(np.float32)
    O = rand_omega(p, 3 * p).astype(np.float32)
    Xd, Od = X.astype(np.float64), O.astype(np.float64)
    GX = A.accord_grad_x(dev(X), dev(O)).double().cpu().numpy()
    rX = R.smooth_loss_grad_x(Od, Xd)
    # split-BF16 products: error relative to the sum of |terms| (|X| |Omega^T| |Omega| / n)
    scale = np.max(np.abs(Xd) @ (np.abs(Od).T @ np.abs(Od))) / n
    assert np.max(np.abs(GX - rX)) <= 3e-5 * scale


def test_autograd_function(A):
    """SmoothLoss: forward equals the oracle loss; backward gives the oracle
    gradients in Omega and X; torch.autograd.gradcheck passes in FP64."""
    n, p = 40, 60
    X = np.random.Generator(np.random.PCG64(5)).standard_normal((n, p)).astype(np.float32)
    O = rand_omega(p, 11, density=0.1)
    Om = dev(O, torch.float64).requires_grad_(True)
    Xt = dev(X).requires_grad_(True)
    L = A.smooth_loss(Om, Xt)
    Xd = X.astype(np.float64)
    assert abs(L.item() - R.smooth_loss(O, Xd)) <= 1e-12 * abs(L.item())
    L.backward()
    assert np.max(np.abs(Om.grad.cpu().numpy() - R.smooth_loss_grad_omega(O, Xd))) <= 1e-11
    rX = R.smooth_loss_grad_x(O, Xd)
    assert np.max(np.abs(Xt.grad.double().cpu().numpy() - rX)) <= 1e-6 * np.max(np.abs(rX))  # stored in FP32
    # chain rule with a non-unit upstream gradient
    Om.grad = None
    (3.0 * A.smooth_loss(Om, dev(X))).backward()
    assert np.max(np.abs(Om.grad.cpu().numpy() - 3.0 * R.smooth_loss_grad_omega(O, Xd))) <= 3e-11
    O2 = dev(rand_omega(12, 7, density=0.3), torch.float64).requires_grad_(True)
    X2 = dev(np.random.Generator(np.random.PCG64(6)).standard_normal((10, 12)))
    assert torch.autograd.gradcheck(lambda o: A.smooth_loss(o, X2), (O2,), eps=1e-6, atol=1e-8, rtol=1e-6)


def test_implicit_derivative_matches_oracle(A):
    """Same estimate in, same derivative out: the GPU row solves against the
    oracle's (FP64, p = 300)."""
    w = diff_workload(p=300, n=120, n_val=60)
    r = R.fit(w.X_train, w.lam, kkt_tol=1e-10, max_iter=20000)
    assert r.status == R.OK
    d_ref, dO_ref = R.implicit_dloglam(r.Omega, w.X_train, w.X_val, w.lam)
    d, lv, dO = A.accord_dloss_dloglam(dev(w.X_train), dev(w.X_val), dev(r.Omega, torch.float64), w.lam,
                                       want_domega=True)
    assert abs(d - d_ref) <= 1e-10 * max(1.0, abs(d_ref))
    assert abs(lv - R.smooth_loss(r.Omega, w.X_val)) <= 1e-12 * abs(lv)
    assert np.max(np.abs(dO.cpu().numpy() - dO_ref)) <= 1e-10 * max(1.0, np.max(np.abs(dO_ref)))
    # penalize_diag off: the diagonal row of the right-hand side is 0
    r0 = R.fit(w.X_train, w.lam, kkt_tol=1e-10, max_iter=20000, penalize_diag=False)
    d0_ref, _ = R.implicit_dloglam(r0.Omega, w.X_train, w.X_val, w.lam, penalize_diag=False)
    d0, _, _ = A.accord_dloss_dloglam(dev(w.X_train), dev(w.X_val), dev(r0.Omega, torch.float64), w.lam,
                                      penalize_diag=False)
    assert abs(d0 - d0_ref) <= 1e-10 * max(1.0, abs(d0_ref))


def test_implicit_derivative_large_active_sets(A):
    """Rows whose active set exceeds the 128 entries of the shared-memory
    solve go to the second pass, whose systems sit in the workspace: a nearly
    dense estimate (p = 300, n = 600, lambda = 0.01) against the oracle in FP64
    mode and, on the same estimate in FP32, the mixed mode against FP64.  An
    active set over 1024 entries is refused with EUNSUPPORTED."""
    from paper_2412_11554_gb300 import accord
    rng = np.random.Generator(np.random.PCG64(77))
    X = rng.standard_normal((600, 300)).astype(np.float32)
    Xv = rng.standard_normal((100, 300)).astype(np.float32)
    lam = 0.01
    r = R.fit(X, lam, kkt_tol=1e-10, max_iter=20000)
    assert r.status == R.OK
    m = (r.Omega != 0).sum(axis=1)
    assert m.max() > 128 and m.min() <= 300
    d_ref, dO_ref = R.implicit_dloglam(r.Omega, X, Xv, lam)
    d, lv, dO = A.accord_dloss_dloglam(dev(X), dev(Xv), dev(r.Omega, torch.float64), lam, want_domega=True)
    assert abs(d - d_ref) <= 1e-9 * max(1.0, abs(d_ref)), (d, d_ref)
    assert np.max(np.abs(dO.cpu().numpy() - dO_ref)) <= 1e-9 * max(1.0, np.max(np.abs(dO_ref)))
    O32 = dev(r.Omega, torch.float32)
    d32, _, _ = A.accord_dloss_dloglam(dev(X), dev(Xv), O32, lam)
    d64, _, _ = A.accord_dloss_dloglam(dev(X), dev(Xv), O32.double(), lam)
    assert abs(d32 - d64) <= 1e-3 * abs(d64), (d32, d64)
    # 1100 active entries in every row
    p = 1100
    Ob = np.full((p, p), 1e-3)
    np.fill_diagonal(Ob, 1.0)
    Xb = rng.standard_normal((40, p)).astype(np.float32)
    with pytest.raises(accord.AccordError) as e:
        A.accord_dloss_dloglam(dev(Xb), dev(Xb), dev(Ob, torch.float64), 0.1)
    assert e.value.status == accord.EUNSUPPORTED
    assert "1024" in accord.accord_last_error()


def test_mixed_derivative_matches_fp64_on_same_estimate(A):
    """The mixed mode (tensor-core S and held-out products) against the FP64
    mode on the same FP32 estimate (p = 2000)."""
    w = diff_workload()
    Xt, Xv = dev(w.X_train), dev(w.X_val)
    O32, st = A.accord_fit(Xt, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=20000)
    assert st.status == 0
    d32, l32, dO32 = A.accord_dloss_dloglam(Xt, Xv, O32, w.lam, want_domega=True)
    d64, l64, dO64 = A.accord_dloss_dloglam(Xt, Xv, O32.double(), w.lam, want_domega=True)
    assert abs(d32 - d64) <= 1e-3 * abs(d64), (d32, d64)
    assert abs(l32 - l64) <= 1e-5 * abs(l64)
    dd = dO64.cpu().numpy()
    assert np.max(np.abs(dO32.double().cpu().numpy() - dd)) <= 1e-3 * np.max(np.abs(dd))


def test_implicit_derivative_full_size_finite_differences(A):
    """p = 2000, n = 300 + 100 held out, lambda = 0.2: the implicit derivative
    at the FP64 GPU estimate equals the central difference (h = 1e-4) of the
    held-out loss at the FP64 GPU estimates for lambda e^(+-h); the mixed
    estimate's derivative agrees to the accuracy of its KKT tolerance."""
    w = diff_workload()
    Xt, Xv = dev(w.X_train), dev(w.X_val)
    h = 1e-4
    fit = dict(precision="fp64", kkt_tol=1e-10, max_iter=20000)
    O, st = A.accord_fit(Xt, w.lam, **fit)
    assert st.status == 0
    Op, sp = A.accord_fit(Xt, w.lam * math.exp(h), Omega=O.clone(), init_from_omega=True, **fit)
    Om, sm = A.accord_fit(Xt, w.lam * math.exp(-h), Omega=O.clone(), init_from_omega=True, **fit)
    assert sp.status == 0 and sm.status == 0
    # the implicit derivative holds where the active set is locally constant:
    # at most a few entries may enter or leave within +-h, and only tiny ones
    Oc, Opc, Omc = O.cpu().numpy(), Op.cpu().numpy(), Om.cpu().numpy()
    changed = ((Oc != 0) != (Opc != 0)) | ((Oc != 0) != (Omc != 0))
    assert changed.sum() <= 3, int(changed.sum())
    scale = np.max(np.abs(Oc - np.diag(np.diag(Oc))))
    assert np.all(np.abs(np.stack([Oc, Opc, Omc])[:, changed]) <= 1e-4 * scale)
    assert np.count_nonzero(Oc) - 2000 > 500  # a real (off-diagonal) active set
    d, lv, dO = A.accord_dloss_dloglam(Xt, Xv, O, w.lam, want_domega=True)
    _, lp, _ = A.accord_dloss_dloglam(Xt, Xv, Op, w.lam * math.exp(h))
    _, lm, _ = A.accord_dloss_dloglam(Xt, Xv, Om, w.lam * math.exp(-h))
    fd = (lp - lm) / (2 * h)
    assert abs(d - fd) <= 1e-4 * abs(fd) + 1e-9, (d, fd)
    dfd = (Opc - Omc) / (2 * h)
    # rows decouple: compare the rows whose active set stays fixed
    keep = ~np.any(changed, axis=1)
    assert keep.sum() >= 1990
    assert np.max(np.abs(dO.cpu().numpy()[keep] - dfd[keep])) <= 1e-4 * np.max(np.abs(dfd[keep]))
    # mixed precision: estimate at KKT 2e-5, derivative in FP64 from it
    O32, s32 = A.accord_fit(Xt, w.lam, precision="mixed", kkt_tol=2e-5, max_iter=20000)
    assert s32.status == 0
    d32, _, _ = A.accord_dloss_dloglam(Xt, Xv, O32, w.lam)
    assert abs(d32 - fd) <= 2e-2 * abs(fd), (d32, fd)


@pytest.mark.parametrize("p", [1, 33, 300, 4000])
def test_postprocess_matches_oracle(A, p):
    """Theta-hat = Omega_D Omega and the partial correlations of Sec 3.1 on an
    asymmetric sparse Omega with positive diagonal, ragged tile edges."""
    O = rand_omega(p, 17 + p)
    T64, R64 = A.accord_postprocess(dev(O, torch.float64))
    assert np.max(np.abs(T64.cpu().numpy() - R.theta_hat(O))) <= 1e-15 * max(1.0, np.max(np.abs(R.theta_hat(O))))
    assert np.max(np.abs(R64.cpu().numpy() - R.partial_correlation(O))) <= 1e-15
    O32 = O.astype(np.float32)
    T32, R32 = A.accord_postprocess(dev(O32))
    Od = O32.astype(np.float64)
    assert np.max(np.abs(T32.double().cpu().numpy() - R.theta_hat(Od))) <= 1e-6 * max(1.0, np.max(np.abs(O)))
    assert np.max(np.abs(R32.double().cpu().numpy() - R.partial_correlation(Od))) <= 1e-6
    _, only_rho = A.accord_postprocess(dev(O, torch.float64), theta=False)
    assert torch.equal(only_rho, R64)


def test_postprocess_recovers_theta(A):
    """T^-1 undoes T (Thm 3.1): Omega = Theta_D^-1/2 Theta maps back to Theta."""
    rng = np.random.Generator(np.random.PCG64(91))
    B = rng.standard_normal((70, 70))
    Theta = B @ B.T + 70 * np.eye(70)
    Om = Theta / np.sqrt(np.diag(Theta))[:, None]
    T, Rh = A.accord_postprocess(dev(Om, torch.float64))
    assert np.allclose(T.cpu().numpy(), Theta, rtol=1e-14, atol=1e-12)
    d = np.sqrt(np.diag(Theta))
    want = -Theta / np.outer(d, d)
    np.fill_diagonal(want, 1.0)
    assert np.allclose(Rh.cpu().numpy(), want, rtol=1e-13, atol=1e-14)
