"""GPU parity of the sparse export accord_to_csr: the compressed rows of an
estimate against scipy's CSR of the same dense matrix (exact: indices,
offsets and values bit for bit), over ragged sizes, empty and full rows, both
element types, signed zeros and NaN, the short-buffer retry, and the
benchmark's p = 40000 estimate."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
sp = pytest.importorskip("scipy.sparse")


def check_csr(A, O, **kw):
    """accord_to_csr(O) equals scipy's CSR of O (which drops +-0, keeps NaN)."""
    rp, ci, va = A.accord_to_csr(torch.as_tensor(O, device="cuda"), **kw)
    ref = sp.csr_matrix(O)
    ref.sort_indices()
    assert np.array_equal(rp.cpu().numpy(), ref.indptr.astype(np.int64))
    assert np.array_equal(ci.cpu().numpy(), ref.indices.astype(np.int32))
    assert np.array_equal(va.cpu().numpy(), ref.data, equal_nan=True)
    return rp, ci, va


@pytest.mark.parametrize("p", [1, 33, 257, 1000])
@pytest.mark.parametrize("density", [0.0, 0.01, 0.3, 1.0])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_csr_matches_scipy(A, p, density, dtype):
    rng = np.random.Generator(np.random.PCG64(p * 7 + int(density * 100)))
    O = (rng.standard_normal((p, p)) * (rng.random((p, p)) < density)).astype(dtype)
    np.fill_diagonal(O, 1.0 + rng.random(p))
    if p > 2:
        O[p - 1, :] = 0.0       # an empty row (diagonal cleared too)
        O[0, 1] = -0.0          # a signed zero is not an entry
    check_csr(A, O)


def test_csr_nan_and_retry(A):
    rng = np.random.Generator(np.random.PCG64(5))
    O = (rng.standard_normal((300, 300)) * (rng.random((300, 300)) < 0.2)).astype(np.float32)
    O[7, 11] = np.nan           # a NaN is an entry
    # the first attempt's buffer holds one entry: ENOMEM, then the exact size
    check_csr(A, O, nnz_hint=1)


def test_csr_of_fits(A):
    """The export of a fit's estimate, sized by the fit's own nonzero count."""
    from synth import workload
    w = workload("hubblock", p=600, n=300)
    X = torch.as_tensor(w.X, device="cuda")
    for prec in ("mixed", "fp64"):
        Om, st = A.accord_fit(X, w.lam, precision=prec, kkt_tol=1e-5, max_iter=3000)
        rp, _, _ = check_csr(A, Om.cpu().numpy(), nnz_hint=st.nnz_offdiag + 600)
        assert int(rp[-1]) == st.nnz_offdiag + 600


def test_csr_full_size(A):
    """The benchmark's estimate (hub-and-block p = 40000, n = 1000): the
    row offsets against the dense pattern's row counts, and sampled rows
    entry by entry."""
    from synth import workload
    w = workload("hubblock")
    X = torch.as_tensor(w.X, device="cuda")
    Om, st = A.accord_fit(X, w.lam, precision="mixed", kkt_tol=1e-4, max_iter=500)
    rp, ci, va = A.accord_to_csr(Om, nnz_hint=st.nnz_offdiag + w.p)
    counts = (Om != 0).sum(dim=1).cpu().numpy()
    rp = rp.cpu().numpy()
    assert rp[0] == 0 and np.array_equal(np.diff(rp), counts)
    assert rp[-1] == st.nnz_offdiag + w.p
    ci, va = ci.cpu().numpy(), va.cpu().numpy()
    for i in np.random.Generator(np.random.PCG64(3)).choice(w.p, size=16, replace=False):
        row = Om[int(i)].cpu().numpy()
        nzc = np.nonzero(row)[0]
        assert np.array_equal(ci[rp[i]:rp[i + 1]], nzc)
        assert np.array_equal(va[rp[i]:rp[i + 1]], row[nzc])
