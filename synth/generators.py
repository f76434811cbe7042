"""Seeded generators for precision matrices and Gaussian data.

Shapes follow the simulation designs of the paper: sparse precision matrices
(chain, scale-free tree, hub-and-block, Erdos-Renyi), X ~ N(0, Theta^-1) drawn
through a Cholesky factor of Theta (Sec 5.2 draws its data the same way, by
back-substitution with a triangular factor), p >> n.

Everything here is random-input plumbing: no step of the estimator (loss,
gradient, prox, line search) is computed in this module.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _signed_uniform(rng: np.random.Generator, size: int, lo: float, hi: float) -> np.ndarray:
    mag = rng.uniform(lo, hi, size=size)
    sign = np.where(rng.random(size) < 0.5, -1.0, 1.0)
    return sign * mag


def _assemble(p: int, rows, cols, vals) -> sp.csr_matrix:
    """Symmetric off-diagonal pattern from an edge list (each edge once)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    r = np.concatenate([rows, cols])
    c = np.concatenate([cols, rows])
    v = np.concatenate([vals, vals])
    return sp.csr_matrix((v, (r, c)), shape=(p, p))


def _diag_dominant(offdiag: sp.csr_matrix, factor: float = 1.5, floor: float = 1.0) -> sp.csr_matrix:
    """theta_ii = max(factor * sum_j |theta_ij|, floor) (Sec 5.1 uses factor 1.5)."""
    rowsum = np.asarray(abs(offdiag).sum(axis=1)).ravel()
    d = np.maximum(factor * rowsum, floor)
    return (offdiag + sp.diags(d)).tocsr()


def _unit_diagonal(theta: sp.csr_matrix) -> sp.csr_matrix:
    d = 1.0 / np.sqrt(theta.diagonal())
    D = sp.diags(d)
    return (D @ theta @ D).tocsr()


def ar1_precision(p: int, rho: float = 0.4) -> sp.csr_matrix:
    """Chain graph: theta_ii = 1, theta_{i,i+-1} = rho (Sec 5.4 chain design)."""
    off = np.full(p - 1, rho)
    return sp.diags([off, np.ones(p), off], [-1, 0, 1], format="csr")


def ba_tree_precision(p: int, seed: int, wlo: float = 0.1, whi: float = 0.4) -> sp.csr_matrix:
    """Barabasi-Albert tree (m = 1), signed uniform weights, diagonal dominance
    with factor 1.5, then scaled to unit diagonal."""
    rng = _rng(seed)
    rows, cols = [0], [1]
    ends = [0, 1]
    for v in range(2, p):
        u = ends[int(rng.integers(len(ends)))]
        rows.append(u)
        cols.append(v)
        ends.extend((u, v))
    w = _signed_uniform(rng, len(rows), wlo, whi)
    theta = _diag_dominant(_assemble(p, rows, cols, w))
    return _unit_diagonal(theta)


def hub_block_precision(nblocks: int, bsize: int, nlinks: int, seed: int,
                        wlo: float = 0.2, whi: float = 0.5) -> sp.csr_matrix:
    """Block-diagonal design: in every block one random hub linked to `nlinks`
    random members of the same block; diagonal dominance with factor 1.5 and
    floor 1 (nodes without edges get theta_ii = 1)."""
    rng = _rng(seed)
    rows, cols = [], []
    for b in range(nblocks):
        base = b * bsize
        hub = int(rng.integers(bsize))
        others = np.array([j for j in range(bsize) if j != hub])
        pick = rng.choice(others, size=min(nlinks, bsize - 1), replace=False)
        rows.extend([base + hub] * len(pick))
        cols.extend((base + pick).tolist())
    w = _signed_uniform(rng, len(rows), wlo, whi)
    p = nblocks * bsize
    return _diag_dominant(_assemble(p, rows, cols, w))


def er_precision(p: int, density: float, seed: int, wlo: float = 0.5, whi: float = 1.0) -> sp.csr_matrix:
    """Erdos-Renyi design of Sec 5.1: signed U[wlo, whi] weights, W + W^T,
    diagonal = 1.5 x absolute row sum, unit diagonal scaling, then a second
    diagonal scaling with entries uniform on [1, sqrt(3)]."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(p, k=1)
    keep = rng.random(iu.size) < density
    iu, ju = iu[keep], ju[keep]
    w = _signed_uniform(rng, iu.size, wlo, whi)
    off = _assemble(p, iu, ju, w)
    rowsum = np.asarray(abs(off).sum(axis=1)).ravel()
    theta = (off + sp.diags(1.5 * np.maximum(rowsum, 1e-12))).tocsr()
    theta = _unit_diagonal(theta)
    d = sp.diags(rng.uniform(1.0, math.sqrt(3.0), size=p))
    return (d @ theta @ d).tocsr()


def _blocks(theta: sp.csr_matrix):
    """Split a precision matrix into its connected diagonal blocks (contiguous
    index ranges with no coupling across them)."""
    p = theta.shape[0]
    coo = theta.tocoo()
    reach = np.arange(p)
    np.maximum.at(reach, coo.row, coo.col)
    starts = []
    s = 0
    hi = -1
    for i in range(p):
        hi = max(hi, reach[i])
        if hi == i:
            starts.append((s, i + 1))
            s = i + 1
    return starts


def sample_gaussian(theta: sp.csr_matrix, n: int, seed: int) -> np.ndarray:
    """n rows of N(0, Theta^-1): Theta_B = L L^T per independent block B and
    x_B = L^-T z_B with z ~ N(0, I).  Returned in float64 (n x p)."""
    rng = _rng(seed)
    p = theta.shape[0]
    Z = rng.standard_normal((n, p))
    X = np.empty((n, p))
    for a, b in _blocks(theta):
        blk = theta[a:b, a:b].toarray()
        Lc = np.linalg.cholesky(blk)
        X[:, a:b] = sla.solve_triangular(Lc.T, Z[:, a:b].T, lower=False).T
    return X


def orthogonal_design(n: int, s: np.ndarray, seed: int) -> np.ndarray:
    """X = sqrt(n) Q diag(sqrt(s)) with orthonormal Q (n x p, n >= p), so that
    X^T X / n = diag(s) up to rounding."""
    p = s.size
    if n < p:
        raise ValueError("orthogonal design needs n >= p")
    rng = _rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, p)))
    return math.sqrt(n) * Q * np.sqrt(s)[None, :]


@dataclasses.dataclass
class Workload:
    name: str
    X: np.ndarray            # float32, n x p, row-major (rows = samples)
    lam: float
    theta: sp.csr_matrix     # generating precision matrix (truth), float64
    recipe: str

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def p(self) -> int:
        return self.X.shape[1]


def workload(kind: str, p: int | None = None, n: int | None = None, k: int | None = None) -> Workload:
    """Build one seeded workload.  `kind` is one of

    - "ar1"       chain, theta_ii = 1, theta_{i,i+-1} = 0.4, lambda = 0.2
    - "scalefree" BA tree (m=1), +-U[0.1,0.4], unit diagonal, lambda = 0.15
    - "hubblock"  200-node blocks, one hub linked to 10% of its block,
                  +-U[0.2,0.5], diagonally dominant, lambda = 0.1
    - "er"        Erdos-Renyi 15% density design of Sec 5.1, lambda = 0.2

    Seeds: graph seed 1000 + k, data seed 2000 + k, with k fixed per kind.
    """
    defaults = {"ar1": (200, 100, 1), "scalefree": (5000, 1000, 2),
                "hubblock": (40000, 1000, 3), "er": (300, 150, 6)}
    if kind not in defaults:
        raise ValueError(f"unknown workload kind {kind!r}")
    p0, n0, k0 = defaults[kind]
    p = p0 if p is None else p
    n = n0 if n is None else n
    k = k0 if k is None else k
    gseed, dseed = 1000 + k, 2000 + k
    if kind == "ar1":
        theta, lam = ar1_precision(p, 0.4), 0.2
        recipe = f"AR(1) chain rho=0.4, p={p}, n={n}, data seed {dseed}"
    elif kind == "scalefree":
        theta, lam = ba_tree_precision(p, gseed), 0.15
        recipe = f"BA tree m=1 +-U[0.1,0.4] unit diag, p={p}, n={n}, seeds {gseed}/{dseed}"
    elif kind == "hubblock":
        bsize = 200 if p >= 200 else p
        if p % bsize:
            raise ValueError("hubblock needs p to be a multiple of the 200-node block")
        theta = hub_block_precision(p // bsize, bsize, max(1, bsize // 10), gseed)
        lam = 0.1
        recipe = (f"hub-and-block {p // bsize}x{bsize}, hub->10% of block, +-U[0.2,0.5], "
                  f"diag rule 1.5, p={p}, n={n}, seeds {gseed}/{dseed}")
    else:
        theta, lam = er_precision(p, 0.15, gseed), 0.2
        recipe = f"ER 15% +-U[0.5,1], unit then U[1,sqrt3] diag scaling, p={p}, n={n}, seeds {gseed}/{dseed}"
    X = sample_gaussian(theta, n, dseed).astype(np.float32)
    return Workload(name=f"{kind}_p{p}_n{n}", X=np.ascontiguousarray(X), lam=lam, theta=theta, recipe=recipe)


WORKLOADS = {
    "ar1_p200_n100": dict(kind="ar1", p=200, n=100),
    "scalefree_p5000_n1000": dict(kind="scalefree", p=5000, n=1000),
    "hubblock_p40000_n1000": dict(kind="hubblock", p=40000, n=1000),
}


@dataclasses.dataclass
class PathWorkload:
    name: str
    X: np.ndarray            # float32, n_total x p (the whole data set)
    lambdas: np.ndarray      # penalties in solve order (decreasing)
    subsamples: list         # row-index arrays (bootstrap: drawn with replacement)
    kkt_tol: float
    recipe: str


def path_workload(p: int = 4000, n_total: int = 400, n_lambda: int = 32, n_sub: int = 16,
                  lam_lo: float = 0.05, lam_hi: float = 0.5, n_min: int = 200, n_max: int = 400,
                  kkt_tol: float = 1e-4, k: int = 4) -> PathWorkload:
    """Penalty grid x bootstrap subsamples of one scale-free data set: n_lambda
    penalties log-spaced from lam_hi down to lam_lo; n_sub subsamples whose
    sizes are uniform integers in [n_min, n_max], rows drawn with replacement
    from the n_total rows.  Seeds: graph 1000 + k, data 2000 + k, subsamples
    3000 + k."""
    theta = ba_tree_precision(p, 1000 + k)
    X = sample_gaussian(theta, n_total, 2000 + k).astype(np.float32)
    rng = _rng(3000 + k)
    sizes = rng.integers(n_min, n_max + 1, size=n_sub)
    subs = [rng.integers(0, n_total, size=int(m)) for m in sizes]
    lams = np.geomspace(lam_hi, lam_lo, n_lambda)
    recipe = (f"BA tree m=1 +-U[0.1,0.4] unit diag, p={p}, n_total={n_total}; {n_lambda} penalties log-spaced "
              f"{lam_hi}..{lam_lo}; {n_sub} bootstrap subsamples, n uniform in [{n_min},{n_max}]; "
              f"seeds {1000 + k}/{2000 + k}/{3000 + k}")
    return PathWorkload(name=f"path_p{p}_L{n_lambda}_S{n_sub}", X=np.ascontiguousarray(X), lambdas=lams,
                        subsamples=subs, kkt_tol=kkt_tol, recipe=recipe)


def ar1_random_precision(p: int, extra: float, weight: float, seed: int, rho: float = 0.4,
                         min_eig: float = 0.2) -> sp.csr_matrix:
    """Unit diagonal, AR(1) chain (rho off the diagonal) plus a random `extra`
    fraction of the other off-diagonal pairs with weights +-weight; the
    diagonal is then raised just enough for the smallest eigenvalue to be
    min_eig (the rule of the paper's Sec 5.2 simulations)."""
    rng = _rng(seed)
    iu, ju = np.triu_indices(p, k=2)
    take = rng.random(iu.size) < extra
    ri, rj = iu[take], ju[take]
    vals = _signed_uniform(rng, int(take.sum()), weight, weight)
    chain = np.arange(p - 1)
    rows = np.concatenate([chain, ri])
    cols = np.concatenate([chain + 1, rj])
    v = np.concatenate([np.full(p - 1, rho), vals])
    theta = (_assemble(p, rows, cols, v) + sp.eye(p)).tocsr()
    lmin = float(np.linalg.eigvalsh(theta.toarray())[0])
    if lmin < min_eig:
        theta = (theta + (min_eig - lmin) * sp.eye(p)).tocsr()
    return theta


@dataclasses.dataclass
class DiffWorkload:
    name: str
    X_train: np.ndarray      # float32, n x p
    X_val: np.ndarray        # float32, n_val x p (held out)
    lam: float
    theta: sp.csr_matrix
    recipe: str


def diff_workload(p: int = 2000, n: int = 300, n_val: int = 100, lam: float = 0.2, k: int = 5) -> DiffWorkload:
    """Training and held-out rows from one AR(1) + 1% random-edge precision
    (weights +-0.2).  Seeds: graph 1000 + k, data 2000 + k."""
    theta = ar1_random_precision(p, 0.01, 0.2, 1000 + k)
    X = sample_gaussian(theta, n + n_val, 2000 + k).astype(np.float32)
    recipe = (f"AR(1) rho=0.4 + 1% random edges +-0.2, min eigenvalue 0.2, p={p}, n={n} + {n_val} held out, "
              f"lambda={lam}, seeds {1000 + k}/{2000 + k}")
    return DiffWorkload(name=f"diff_p{p}_n{n}", X_train=np.ascontiguousarray(X[:n]),
                        X_val=np.ascontiguousarray(X[n:]), lam=lam, theta=theta, recipe=recipe)
