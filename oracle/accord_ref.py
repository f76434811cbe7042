"""Plain FP64 CPU oracle for ACCORD-FBS (HP-ACCORD, Sec 3).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
reference that the CUDA library is graded against.  Only the test-suite, the
package smoke check and the benchmark's CPU-baseline leg may import it; the
library never calls it and has no CPU fallback.

Notation follows the paper: X is n x p (rows are samples), S = X^T X / n,
Omega is p x p and asymmetric, g(Omega) = 1/2 tr(Omega^T Omega S) (Eq. 3.4),
h(Omega) = -log det Omega_D + lambda ||Omega||_1 (Eq. 3.4), f = g + h (Eq. 3.2).

Every array here is float64; numpy's matmul and symmetric eigensolver serve as
library primitives.  Nothing is blocked, fused or reordered beyond what the
definitions and Algorithm 1 state.

Readings of the paper taken here, where it is silent or ambiguous:
  * lambda penalises every entry, the diagonal included (Eq. 3.2; the diagonal
    prox of Eq. 3.5 carries tau*lambda).  `penalize_diag=False` drops it from
    the diagonal only.
  * The line-search inner product is <Delta, grad g(Omega^t)> (the proof of
    Thm 3.3 writes the gradient; Algorithm 1's printed "g" is a typo).
  * Since g is quadratic, g(Omega+) - g(Omega) - <Delta, grad g> equals
    ||Delta X^T||_F^2 / (2n) exactly, so the sufficient-decrease test is
    evaluated as ||Y+ - Y||^2 / n <= ||Delta||^2 / tau.  The printed form is
    computed alongside and returned in the log for comparison.
  * grad g does not depend on tau, so it is formed once per outer iteration.
  * tau_0 = 1, beta = 1/2, restart at tau_0 every outer iteration unless
    `tau_warm` (then min(tau_0, tau_{t-1}/beta)); beta == 1 is the fixed-step
    variant (every trial accepted).
  * Omega^0 = I.  Stopping: the KKT residual r(Omega^t) <= tol, checked before
    step t is taken; r is the max-abs entry of the minimum-norm element of the
    subdifferential of Eq. 3.3.
  * Diagonal root of Eq. 3.5 written in the cancellation-free form when
    b = y - tau*lambda < 0 (algebraically identical).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

OK, NOT_CONVERGED, EBACKTRACK, ENONFINITE = 0, 1, -4, -3


# ----------------------------------------------------------------- basics ---

def sample_covariance(X: np.ndarray) -> np.ndarray:
    """S = X^T X / n (Sec 2, sample covariance of the centred data matrix)."""
    X = np.asarray(X, dtype=np.float64)
    return X.T @ X / X.shape[0]


def smooth_g(Omega: np.ndarray, X: np.ndarray) -> float:
    """g(Omega) = 1/2 tr(Omega^T Omega S) = ||Omega X^T||_F^2 / (2n) (Eq. 3.4)."""
    X = np.asarray(X, dtype=np.float64)
    Y = Omega @ X.T
    return float(np.sum(Y * Y)) / (2.0 * X.shape[0])


def grad_g(Omega: np.ndarray, X: np.ndarray) -> np.ndarray:
    """grad g(Omega) = Omega S, formed in the two steps Y = Omega X^T and
    (1/n) Y X (Remark after Thm 3.3; Sec 3.3)."""
    X = np.asarray(X, dtype=np.float64)
    Y = Omega @ X.T
    return Y @ X / X.shape[0]


def diag_entries(Omega: np.ndarray, row0: int = 0) -> np.ndarray:
    """Entries omega_ii of a block of rows [row0, row0 + m) of Omega: the
    entries of Omega_D in the log-barrier -log det Omega_D of Eq. 3.2."""
    m = Omega.shape[0]
    idx = np.arange(m)
    return Omega[idx, row0 + idx]


def offdiag_penalty(Omega: np.ndarray, lam, row0: int = 0) -> float:
    """sum_{i != j} lambda_ij |omega_ij|; lam is a scalar or a matrix of
    per-entry weights (np.inf allowed where omega_ij must be 0, Eq. 3.8)."""
    m = Omega.shape[0]
    off = np.ones(Omega.shape, dtype=bool)
    off[np.arange(m), row0 + np.arange(m)] = False
    w = np.broadcast_to(np.asarray(lam, dtype=np.float64), Omega.shape)
    nz = off & (Omega != 0)
    return float(np.sum(w[nz] * np.abs(Omega[nz])))


def objective(Omega: np.ndarray, X: np.ndarray, lam, penalize_diag: bool = True, lam_diag=None) -> float:
    """f(Omega) = -sum log omega_ii + 1/2 tr(Omega^T Omega S) + lambda ||Omega||_1
    (Eq. 3.2).  +inf outside dom f (some omega_ii <= 0).  lam may be a matrix
    of off-diagonal weights; lam_diag overrides the diagonal weight."""
    d = np.diag(Omega)
    if np.any(d <= 0):
        return math.inf
    lam_d = lam_diag if lam_diag is not None else (float(lam) if penalize_diag else 0.0)
    return smooth_g(Omega, X) - float(np.sum(np.log(d))) + offdiag_penalty(Omega, lam) + lam_d * float(d.sum())


def soft_threshold(x: np.ndarray, a: float) -> np.ndarray:
    """S_a(x) = (|x| - a)_+ sign(x) (Eq. 3.5)."""
    return np.sign(x) * np.maximum(np.abs(x) - a, 0.0)


def diag_prox(y: np.ndarray, tau: float, lam_d: float) -> np.ndarray:
    """Diagonal update of Eq. 3.5: the positive root of w^2 - b w - tau = 0 with
    b = y - tau*lambda, i.e. w = (b + sqrt(b^2 + 4 tau)) / 2; for b < 0 the
    equal value 2 tau / (sqrt(b^2 + 4 tau) - b) is used."""
    b = y - tau * lam_d
    root = np.sqrt(b * b + 4.0 * tau)
    return np.where(b >= 0, 0.5 * (b + root), 2.0 * tau / (root - b))


def prox(A: np.ndarray, tau: float, lam, lam_d: float, row0: int = 0) -> np.ndarray:
    """Backward step of Eq. 3.5 applied to A = Omega - tau * grad g(Omega):
    soft-threshold off the diagonal, log-barrier root on it.  `row0` places a
    block of rows [row0, row0 + m) inside the full matrix.  lam may be a
    matrix of per-entry weights; an infinite weight gives 0 (Eq. 3.8)."""
    out = soft_threshold(A, tau * np.asarray(lam, dtype=np.float64))
    m = A.shape[0]
    idx = np.arange(m)
    out[idx, row0 + idx] = diag_prox(A[idx, row0 + idx], tau, lam_d)
    return out


def kkt_residual(Omega: np.ndarray, G: np.ndarray, lam, lam_d: float, row0: int = 0) -> float:
    """max_ij of the minimum-norm element of the subdifferential of f (Eq. 3.3,
    with z_ii = 1 and z_ij in [-1, 1] at zero entries):
      diagonal            |G_ii - 1/omega_ii + lambda_d|
      omega_ij != 0       |G_ij + lambda sign(omega_ij)|
      omega_ij == 0       max(|G_ij| - lambda, 0)."""
    lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), Omega.shape)
    with np.errstate(invalid="ignore"):
        R = np.where(Omega != 0, np.abs(G + lam * np.sign(Omega)), np.maximum(np.abs(G) - lam, 0.0))
    m = Omega.shape[0]
    idx = np.arange(m)
    d = Omega[idx, row0 + idx]
    R[idx, row0 + idx] = np.abs(G[idx, row0 + idx] - 1.0 / d + lam_d)
    return float(R.max()) if R.size else 0.0


def lipschitz(X: np.ndarray) -> float:
    """L = sigma_max(S) = lambda_max(X X^T) / n (Sec 3.2); the n x n Gram has
    the same nonzero spectrum as S."""
    X = np.asarray(X, dtype=np.float64)
    K = X @ X.T / X.shape[0]
    return float(np.linalg.eigvalsh(K)[-1])


# ------------------------------------------------------------ Algorithm 1 ---

def fbs_trial(Omega: np.ndarray, Y: np.ndarray, G: np.ndarray, X: np.ndarray, tau: float, lam: float,
              lam_d: float, row0: int = 0):
    """One trial of Algorithm 1's inner loop: forward step A = Omega - tau G,
    backward step of Eq. 3.5, Delta = Omega+ - Omega and Y+ = Omega+ X^T.
    Returns (Omega+, Y+, ||Delta||^2, ||Y+ - Y||^2, g(Omega+), <Delta, G>).
    Works on a block of rows [row0, row0 + m) as well (the objective separates
    over the rows of Omega)."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    A = Omega - tau * G                      # forward step
    Op = prox(A, tau, lam, lam_d, row0)      # backward step, Eq. 3.5
    Delta = Op - Omega
    Yp = Op @ X.T
    d2 = float(np.sum(Delta * Delta))
    dy2 = float(np.sum((Yp - Y) ** 2))
    gp = float(np.sum(Yp * Yp)) / (2.0 * n)
    dG = float(np.sum(Delta * G))
    return Op, Yp, d2, dy2, gp, dG


@dataclasses.dataclass
class FitResult:
    """Output of `fit`: the last iterate of Algorithm 1 and its per-iteration
    log (objective of Eq. 3.2, KKT residual of Eq. 3.3, accepted steps)."""
    Omega: np.ndarray
    status: int
    iters: int                 # accepted steps taken
    trials: int                # prox evaluations (accepted + rejected)
    L: float
    f: list                    # f(Omega^t), t = 0..iters
    kkt: list                  # r(Omega^t), t = 0..iters
    tau: list                  # accepted tau_t, t = 0..iters-1
    ntrials: list              # trials spent on step t
    nnz: list                  # off-diagonal nonzeros of Omega^t
    delta_fro: list            # ||Omega^{t+1} - Omega^t||_F
    margin: list               # accepted test: ||Delta||^2/tau - ||Y+ - Y||^2/n
    printed_form_agrees: list  # per trial: printed Alg. 1 test gives the same verdict


def fit(X: np.ndarray, lam, *, tau0: float = 1.0, beta: float = 0.5, tau_warm: bool = False,
        max_iter: int = 500, max_backtracks: int = 60, kkt_tol: float = 1e-8,
        penalize_diag: bool = True, Omega0: np.ndarray | None = None, L: float | None = None,
        lam_diag: float | None = None) -> FitResult:
    """ACCORD-FBS with backtracking (Algorithm 1, update Eq. 3.5).  lam is the
    penalty weight, or a p x p matrix of off-diagonal weights (Eq. 3.8 refit);
    lam_diag overrides the diagonal weight."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    lam_d = lam_diag if lam_diag is not None else (float(lam) if penalize_diag else 0.0)
    if L is None:
        L = lipschitz(X)
    if tau0 <= 0:
        tau0 = 1.0 / L
    Omega = np.eye(p) if Omega0 is None else np.array(Omega0, dtype=np.float64)
    Y = Omega @ X.T
    G = Y @ X / n
    g = float(np.sum(Y * Y)) / (2.0 * n)

    res = FitResult(Omega, NOT_CONVERGED, 0, 0, L, [], [], [], [], [], [], [], [])
    t = 0
    tau_prev = tau0
    while True:
        d = np.diag(Omega)
        f = g - float(np.sum(np.log(d))) + offdiag_penalty(Omega, lam) + lam_d * float(d.sum())
        r = kkt_residual(Omega, G, lam, lam_d)
        res.f.append(f)
        res.kkt.append(r)
        res.nnz.append(int(np.count_nonzero(Omega)) - int(np.count_nonzero(d)))
        if not (math.isfinite(f) and math.isfinite(r)):
            res.status = ENONFINITE
            break
        if r <= kkt_tol:
            res.status = OK
            break
        if t >= max_iter:
            res.status = NOT_CONVERGED
            break
        tau = min(tau0, tau_prev / beta) if (tau_warm and t > 0) else tau0
        accepted = False
        for k in range(max_backtracks + 1):
            res.trials += 1
            Op, Yp, d2, dy2, gp, dG = fbs_trial(Omega, Y, G, X, tau, lam, lam_d)
            ok_diff = dy2 / n <= d2 / tau
            ok_printed = gp <= g + dG + d2 / (2.0 * tau)
            res.printed_form_agrees.append(ok_diff == ok_printed)
            if ok_diff or tau <= 1.0 / L or beta == 1.0:
                accepted = True
                res.margin.append(d2 / tau - dy2 / n)
                break
            tau *= beta
        if not accepted:
            res.status = EBACKTRACK
            break
        res.tau.append(tau)
        res.ntrials.append(k + 1)
        res.delta_fro.append(math.sqrt(d2))
        Omega, Y, g = Op, Yp, gp
        G = Y @ X / n
        tau_prev = tau
        t += 1
    res.Omega = Omega
    res.iters = t
    return res


# -------------------------------------------------------- Sec 3.4 and 3.5 ---

def epbic(Omega: np.ndarray, X: np.ndarray, gamma: float) -> float:
    """Extended pseudo-BIC of Eq. 3.7:
    2n { -log det Omega_D + 1/2 tr(Omega^T Omega S) } + ||Omega||_0 log n
    + 4 gamma ||Omega||_0 log p, with ||.||_0 the off-diagonal nonzeros."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    d = np.diag(Omega)
    l0 = int(np.count_nonzero(Omega)) - int(np.count_nonzero(d))
    return 2.0 * n * (-float(np.sum(np.log(d))) + smooth_g(Omega, X)) + l0 * math.log(n) + 4.0 * gamma * l0 * math.log(p)


def refit(X: np.ndarray, lam: float, support: np.ndarray, phi: float, *, penalize_diag: bool = True,
          **kw) -> FitResult:
    """Bias-corrected refit of Eq. 3.8: Algorithm 1 with the weight phi*lambda
    on the support (the diagonal always belongs to it) and infinity off it."""
    p = support.shape[0]
    sup = np.asarray(support, dtype=bool) | np.eye(p, dtype=bool)
    W = np.where(sup, phi * lam, np.inf)
    return fit(X, W, lam_diag=(phi * lam if penalize_diag else 0.0), **kw)


# ------------------------------------------------------- lambda path (3.4) ---

@dataclasses.dataclass
class PathResult:
    """Output of `lambda_path` (Sec 3.4): every estimate of the grid and the
    one each subsample selects by the smallest epBIC (Eq. 3.7)."""
    lambdas: list              # penalty values, in the order they were solved
    fits: list                 # fits[s][k]: FitResult of subsample s at lambdas[k]
    epbic: np.ndarray          # (n_lambda, n_sub) Eq. 3.7 of each estimate
    best: list                 # per subsample: index k of the smallest epBIC
    Omega_best: list           # per subsample: the estimate at that index


def lambda_path(X: np.ndarray, rows: list, lambdas, *, gamma: float = 0.5, cold_every: int = 0,
                **fit_kw) -> PathResult:
    """Sec 3.4 tuning on subsamples of one data set.  Subsample s is the data
    matrix X[rows[s]] (indices may repeat: a bootstrap sample).  For each
    subsample the penalties are solved in the given order, each fit starting
    from the previous estimate (warm start; cold_every = c > 0 restarts from
    Omega = I at every c-th penalty instead), and each estimate is scored by
    epBIC; the subsample's selected estimate minimises it."""
    X = np.asarray(X, dtype=np.float64)
    lambdas = [float(v) for v in lambdas]
    ns = len(rows)
    fits = []
    score = np.zeros((len(lambdas), ns))
    best, Omega_best = [], []
    for s in range(ns):
        Xs = X[np.asarray(rows[s], dtype=np.int64)]
        chain = []
        Om = None
        for k, lam in enumerate(lambdas):
            if cold_every > 0 and k % cold_every == 0:
                Om = None
            r = fit(Xs, lam, Omega0=Om, **fit_kw)
            chain.append(r)
            score[k, s] = epbic(r.Omega, Xs, gamma)
            Om = r.Omega
        fits.append(chain)
        kb = int(np.argmin(score[:, s]))
        best.append(kb)
        Omega_best.append(chain[kb].Omega)
    return PathResult(lambdas, fits, score, best, Omega_best)


# ------------------------------------------------------ post-processing ---

def theta_hat(Omega: np.ndarray) -> np.ndarray:
    """Theta-hat = T^-1(Omega-hat) = Omega_D Omega (Sec 3.1): theta_ij = omega_ii omega_ij."""
    return np.diag(Omega)[:, None] * Omega


def partial_correlation(Omega: np.ndarray) -> np.ndarray:
    """rho_ij = -(1/2)(omega_ij / omega_jj + omega_ji / omega_ii) off the
    diagonal (Sec 3.1); the diagonal is 1 by convention."""
    d = np.diag(Omega)
    R = -0.5 * (Omega / d[None, :] + Omega.T / d[:, None])
    np.fill_diagonal(R, 1.0)
    return R


# ------------------------------------------------------ differentiation ---

def smooth_loss(Omega: np.ndarray, X: np.ndarray) -> float:
    """The pseudolikelihood part of Eq. 3.2 without the penalty:
    L(Omega; X) = -sum_i log omega_ii + 1/2 tr(Omega^T Omega S)."""
    return -float(np.sum(np.log(np.diag(Omega)))) + smooth_g(Omega, X)


def smooth_loss_grad_omega(Omega: np.ndarray, X: np.ndarray) -> np.ndarray:
    """dL/dOmega = -diag(1/omega_ii) + Omega S (Sec 3.2 gradient plus the log term)."""
    return grad_g(Omega, X) - np.diag(1.0 / np.diag(Omega))


def smooth_loss_grad_x(Omega: np.ndarray, X: np.ndarray) -> np.ndarray:
    """dL/dX of the smooth part of Eq. 3.2: only g (Eq. 3.4) depends on X,
    and g = ||Omega X^T||_F^2 / (2n), so
    dL/dX = (1/n) (Omega X^T)^T Omega = (1/n) X Omega^T Omega."""
    X = np.asarray(X, dtype=np.float64)
    return (Omega @ X.T).T @ Omega / X.shape[0]


def implicit_dloglam(Omega_hat: np.ndarray, X_train: np.ndarray, X_val: np.ndarray, lam: float,
                     penalize_diag: bool = True):
    """d L(Omega-hat(lambda); X_val) / d log(lambda) by implicit differentiation
    of the stationarity conditions (Eq. 3.3) on the active set.  The
    objective separates over rows (proof of Thm 3.2, vectorised form); on row
    i with active set A (nonzero entries, i included) and fixed signs s the
    conditions read S_AA w - (1/w_i) e_i + lambda v = 0, v_j = s_j (j != i),
    v_i = 1 when the diagonal is penalised (else 0).  Differentiating in
    lambda gives (S_AA + w_i^-2 e_i e_i^T) dw/dlambda = -v.  Returns the
    derivative and the p x p matrix dOmega-hat / dlog(lambda)."""
    S = sample_covariance(X_train)
    Gv = smooth_loss_grad_omega(Omega_hat, X_val)
    p = Omega_hat.shape[0]
    dOm = np.zeros((p, p))
    for i in range(p):
        A = np.nonzero(Omega_hat[i] != 0)[0]
        pos = int(np.nonzero(A == i)[0][0])
        w = Omega_hat[i, A]
        H = S[np.ix_(A, A)].copy()
        H[pos, pos] += 1.0 / (w[pos] * w[pos])
        v = np.sign(w)
        v[pos] = 1.0 if penalize_diag else 0.0
        dOm[i, A] = -lam * np.linalg.solve(H, v)
    return float(np.sum(Gv * dOm)), dOm


# --------------------------------------------------------- exact row solve ---

def row_solution(S: np.ndarray, i: int, active: np.ndarray, signs: np.ndarray,
                 lam: float, lam_d: float) -> np.ndarray | None:
    """Row i of the minimiser on a given support.  f separates over the rows of
    Omega (proof of Thm 3.2, vectorised objective); restricted to an active set
    A (containing i) with fixed signs s, the stationarity condition of Eq. 3.3 is
    S_AA w_A = (1/w_i) e_i - v with v_j = lambda s_j (j != i), v_i = lambda_d.
    With c = S_AA^-1 e_i and d = S_AA^-1 v this gives w_i^2 + d_i w_i - c_i = 0,
    w_i = (-d_i + sqrt(d_i^2 + 4 c_i)) / 2 and w_A = c / w_i - d.
    Returns the dense row (zeros off A), or None if S_AA is singular."""
    p = S.shape[0]
    A = np.asarray(active, dtype=np.int64)
    pos = int(np.nonzero(A == i)[0][0])
    SAA = S[np.ix_(A, A)]
    v = lam * np.asarray(signs, dtype=np.float64).copy()
    v[pos] = lam_d
    e = np.zeros(A.size)
    e[pos] = 1.0
    try:
        c = np.linalg.solve(SAA, e)
        d = np.linalg.solve(SAA, v)
    except np.linalg.LinAlgError:
        return None
    if c[pos] <= 0:
        return None
    wi = 0.5 * (-d[pos] + math.sqrt(d[pos] ** 2 + 4.0 * c[pos]))
    w = c / wi - d
    w[pos] = wi
    row = np.zeros(p)
    row[A] = w
    return row


def polish(Omega: np.ndarray, S: np.ndarray, lam: float, lam_d: float, rows=None) -> np.ndarray:
    """Re-solve each requested row exactly on the support and signs of Omega
    (row_solution: Eq. 3.3 restricted to the row's active set; f separates
    over rows, proof of Thm 3.2); a converged Omega becomes the minimiser to
    rounding."""
    out = np.array(Omega, dtype=np.float64)
    p = Omega.shape[0]
    for i in (range(p) if rows is None else rows):
        A = np.nonzero(Omega[i] != 0)[0]
        if i not in A:
            A = np.sort(np.append(A, i))
        s = np.sign(Omega[i, A])
        r = row_solution(S, i, A, s, lam, lam_d)
        if r is not None:
            out[i] = r
    return out


def brute_force(S: np.ndarray, lam: float, lam_d: float) -> np.ndarray:
    """Exact minimiser for tiny p (p <= 3): for each row enumerate all 3^(p-1)
    sign patterns of the off-diagonal entries, solve each with row_solution,
    keep the patterns that satisfy Eq. 3.3 (signs consistent, |(S w)_j| <= lambda
    off the support) and return the one with the smallest row objective."""
    p = S.shape[0]
    if p > 3:
        raise ValueError("brute force is meant for p <= 3")
    Om = np.zeros((p, p))
    for i in range(p):
        others = [j for j in range(p) if j != i]
        best, best_val = None, math.inf
        for code in range(3 ** len(others)):
            pat, c = [], code
            for _ in others:
                pat.append(c % 3 - 1)
                c //= 3
            act = sorted([i] + [j for j, s in zip(others, pat) if s != 0])
            sg = np.array([1.0 if j == i else float(pat[others.index(j)]) for j in act])
            w = row_solution(S, i, np.array(act), sg, lam, lam_d)
            if w is None:
                continue
            ok = all(np.sign(w[j]) == pat[others.index(j)] for j in act if j != i)
            Sw = S @ w
            ok = ok and all(abs(Sw[j]) <= lam * (1 + 1e-12) + 1e-14 for j in others if w[j] == 0)
            if not ok:
                continue
            val = row_objective(S, i, w, lam, lam_d)
            if val < best_val:
                best, best_val = w, val
        Om[i] = best
    return Om


def row_objective(S: np.ndarray, i: int, w: np.ndarray, lam: float, lam_d: float) -> float:
    """Row i's share of f (Eq. 3.2 split over the rows of Omega, proof of
    Thm 3.2): -log w_i + 1/2 w^T S w + lambda sum_{j != i} |w_j| + lambda_d w_i."""
    if w[i] <= 0:
        return math.inf
    off = np.abs(w).sum() - abs(w[i])
    return -math.log(w[i]) + 0.5 * float(w @ S @ w) + lam * off + lam_d * w[i]
