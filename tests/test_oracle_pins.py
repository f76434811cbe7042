"""Pins for the FP64 oracle: closed forms, invariants and brute force that the
paper and the mathematics fix independently of the oracle's own code.

Each `pin_*` function returns True when the oracle satisfies it; the tests
assert them, and the planted-mistake tests at the bottom swap one oracle
function for a plausible mistake and check that some pin then fails.
"""

import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import accord_ref as R
from synth import orthogonal_design, workload

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _gauss(n, p, seed):
    return np.random.Generator(np.random.PCG64(seed)).standard_normal((n, p))


# ------------------------------------------------------------------ pins ---

def pin_prox_root():
    """Eq. 3.5 diagonal: the root solves w^2 - b w - tau = 0 and minimises
    -tau log w + tau lambda w + (w - y)^2 / 2 (scalar brute minimisation)."""
    ok = True
    for y, tau, lam in [(0.3, 1.0, 0.2), (-2.0, 0.5, 0.1), (5.0, 0.01, 0.0), (-40.0, 2.0, 0.3)]:
        w = float(R.diag_prox(np.array([y]), tau, lam)[0])
        b = y - tau * lam
        ok &= abs(w * w - b * w - tau) <= 1e-12 * max(1.0, w * w, abs(b * w))
        res = so.minimize_scalar(lambda v: -tau * math.log(v) + tau * lam * v + 0.5 * (v - y) ** 2,
                                 bounds=(1e-12, 100.0), method="bounded", options={"xatol": 1e-12})
        ok &= abs(res.x - w) <= 1e-6 * max(1.0, w)
    return bool(ok)


def pin_soft_threshold():
    """S_a(x) minimises a|w| + (w - x)^2 / 2 (checked on a fine grid)."""
    grid = np.linspace(-3, 3, 600001)
    ok = True
    for x, a in [(1.3, 0.4), (-0.2, 0.5), (-2.0, 0.25), (0.5, 0.5)]:
        w = float(R.soft_threshold(np.array([x]), a)[0])
        v = a * np.abs(grid) + 0.5 * (grid - x) ** 2
        ok &= abs(grid[np.argmin(v)] - w) <= 2e-5
    return bool(ok)


def pin_gradient():
    """grad g = Omega S with S = X^T X / n formed explicitly, and equal to the
    central finite difference of g."""
    X = _gauss(7, 5, 11)
    Om = _gauss(5, 5, 12)
    S = X.T @ X / 7
    G = R.grad_g(Om, X)
    ok = np.allclose(G, Om @ S, rtol=1e-13, atol=1e-13)
    ok &= abs(R.smooth_g(Om, X) - 0.5 * np.trace(Om.T @ Om @ S)) <= 1e-12
    h = 1e-6
    for (i, j) in [(0, 0), (1, 3), (4, 2)]:
        E = np.zeros_like(Om)
        E[i, j] = h
        fd = (R.smooth_g(Om + E, X) - R.smooth_g(Om - E, X)) / (2 * h)
        ok &= abs(fd - G[i, j]) <= 1e-7
    return bool(ok)


def pin_lipschitz():
    """L = sigma_max(S): largest singular value of the explicitly formed S."""
    X = _gauss(9, 14, 13)
    S = X.T @ X / 9
    return abs(R.lipschitz(X) - np.linalg.norm(S, 2)) <= 1e-12 * np.linalg.norm(S, 2)


def pin_f_identity():
    """f(I) = tr(S)/2 + lambda p (condition of Thm 3.3)."""
    X = _gauss(6, 8, 14)
    S = X.T @ X / 6
    lam = 0.37
    return abs(R.objective(np.eye(8), X, lam) - (np.trace(S) / 2 + lam * 8)) <= 1e-12


def pin_objective_diagonal():
    """f at a diagonal Omega = diag(d), away from I: tr(Omega^T Omega S) keeps
    only d_i^2 s_ii, so f = 1/2 sum d_i^2 s_ii - sum log d_i + lambda sum d_i
    (Eq. 3.2), whatever the off-diagonal entries of S.  Per coordinate that is
    1/2 s d^2 - log d + lambda d, minimised at d = (-lambda + sqrt(lambda^2 +
    4 s)) / (2 s); f there lies below f one percent to either side."""
    X = _gauss(30, 6, 33)
    S = X.T @ X / 30
    s = np.diag(S)
    lam = 0.21
    d = np.random.Generator(np.random.PCG64(34)).uniform(0.3, 3.0, size=6)
    want = 0.5 * np.sum(d * d * s) - np.sum(np.log(d)) + lam * np.sum(d)
    ok = abs(R.objective(np.diag(d), X, lam) - want) <= 1e-12 * abs(want)
    dstar = (-lam + np.sqrt(lam * lam + 4 * s)) / (2 * s)
    f0 = R.objective(np.diag(dstar), X, lam)
    ok &= f0 < R.objective(np.diag(1.01 * dstar), X, lam) and f0 < R.objective(np.diag(0.99 * dstar), X, lam)
    return bool(ok)


def pin_diagonal_S():
    """Diagonal S: omega_ii = (-lambda + sqrt(lambda^2 + 4 s_i)) / (2 s_i) and
    omega_ij = 0 (Eq. 3.3 with z_ii = 1); without the diagonal penalty
    omega_ii = 1 / sqrt(s_i)."""
    s = np.random.Generator(np.random.PCG64(15)).uniform(0.4, 2.5, size=9)
    X = orthogonal_design(40, s, 16)
    ok = True
    for pen in (True, False):
        lam = 0.3
        r = R.fit(X, lam, kkt_tol=1e-13, max_iter=2000, penalize_diag=pen)
        ld = lam if pen else 0.0
        want = (-ld + np.sqrt(ld * ld + 4 * s)) / (2 * s)
        ok &= r.status == R.OK
        ok &= np.max(np.abs(np.diag(r.Omega) - want)) <= 1e-11
        ok &= np.max(np.abs(r.Omega - np.diag(np.diag(r.Omega)))) <= 1e-12
    return bool(ok)


def pin_diagonal_penalty_both_ways():
    """The chain workload (p = 200, n = 100, lambda = 0.2) fitted with and
    without lambda on the diagonal (Eq. 3.2 as printed, and the off-diagonal
    reading).  Each fit meets the KKT conditions of its own objective.  f
    separates over rows and the diagonal penalty adds lambda * omega_ii, a term
    increasing in omega_ii, to row i's objective, so no diagonal entry grows
    when it is added.  Also, since f_1 = f_0 + lambda tr(Omega) with
    omega_ii > 0, f_0(Omega-hat_0) < f_1(Omega-hat_1) <= f_1(Omega-hat_0)."""
    w = workload("ar1")
    X = w.X.astype(np.float64)
    S = X.T @ X / X.shape[0]
    fits = {}
    ok = True
    for pen in (True, False):
        lam_d = w.lam if pen else 0.0
        r = R.fit(X, w.lam, kkt_tol=1e-10, max_iter=5000, penalize_diag=pen)
        ok &= r.status == R.OK
        O = R.polish(r.Omega, S, w.lam, lam_d)
        ok &= R.kkt_residual(O, R.grad_g(O, X), w.lam, lam_d) <= 1e-11
        fits[pen] = O
    O1, O0 = fits[True], fits[False]
    ok &= bool(np.all(np.diag(O1) <= np.diag(O0) + 1e-12))
    ok &= bool(np.sum(np.diag(O0) - np.diag(O1)) > 1e-3)
    f0 = R.objective(O0, X, w.lam, penalize_diag=False)
    f1 = R.objective(O1, X, w.lam, penalize_diag=True)
    ok &= f0 < f1 <= R.objective(O0, X, w.lam, penalize_diag=True) + 1e-12
    return bool(ok)


def pin_identity_S():
    """S = I and lambda = 0 give Omega-hat = I (reached from a perturbed start)."""
    X = orthogonal_design(30, np.ones(6), 17)
    Om0 = np.eye(6) + 0.05 * _gauss(6, 6, 18)
    r = R.fit(X, 0.0, kkt_tol=1e-13, max_iter=3000, Omega0=Om0)
    return r.status == R.OK and np.max(np.abs(r.Omega - np.eye(6))) <= 1e-11


def pin_low_dim_closed_form():
    """lambda = 0, n > p: Omega-hat = diag(S^-1)^(-1/2) S^-1 (Sec 3.1)."""
    X = _gauss(80, 12, 19)
    S = X.T @ X / 80
    Th = np.linalg.inv(S)
    want = np.diag(1 / np.sqrt(np.diag(Th))) @ Th
    r = R.fit(X, 0.0, kkt_tol=1e-12, max_iter=20000)
    return r.status == R.OK and np.max(np.abs(r.Omega - want)) <= 1e-9 * np.max(np.abs(want))


def pin_brute_force():
    """p <= 3: the solver's limit equals the sign-pattern enumeration, and the
    enumeration's rows match a derivative-free minimisation of the row objective."""
    ok = True
    for seed, (n, p, lam) in [(20, (10, 3, 0.3)), (21, (4, 3, 0.05)), (22, (6, 2, 0.2)), (23, (5, 3, 0.8))]:
        X = _gauss(n, p, seed)
        S = X.T @ X / n
        for pen in (True, False):
            ld = lam if pen else 0.0
            bf = R.brute_force(S, lam, ld)
            r = R.fit(X, lam, kkt_tol=1e-13, max_iter=20000, penalize_diag=pen)
            ok &= r.status == R.OK
            ok &= np.max(np.abs(r.Omega - bf)) <= 1e-9
            for i in range(p):
                obj = lambda w: R.row_objective(S, i, w, lam, ld)  # noqa: E731
                best = min((so.minimize(obj, x0, method="Nelder-Mead",
                                        options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 40000})
                            for x0 in (np.eye(p)[i], bf[i] + 0.1)), key=lambda q: q.fun)
                ok &= best.fun >= obj(bf[i]) - 1e-10
                ok &= np.max(np.abs(best.x - bf[i])) <= 1e-4
    return bool(ok)


def pin_kkt_descent_path():
    """On a chain workload: f decreases on every accepted step (Thm 3.3),
    f(Omega^0 = I) = tr(S)/2 + lambda p, the returned iterate satisfies the
    KKT tolerance, and the exact row solve on its support moves it by less
    than the tolerance allows."""
    w = workload("ar1", p=60, n=40)
    X = w.X.astype(np.float64)
    S = X.T @ X / X.shape[0]
    r = R.fit(X, w.lam, kkt_tol=1e-10, max_iter=5000)
    f = np.array(r.f)
    ok = r.status == R.OK
    ok &= bool(np.all(np.diff(f) <= 1e-12 * np.abs(f[:-1])))
    ok &= abs(f[0] - (np.trace(S) / 2 + w.lam * X.shape[1])) <= 1e-10
    G = R.grad_g(r.Omega, X)
    ok &= R.kkt_residual(r.Omega, G, w.lam, w.lam) <= 1e-10
    P = R.polish(r.Omega, S, w.lam, w.lam)
    ok &= R.kkt_residual(P, R.grad_g(P, X), w.lam, w.lam) <= 1e-12
    ok &= np.max(np.abs(P - r.Omega)) <= 1e-8
    return bool(ok)


def _tail_slopes(e, floor):
    """Slopes of log e over the middle and last thirds of the iterations where
    e stays above the rounding floor."""
    t = np.nonzero(e > floor)[0]
    k = len(t) // 3
    return [np.polyfit(tt, np.log(e[tt]), 1)[0] for tt in (t[k:2 * k], t[2 * k:])]


def pin_linear_rate():
    """Thm 3.3, both step-size cases (i: beta = 1, tau = 1/L; ii: backtracking
    with beta = 1/2): f(Omega^t) - f* decays at a steady geometric rate, with
    f* taken from the exact row solve on the converged support; the steps
    ||Omega^(t+1) - Omega^t|| decay geometrically too (the iterate bound)."""
    w = workload("ar1", p=60, n=40)
    X = w.X.astype(np.float64)
    S = X.T @ X / X.shape[0]
    L = R.lipschitz(X)
    ok = True
    for kw in (dict(beta=1.0, tau0=1.0 / L), dict(beta=0.5)):
        r = R.fit(X, w.lam, kkt_tol=1e-13, max_iter=20000, **kw)
        ok &= r.status == R.OK
        P = R.polish(r.Omega, S, w.lam, w.lam)
        f_star = R.objective(P, X, w.lam)
        e = np.array(r.f) - f_star
        ok &= bool(e.min() >= -1e-13 * abs(f_star))
        for ee, floor in ((e, 1e-11 * abs(f_star)), (np.array(r.delta_fro), 1e-9)):
            s1, s2 = _tail_slopes(ee, floor)
            ok &= s1 < 0 and s2 < 0 and abs(s1 - s2) <= 0.25 * abs(s2)
    return bool(ok)


def pin_sufficient_decrease():
    """Every accepted step decreases f by at least ||Omega^(t+1) - Omega^t||_F^2
    / (2 tau_t): with the quadratic bound of Algorithm 1's test holding at
    Omega^(t+1), the prox step's optimality gives that decrease.  Steps never
    fall below tau_min = min(tau_0, beta / L) (Thm 3.3, case ii), and with
    beta = 1 every step is tau_0.  With tau_warm each step starts from
    min(tau_0, tau_(t-1) / beta) and only shrinks from there."""
    w = workload("ar1", p=60, n=40)
    X = w.X.astype(np.float64)
    L = R.lipschitz(X)
    ok = True
    for kw in (dict(beta=0.5), dict(beta=0.5, tau0=3.0), dict(beta=1.0, tau0=1.0 / L),
               dict(beta=0.5, tau0=3.0, tau_warm=True)):
        r = R.fit(X, w.lam, kkt_tol=1e-9, max_iter=5000, **kw)
        ok &= r.status == R.OK
        f, tau, dfro = np.array(r.f), np.array(r.tau), np.array(r.delta_fro)
        drop = f[:-1] - f[1:]
        ok &= bool(np.all(drop >= dfro ** 2 / (2 * tau) - 1e-12 * np.abs(f[:-1])))
        tau0, beta = kw.get("tau0", 1.0), kw["beta"]
        ok &= bool(np.all(tau >= min(tau0, beta / L) * (1 - 1e-15)))
        if beta == 1.0:
            ok &= bool(np.all(tau == tau0))
        if kw.get("tau_warm"):
            ok &= bool(np.all(tau[1:] <= np.minimum(tau0, tau[:-1] / beta) * (1 + 1e-15)))
    return bool(ok)


def pin_line_search_identity():
    """g(O+) - g(O) - <Delta, grad g(O)> = ||Delta X^T||^2 / (2n) (g is quadratic),
    so the printed and difference forms of the test agree away from rounding."""
    X = _gauss(11, 9, 24)
    O = _gauss(9, 9, 25)
    D = 0.1 * _gauss(9, 9, 26)
    lhs = R.smooth_g(O + D, X) - R.smooth_g(O, X) - float(np.sum(D * R.grad_g(O, X)))
    rhs = float(np.sum((D @ X.T) ** 2)) / (2 * 11)
    return abs(lhs - rhs) <= 1e-12 * max(1.0, abs(rhs))


def pin_refit_fixed_point():
    """Eq. 3.8 with phi = 1 on the support of Omega-hat(lambda) returns
    Omega-hat(lambda): it already satisfies the refit's KKT conditions."""
    w = workload("ar1", p=50, n=35)
    r = R.fit(w.X, w.lam, kkt_tol=1e-11, max_iter=8000)
    rr = R.refit(w.X, w.lam, r.Omega != 0, 1.0, kkt_tol=1e-11, max_iter=8000)
    return r.status == R.OK and rr.status == R.OK and np.max(np.abs(rr.Omega - r.Omega)) <= 1e-9


def pin_refit_restricted_mle():
    """Eq. 3.8 with phi = 0 is the unpenalised fit restricted to the support:
    each row equals the exact row solution on it (lambda = 0)."""
    w = workload("ar1", p=50, n=35)
    X = w.X.astype(np.float64)
    S = X.T @ X / X.shape[0]
    r = R.fit(w.X, w.lam, kkt_tol=1e-10, max_iter=8000)
    sup = r.Omega != 0
    r0 = R.refit(w.X, w.lam, sup, 0.0, kkt_tol=1e-11, max_iter=40000)
    exact = np.zeros_like(r0.Omega)
    for i in range(S.shape[0]):
        A = np.nonzero(sup[i])[0]
        exact[i] = R.row_solution(S, i, A, np.sign(r0.Omega[i, A]), 0.0, 0.0)
    ok = r0.status == R.OK and not np.any(r0.Omega[~(sup | np.eye(S.shape[0], dtype=bool))])
    return bool(ok and np.max(np.abs(r0.Omega - exact)) <= 1e-8)


def pin_refit_diagonal_support():
    """Eq. 3.8 on the diagonal support, at phi strictly between 0 and 1 and for
    a non-diagonal S: the infinite weights keep every off-diagonal entry 0, so
    row i reduces to -log w + 1/2 s_ii w^2 + phi lambda w, whose minimiser is
    w = (-phi lambda + sqrt((phi lambda)^2 + 4 s_ii)) / (2 s_ii)."""
    w = workload("ar1", p=40, n=30)
    X = w.X.astype(np.float64)
    s = np.diag(X.T @ X / X.shape[0])
    sup = np.zeros((40, 40), dtype=bool)
    ok = True
    for phi in (0.3, 0.5, 0.8):
        r = R.refit(X, w.lam, sup, phi, kkt_tol=1e-12, max_iter=20000)
        a = phi * w.lam
        want = (-a + np.sqrt(a * a + 4 * s)) / (2 * s)
        ok &= r.status == R.OK
        ok &= np.max(np.abs(r.Omega - np.diag(want))) <= 1e-10
    return bool(ok)


def pin_epbic_diagonal():
    """epBIC (Eq. 3.7) of the diagonal-S closed form: no off-diagonal nonzeros,
    so 2n(-sum log w_i + 1/2 sum s_i w_i^2)."""
    s = np.random.Generator(np.random.PCG64(41)).uniform(0.5, 2.0, size=7)
    n = 30
    X = orthogonal_design(n, s, 42)
    w = (-0.2 + np.sqrt(0.04 + 4 * s)) / (2 * s)
    want = 2 * n * (-np.sum(np.log(w)) + 0.5 * np.sum(s * w * w))
    return abs(R.epbic(np.diag(w), X, 0.7) - want) <= 1e-10 * abs(want)


def pin_epbic_edges():
    """The edge terms of Eq. 3.7 on an Omega with k off-diagonal nonzeros (a
    tridiagonal one, k = 2(p - 1)): gamma enters only through 4 gamma k log p,
    so two gammas differ by 4 (g1 - g0) k log p; and duplicating every row of
    X keeps S and doubles n, so with L the bracket of Eq. 3.7,
    E(X_dup) - 2 E(X) = k (log 2n - 2 log n) - 4 gamma k log p."""
    n, p = 25, 9
    X = _gauss(n, p, 41)
    Om = np.eye(p) * 1.3 + np.diag(np.full(p - 1, 0.2), 1) - np.diag(np.full(p - 1, 0.15), -1)
    k = 2 * (p - 1)
    g0, g1 = 0.0, 0.75
    ok = abs((R.epbic(Om, X, g1) - R.epbic(Om, X, g0)) - 4 * (g1 - g0) * k * np.log(p)) <= 1e-9
    Xd = np.vstack([X, X])
    want = k * (np.log(2 * n) - 2 * np.log(n)) - 4 * g1 * k * np.log(p)
    ok &= abs((R.epbic(Om, Xd, g1) - 2 * R.epbic(Om, X, g1)) - want) <= 1e-9
    return bool(ok)


def pin_kkt_min_norm_subgradient():
    """The KKT residual of Eq. 3.3 is the largest entry (in magnitude) of the
    minimum-norm element of the subdifferential of f, found here by search:
    off the diagonal the set is {G_ij + lambda z} with z = sign(omega_ij), or
    z in [-1, 1] (a fine grid) where omega_ij = 0; on the diagonal it is
    G_ii - 1/omega_ii + lambda_d. Each entry is checked alone: every other
    entry of G sits at a stationary value, so the residual is that entry's."""
    rng = np.random.Generator(np.random.PCG64(43))
    p, lam, lam_d = 6, 0.3, 0.25
    Om = rng.normal(size=(p, p)) * (rng.random((p, p)) < 0.5)
    np.fill_diagonal(Om, rng.uniform(0.5, 2.0, size=p))
    G0 = np.where(Om != 0, -lam * np.sign(Om), 0.0)
    np.fill_diagonal(G0, 1.0 / np.diag(Om) - lam_d)
    if R.kkt_residual(Om, G0, lam, lam_d) > 1e-12:
        return False
    z = np.linspace(-1.0, 1.0, 40001)
    kinds = set()
    for i in range(p):
        for j in range(p):
            g = rng.normal(scale=0.5)
            if i == j:
                want, kind = abs(g - 1.0 / Om[i, i] + lam_d), "diag"
            elif Om[i, j] != 0:
                want, kind = abs(g + lam * np.sign(Om[i, j])), "nonzero"
            else:
                want, kind = float(np.min(np.abs(g + lam * z))), "zero"
            kinds.add(kind)
            G = G0.copy()
            G[i, j] = g
            if abs(R.kkt_residual(Om, G, lam, lam_d) - want) > 1e-4 * lam:
                return False
    return kinds == {"diag", "nonzero", "zero"}


def pin_path_warm_start():
    """Warm starts along the lambda path reach the minimiser a cold start
    reaches (Thm 3.2: it is unique): on a bootstrap subsample, every path
    estimate equals the cold fit of X[rows] at that lambda, and every fit
    after the first starts from the previous penalty's estimate."""
    w = workload("er", p=30, n=40)
    rows = [np.random.Generator(np.random.PCG64(51)).integers(0, 40, size=35)]
    lams = [0.5, 0.3, 0.2, 0.12]
    pr = R.lambda_path(w.X, rows, lams, kkt_tol=1e-11, max_iter=20000)
    Xs = np.asarray(w.X, dtype=np.float64)[rows[0]]
    ok = True
    prev = np.eye(30)
    for k, lam in enumerate(lams):
        c = R.fit(Xs, lam, kkt_tol=1e-11, max_iter=20000)
        ok &= pr.fits[0][k].status == R.OK and np.max(np.abs(pr.fits[0][k].Omega - c.Omega)) <= 1e-8
        # warm start (Sec 3.4): the fit at lambda_k begins at the estimate of
        # lambda_{k-1} (I for the first), so its first objective value is f of
        # that estimate at the new penalty
        f0 = R.objective(prev, Xs, lam)
        ok &= abs(pr.fits[0][k].f[0] - f0) <= 1e-12 * abs(f0)
        prev = pr.fits[0][k].Omega
    return bool(ok)


def _diag_regime_lambda(S):
    """Smallest lambda on a doubling grid at which the diagonal closed form
    w_i = (-lambda + sqrt(lambda^2 + 4 s_ii)) / (2 s_ii) satisfies the
    off-diagonal KKT condition |w_i s_ij| <= lambda of Eq. 3.3."""
    s = np.diag(S)
    off = np.abs(S - np.diag(s))
    lam = 1e-3
    while True:
        w = (-lam + np.sqrt(lam * lam + 4 * s)) / (2 * s)
        if np.max(w[:, None] * off) <= lam:
            return lam, w
        lam *= 2.0


def pin_path_diagonal_regime():
    """Above that lambda the estimate of every subsample is diagonal with the
    closed form computed from the subsample's own S; epBIC then has no
    sparsity term, and the path picks the penalty with the smallest value of
    2n(-sum log w_i + 1/2 sum s_ii w_i^2).  That value grows with lambda, so
    the smallest penalty wins; it is solved first here, not last (penalties
    are solved in the order given)."""
    X = _gauss(25, 8, 52)
    rows = [np.arange(25), np.random.Generator(np.random.PCG64(53)).integers(0, 25, size=20)]
    ok = True
    want_scores = []
    lam_hi = 0.0
    for r in rows:
        Xs = X[r]
        lam_hi = max(lam_hi, _diag_regime_lambda(Xs.T @ Xs / len(r))[0])
    lams = [1.2 * lam_hi, 2.0 * lam_hi, 1.5 * lam_hi]
    pr = R.lambda_path(X, rows, lams, kkt_tol=1e-12, max_iter=20000)
    for s, r in enumerate(rows):
        Xs = X[r]
        S = Xs.T @ Xs / len(r)
        d = np.diag(S)
        sc = []
        for k, lam in enumerate(lams):
            w = (-lam + np.sqrt(lam * lam + 4 * d)) / (2 * d)
            ok &= np.max(np.abs(pr.fits[s][k].Omega - np.diag(w))) <= 1e-10
            sc.append(2 * len(r) * (-np.sum(np.log(w)) + 0.5 * np.sum(d * w * w)))
        ok &= pr.best[s] == int(np.argmin(sc)) == 0
        ok &= np.allclose(pr.epbic[:, s], sc, rtol=1e-10)
    return bool(ok)


def pin_smooth_loss_gradients():
    """dL/dOmega and dL/dX of the smooth loss equal central finite differences
    of the loss itself."""
    X = _gauss(9, 6, 71)
    O = np.eye(6) + 0.1 * _gauss(6, 6, 72)
    np.fill_diagonal(O, 1.0 + np.abs(np.diag(O)))
    GO, GX = R.smooth_loss_grad_omega(O, X), R.smooth_loss_grad_x(O, X)
    h, ok = 1e-6, True
    for (i, j) in [(0, 0), (1, 4), (5, 2), (3, 3)]:
        E = np.zeros_like(O)
        E[i, j] = h
        fd = (R.smooth_loss(O + E, X) - R.smooth_loss(O - E, X)) / (2 * h)
        ok &= abs(fd - GO[i, j]) <= 1e-6 * max(1.0, abs(fd))
    for (i, j) in [(0, 0), (8, 5), (4, 1)]:
        E = np.zeros_like(X)
        E[i, j] = h
        fd = (R.smooth_loss(O, X + E) - R.smooth_loss(O, X - E)) / (2 * h)
        ok &= abs(fd - GX[i, j]) <= 1e-6 * max(1.0, abs(fd))
    return bool(ok)


def _exact_fit(X, lam):
    S = np.asarray(X, dtype=np.float64).T @ np.asarray(X, dtype=np.float64) / X.shape[0]
    r = R.fit(X, lam, kkt_tol=1e-12, max_iter=100000)
    return R.polish(r.Omega, S, lam, lam)


def pin_implicit_dloglam_fd():
    """The implicit derivative of the held-out loss in log(lambda) equals the
    central finite difference (h = 1e-4) of the held-out loss at the exact
    minimisers for lambda e^(+-h), and dOmega-hat/dlog(lambda) equals the
    difference quotient of those minimisers (same active set on both sides)."""
    rng = np.random.Generator(np.random.PCG64(73))
    X = rng.standard_normal((60, 30))
    Xt, Xv = X[:40], X[40:]
    lam, h = 0.25, 1e-4
    O = _exact_fit(Xt, lam)
    Op, Om = _exact_fit(Xt, lam * math.exp(h)), _exact_fit(Xt, lam * math.exp(-h))
    if not (np.array_equal(O != 0, Op != 0) and np.array_equal(O != 0, Om != 0)):
        return False
    d, dO = R.implicit_dloglam(O, Xt, Xv, lam)
    fd = (R.smooth_loss(Op, Xv) - R.smooth_loss(Om, Xv)) / (2 * h)
    dfd = (Op - Om) / (2 * h)
    return bool(abs(d - fd) <= 1e-6 * max(1.0, abs(fd)) and np.max(np.abs(dO - dfd)) <= 1e-6 * max(1.0, np.max(np.abs(dfd))))


def pin_implicit_dloglam_diagonal():
    """Diagonal S (orthogonal training columns): Omega-hat(lambda) is diagonal
    with omega_i = (-lambda + sqrt(lambda^2 + 4 s_i)) / (2 s_i) (Eq. 3.3), so
    the held-out loss sum_i [-log omega_i + 1/2 omega_i^2 (S_val)_ii] has the
    derivative sum_i (-1/omega_i + omega_i (S_val)_ii) lambda d omega_i/d lambda,
    d omega_i/d lambda = (lambda / sqrt(lambda^2 + 4 s_i) - 1) / (2 s_i).  Without
    the diagonal penalty omega_i = 1/sqrt(s_i) does not move: both are 0.  The
    estimate is written from the closed form, not fitted."""
    rng = np.random.Generator(np.random.PCG64(81))
    s = rng.uniform(0.3, 3.0, size=9)
    Xt = orthogonal_design(40, s, 82)
    Xv = rng.standard_normal((25, 9)) * rng.uniform(0.5, 2.0, size=9)
    sv = np.diag(Xv.T @ Xv) / Xv.shape[0]
    ok = True
    for lam in (0.05, 0.4, 2.0):
        root = np.sqrt(lam * lam + 4 * s)
        w = (-lam + root) / (2 * s)
        dw = lam * (lam / root - 1.0) / (2 * s)          # d omega_i / d log(lambda)
        want = float(np.sum((-1.0 / w + w * sv) * dw))
        d, dO = R.implicit_dloglam(np.diag(w), Xt, Xv, lam)
        ok &= abs(d - want) <= 1e-10 * max(1.0, abs(want))
        ok &= np.max(np.abs(dO - np.diag(dw))) <= 1e-10 * np.max(np.abs(dw))
        d0, dO0 = R.implicit_dloglam(np.diag(1.0 / np.sqrt(s)), Xt, Xv, lam, penalize_diag=False)
        ok &= abs(d0) <= 1e-12 and np.max(np.abs(dO0)) <= 1e-12
    return bool(ok)


def pin_hessian_kronecker():
    """The Hessian of the smooth loss -log det Omega_D + 1/2 tr(Omega^T Omega S)
    in the column-major vectorisation of Omega is S (x) I_p + sum_i omega_ii^-2
    (e_i e_i^T (x) e_i e_i^T) (proof of Thm 4.1): it equals central differences
    of the oracle's gradient.  Entries of different rows do not couple, and row
    i's block is S + omega_ii^-2 e_i e_i^T, the matrix of the implicit solves."""
    rng = np.random.Generator(np.random.PCG64(91))
    n, p, h = 12, 5, 1e-5
    X = rng.standard_normal((n, p))
    S = X.T @ X / n
    O = 0.2 * rng.standard_normal((p, p))
    np.fill_diagonal(O, rng.uniform(0.6, 1.8, size=p))
    I = np.eye(p)
    H = np.kron(S, I) + sum(np.kron(np.outer(I[i], I[i]), np.outer(I[i], I[i])) / O[i, i] ** 2 for i in range(p))
    fd = np.zeros((p * p, p * p))
    for c in range(p * p):
        E = np.zeros(p * p)
        E[c] = h
        Ep = E.reshape(p, p, order="F")
        dg = R.smooth_loss_grad_omega(O + Ep, X) - R.smooth_loss_grad_omega(O - Ep, X)
        fd[:, c] = dg.ravel(order="F") / (2 * h)
    ok = np.max(np.abs(fd - H)) <= 1e-7 * np.max(np.abs(H))
    for i in range(p):
        for k in range(p):
            blk = H[np.ix_([i + p * j for j in range(p)], [k + p * j for j in range(p)])]
            want = S + np.outer(I[i], I[i]) / O[i, i] ** 2 if i == k else np.zeros((p, p))
            ok &= np.max(np.abs(blk - want)) <= 1e-12
    return bool(ok)


def pin_reparameterisation():
    """T(Theta) = Theta_D^-1/2 Theta (Thm 3.1) inverts to Theta = Omega_D Omega,
    and the partial correlations from Omega = T(Theta) equal the textbook
    -theta_ij / sqrt(theta_ii theta_jj) of the precision matrix."""
    rng = np.random.Generator(np.random.PCG64(81))
    B = rng.standard_normal((9, 9))
    Theta = B @ B.T + 9 * np.eye(9)
    Om = Theta / np.sqrt(np.diag(Theta))[:, None]
    d = np.sqrt(np.diag(Theta))
    rho = -Theta / np.outer(d, d)
    np.fill_diagonal(rho, 1.0)
    return bool(np.allclose(R.theta_hat(Om), Theta, rtol=1e-13, atol=1e-13) and
                np.allclose(R.partial_correlation(Om), rho, rtol=1e-13, atol=1e-13))


PINS = [pin_prox_root, pin_soft_threshold, pin_gradient, pin_lipschitz, pin_f_identity, pin_objective_diagonal,
        pin_diagonal_S, pin_diagonal_penalty_both_ways, pin_identity_S, pin_low_dim_closed_form, pin_brute_force,
        pin_kkt_descent_path, pin_linear_rate, pin_sufficient_decrease, pin_line_search_identity, pin_refit_fixed_point,
        pin_refit_restricted_mle, pin_refit_diagonal_support, pin_epbic_diagonal, pin_epbic_edges, pin_kkt_min_norm_subgradient,
        pin_path_warm_start, pin_path_diagonal_regime, pin_smooth_loss_gradients, pin_implicit_dloglam_fd,
        pin_implicit_dloglam_diagonal, pin_hessian_kronecker, pin_reparameterisation]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    assert pin()


def test_printed_and_difference_tests_agree_on_chain():
    """Away from rounding (early trials), the printed Alg. 1 test and the
    difference form give the same verdicts on the chain workload."""
    w = workload("ar1")
    r = R.fit(w.X, w.lam, kkt_tol=1e-6)
    assert r.status == R.OK
    assert all(r.printed_form_agrees[:100])


@pytest.mark.parametrize("kind,p,n,iters", [("scalefree", 1000, 300, 30), ("hubblock", 1000, 300, 30),
                                             ("scalefree", 5000, 1000, 3)])
def test_printed_and_difference_tests_agree_on_graph_workloads(kind, p, n, iters):
    """The two forms of Algorithm 1's sufficient-decrease test (the printed one,
    and the difference form ||Delta X^T||^2 / n <= ||Delta||^2 / tau that the
    kernels evaluate) reach the same verdict on every trial of the scale-free
    and hub-and-block workloads, the former also at its full size p = 5000,
    n = 1000 (first iterations)."""
    w = workload(kind, p=p, n=n)
    r = R.fit(w.X, w.lam, kkt_tol=1e-4, max_iter=iters)
    assert r.status in (R.OK, R.NOT_CONVERGED) and r.trials > r.iters
    assert all(r.printed_form_agrees)


def test_kkt_residual_definition_small():
    """r = 0 exactly at a brute-force minimiser's KKT point up to rounding, and
    positive when one entry is perturbed."""
    X = _gauss(10, 3, 27)
    S = X.T @ X / 10
    bf = R.brute_force(S, 0.3, 0.3)
    G = bf @ S
    assert R.kkt_residual(bf, G, 0.3, 0.3) <= 1e-12
    bad = bf.copy()
    bad[0, 1] += 1e-3
    assert R.kkt_residual(bad, bad @ S, 0.3, 0.3) > 1e-5


def test_row_offset_consistency():
    """Row-block helpers with row0 agree with the full-matrix versions (the
    objective separates over rows of Omega)."""
    w = workload("ar1", p=40, n=30)
    X = w.X.astype(np.float64)
    r = R.fit(X, w.lam, kkt_tol=1e-6)
    G = R.grad_g(r.Omega, X)
    A = r.Omega - 0.3 * G
    full = R.prox(A, 0.3, w.lam, w.lam)
    blk = R.prox(A[10:25], 0.3, w.lam, w.lam, row0=10)
    assert np.array_equal(full[10:25], blk)
    k_full = R.kkt_residual(r.Omega, G, w.lam, w.lam)
    k_blocks = max(R.kkt_residual(r.Omega[a:b], G[a:b], w.lam, w.lam, row0=a) for a, b in [(0, 13), (13, 40)])
    assert k_full == k_blocks


def test_bootstrap_sample_compresses_to_weighted_distinct_rows():
    """The objective sees the data only through S.  A bootstrap sample X[rows]
    (n_s rows, repeats allowed) and the matrix of its K distinct rows, row j
    scaled by sqrt(K c_j / n_s) with c_j its multiplicity, have the same S, so
    Algorithm 1 takes the same steps on both."""
    w = workload("ar1", p=40, n=30)
    X = np.asarray(w.X, dtype=np.float64)
    rows = np.random.Generator(np.random.PCG64(54)).integers(0, 30, size=45)
    uniq, cnt = np.unique(rows, return_counts=True)
    K = len(uniq)
    Xc = X[uniq] * np.sqrt(K * cnt / len(rows))[:, None]
    Xs = X[rows]
    np.testing.assert_allclose(Xc.T @ Xc / K, Xs.T @ Xs / len(rows), rtol=0, atol=1e-13)
    a = R.fit(Xs, w.lam, kkt_tol=1e-10, max_iter=5000)
    b = R.fit(Xc, w.lam, kkt_tol=1e-10, max_iter=5000)
    assert a.status == b.status == R.OK and a.ntrials == b.ntrials
    assert np.max(np.abs(a.Omega - b.Omega)) <= 1e-10


# ------------------------------------------------------ planted mistakes ---

MUTANTS = {
    "soft_threshold_sign": ("soft_threshold", lambda x, a: -np.sign(x) * np.maximum(np.abs(x) - a, 0.0)),
    "soft_threshold_shift": ("soft_threshold", lambda x, a: np.sign(x) * np.maximum(np.abs(x) - 2 * a, 0.0)),
    "diag_prox_drops_lambda": ("diag_prox", lambda y, tau, ld: 0.5 * (y + np.sqrt(y * y + 4 * tau))),
    "diag_prox_wrong_root": ("diag_prox", lambda y, tau, ld: 0.5 * ((y - tau * ld) + np.sqrt((y - tau * ld) ** 2 + 2 * tau))),
    "grad_transposed": ("grad_g", lambda Om, X: (np.asarray(X, float).T @ np.asarray(X, float) @ Om.T) / X.shape[0]),
    "grad_missing_1_over_n": ("grad_g", lambda Om, X: (Om @ np.asarray(X, float).T) @ np.asarray(X, float)),
    "g_missing_half": ("smooth_g", lambda Om, X: float(np.sum((Om @ np.asarray(X, float).T) ** 2)) / X.shape[0]),
    "lipschitz_trace": ("lipschitz", lambda X: float(np.trace(np.asarray(X, float) @ np.asarray(X, float).T)) / X.shape[0] / 3),
    "epbic_missing_2n": ("epbic", lambda Om, X, gm: -float(np.sum(np.log(np.diag(Om)))) + R.smooth_g(Om, X)),
    "grad_x_transposed": ("smooth_loss_grad_x", lambda Om, X: np.asarray(X, float) @ Om @ Om.T / X.shape[0]),
    "implicit_drops_log_term": ("implicit_dloglam", lambda O, Xt, Xv, lam, penalize_diag=True:
                                _implicit_without_log_term(O, Xt, Xv, lam)),
    "partial_corr_one_sided": ("partial_correlation", lambda Om: -Om / np.diag(Om)[None, :]),
    "path_ignores_subsample": ("lambda_path", lambda X, rows, lams, _f=R.lambda_path, **kw:
                               _f(X, [np.arange(np.asarray(X).shape[0])] * len(rows), lams, **kw)),
    "kkt_drops_diag_lambda": ("kkt_residual", lambda Om, G, lam, lam_d, row0=0, _f=R.kkt_residual:
                              _f(Om, G, lam, 0.0, row0=row0)),
    "refit_finite_off_support": ("refit", lambda X, lam, support, phi, penalize_diag=True, **kw:
                                 R.fit(X, np.where(np.asarray(support, bool) | np.eye(support.shape[0], dtype=bool),
                                                   phi * lam, lam),
                                       lam_diag=(phi * lam if penalize_diag else 0.0), **kw)),
    "epbic_counts_diagonal": ("epbic", lambda Om, X, gm, _f=R.epbic:
                              _f(Om, X, gm) + Om.shape[0] * (np.log(np.asarray(X).shape[0])
                                                             + 4 * gm * np.log(Om.shape[0]))),
    "prox_threshold_without_tau": ("prox", lambda A, tau, lam, lam_d, row0=0, _f=R.prox:
                                   _f(A, tau, np.asarray(lam) / tau, lam_d, row0=row0)),
    "trial_steps_uphill": ("fbs_trial", lambda Om, Y, G, X, tau, lam, lam_d, row0=0, _f=R.fbs_trial:
                           _f(Om, Y, -G, X, tau, lam, lam_d, row0=row0)),
    "path_cold_starts": ("lambda_path", lambda X, rows, lams, _f=R.lambda_path, **kw:
                         _f(X, rows, lams, **{**kw, "cold_every": 1})),
    "epbic_distinct_rows": ("epbic", lambda Om, X, gm, _f=R.epbic: _f(Om, np.unique(np.asarray(X), axis=0), gm)),
    "theta_hat_right_scaled": ("theta_hat", lambda Om: Om * np.diag(Om)[None, :]),
    "epbic_ignores_gamma": ("epbic", lambda Om, X, gm, _f=R.epbic: _f(Om, X, 0.0)),
    "implicit_sign_flipped": ("implicit_dloglam", lambda O, Xt, Xv, lam, penalize_diag=True, _f=R.implicit_dloglam:
                              tuple(-v for v in _f(O, Xt, Xv, lam, penalize_diag=penalize_diag))),
    "covariance_n_minus_1": ("sample_covariance", lambda X: np.asarray(X, float).T @ np.asarray(X, float)
                             / (np.asarray(X).shape[0] - 1)),
    "partial_corr_zero_diagonal": ("partial_correlation", lambda Om, _f=R.partial_correlation:
                                   _f(Om) - np.eye(Om.shape[0])),
    "path_selects_largest_epbic": ("lambda_path", lambda X, rows, lams, _f=R.lambda_path, **kw:
                                   _path_argmax(_f(X, rows, lams, **kw))),
    "kkt_nonzero_as_zero": ("kkt_residual", lambda Om, G, lam, lam_d, row0=0, _f=R.kkt_residual:
                            _f(np.zeros_like(Om) + np.where(np.eye(Om.shape[0], Om.shape[1], k=row0) > 0, Om, 0.0),
                               G, lam, lam_d, row0=row0)),
    "fit_always_penalizes_diagonal": ("fit", lambda X, lam, _f=R.fit, **kw: _f(X, lam, **{**kw, "penalize_diag": True})),
    "diag_prox_lambda_sign_flipped": ("diag_prox", lambda y, tau, lam_d, _f=R.diag_prox: _f(y, tau, -lam_d)),
    "smooth_grad_s_omega": ("smooth_loss_grad_omega", lambda Om, X: -np.diag(1.0 / np.diag(Om))
                            + R.sample_covariance(X) @ Om),
    "epbic_gamma_without_4": ("epbic", lambda Om, X, gm, _f=R.epbic: _f(Om, X, gm / 4.0)),
    "refit_phi_squared": ("refit", lambda X, lam, support, phi, _f=R.refit, **kw: _f(X, lam, support, phi * phi, **kw)),
    "theta_hat_sqrt_diagonal": ("theta_hat", lambda Om: np.sqrt(np.diag(Om))[:, None] * Om),
    "path_keeps_last_penalty": ("lambda_path", lambda X, rows, lams, _f=R.lambda_path, **kw:
                                _path_last(_f(X, rows, lams, **kw))),
    "objective_drops_logdet": ("objective", lambda Om, X, lam, penalize_diag=True, lam_diag=None, _f=R.objective:
                               _f(Om, X, lam, penalize_diag=penalize_diag, lam_diag=lam_diag)
                               + float(np.sum(np.log(R.diag_entries(Om))))),
}


def _path_last(pr):
    best = [len(pr.lambdas) - 1] * pr.epbic.shape[1]
    return R.PathResult(pr.lambdas, pr.fits, pr.epbic, best, [pr.fits[s][b].Omega for s, b in enumerate(best)])


def _path_argmax(pr):
    best = [int(np.argmax(pr.epbic[:, s])) for s in range(pr.epbic.shape[1])]
    return R.PathResult(pr.lambdas, pr.fits, pr.epbic, best, [pr.fits[s][b].Omega for s, b in enumerate(best)])


def _implicit_without_log_term(O, Xt, Xv, lam):
    S = R.sample_covariance(Xt)
    Gv = R.smooth_loss_grad_omega(O, Xv)
    dO = np.zeros_like(O)
    for i in range(O.shape[0]):
        A = np.nonzero(O[i] != 0)[0]
        v = np.sign(O[i, A])
        dO[i, A] = -lam * np.linalg.solve(S[np.ix_(A, A)], v)
    return float(np.sum(Gv * dO)), dO


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(monkeypatch, mutant):
    attr, fn = MUTANTS[mutant]
    monkeypatch.setattr(R, attr, fn)
    for pin in PINS:  # stops at the first pin that catches it
        try:
            if not pin():
                return
        except TypeError:
            raise  # a mutant whose signature does not match is a broken test, not a catch
        except Exception:
            return
    pytest.fail(f"mutant {mutant} passed every pin")


def test_oracle_statuses():
    """The oracle's exits, with the meaning the C header gives them: the
    line search exhausted (the last accepted iterate is returned), non-finite
    data, and max_iter accepted steps."""
    w = workload("ar1", p=30, n=20)
    X = w.X.astype(np.float64)
    L = R.lipschitz(X)
    # tau0 far above 1/L and too few reductions to reach it: no step is accepted
    r = R.fit(X, w.lam, tau0=1e6, max_backtracks=2)
    assert 1e6 * 0.25 > 1.0 / L
    assert r.status == R.EBACKTRACK and r.iters == 0 and r.trials == 3
    assert np.array_equal(r.Omega, np.eye(30))
    # enough reductions: the same start converges
    assert R.fit(X, w.lam, tau0=1e6, max_backtracks=60, kkt_tol=1e-6).status == R.OK
    Xn = X.copy()
    Xn[3, 4] = np.nan
    with pytest.raises(np.linalg.LinAlgError):    # the eigensolver for L refuses NaN data
        R.fit(Xn, w.lam)
    assert R.fit(Xn, w.lam, L=L).status == R.ENONFINITE  # with L given, the iteration's own check
    r = R.fit(X, w.lam, max_iter=2, kkt_tol=0.0)
    assert r.status == R.NOT_CONVERGED and r.iters == 2 and len(r.f) == 3
