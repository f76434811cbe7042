"""The support comparison used by the parity tests, on hand-made cases: a
flip of an entry far from the soft-threshold is reported, a flip inside the
band is excused, and the two slack forms (zero entries: lambda - |G_ij|;
nonzero entries: |omega_ij| S_jj) are the ones the rules state."""
import numpy as np

from support_rules import fp64_support_ok, offdiag_slack, unexplained_mismatches


def _case():
    ref = np.array([[1.0, 0.0, 0.3, 0.0],
                    [0.0, 1.0, 0.0, 2e-9],
                    [0.3, 0.0, 1.0, 0.0],
                    [0.0, 0.0, 0.0, 1.0]])
    lam = 0.2
    G = np.full((4, 4), 0.05)        # zero entries: slack 0.15
    G[0, 1] = 0.2 - 5e-9             # a zero entry at the threshold
    G[0, 2] = -lam                   # nonzero entries satisfy G = -lam sign(omega)
    G[2, 0] = -lam
    G[1, 3] = -lam
    s_diag = np.array([1.0, 2.0, 4.0, 0.5])
    return ref, G, lam, s_diag


def test_identical_patterns_pass():
    ref, G, lam, s = _case()
    assert fp64_support_ok(ref.copy(), ref, G, lam)
    bad, nmis, _ = unexplained_mismatches(ref.copy(), ref, G, lam, grad_band=1e-3, s_diag=s)
    assert nmis == 0 and not bad.any()


def test_fp64_band_excuses_only_borderline_entries():
    ref, G, lam, _ = _case()
    est = ref.copy()
    est[0, 1] = 1e-6     # zero in ref, lam - |G| = 5e-9: borderline
    est[1, 3] = 0.0      # |ref| = 2e-9: borderline
    assert fp64_support_ok(est, ref, G, lam)
    est[3, 2] = 1e-6     # zero in ref with slack 0.15: a real mismatch
    assert not fp64_support_ok(est, ref, G, lam)
    est = ref.copy()
    est[0, 2] = 0.0      # |ref| = 0.3: a real mismatch (nonzero entries are not excused by G)
    assert not fp64_support_ok(est, ref, G, lam)


def test_mixed_band_in_gradient_units():
    ref, G, lam, s = _case()
    slack = offdiag_slack(ref, G, lam, s)
    assert np.isinf(np.diag(slack)).all()
    assert np.isclose(slack[0, 2], 0.3 * 4.0) and np.isclose(slack[3, 2], 0.15)
    assert np.isclose(slack[1, 3], 2e-9 * 0.5) and np.isclose(slack[0, 1], 5e-9)
    est = ref.copy()
    est[3, 2] = 1e-6
    bad, nmis, slacks = unexplained_mismatches(est, ref, G, lam, grad_band=0.1, s_diag=s)
    assert nmis == 1 and bad[3, 2] and np.allclose(slacks, [0.15])
    bad, _, _ = unexplained_mismatches(est, ref, G, lam, grad_band=0.16, s_diag=s)
    assert not bad.any()
    est = ref.copy()
    est[0, 2] = 0.0      # slack 1.2 in gradient units
    bad, _, _ = unexplained_mismatches(est, ref, G, lam, grad_band=1.0, s_diag=s)
    assert bad[0, 2]
    bad, _, _ = unexplained_mismatches(est, ref, G, lam, grad_band=1.3, s_diag=s)
    assert not bad.any()
