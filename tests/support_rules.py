"""Support comparison for the parity tests.

The minimiser of Eq. 3.2 is unique (Thm 3.2), so its zero pattern is well
defined.  Two computations of it can still disagree on an entry that sits at
the threshold of the soft-threshold in Eq. 3.5: a zero entry whose gradient
is within rounding of the penalty, or a nonzero entry within rounding of 0.
These helpers count the disagreements that such entries do not explain.

Borderline entries, given the reference estimate ref and its gradient
G_ref = ref S (off the diagonal, penalty lam):
  ref_ij == 0:  slack lam - |G_ij|, the change of G_ij that activates it;
  ref_ij != 0:  |ref_ij|, or in gradient units |ref_ij| S_jj (the curvature
                of row i's objective along coordinate j is S_jj, so a change
                of G_ij by that much moves the entry to 0).
FP64 results use the fixed band of the method's FP64 target (1e-8 on both
forms).  Mixed-precision results use a band in gradient units: ten times the
measured gradient error of the mixed product, which is what moves an entry
of the mixed fixed point across the threshold, plus the KKT residuals at
which the two fits stopped, since an iterate stopped at residual r can still
hold an entry within r of its final side of the threshold.
"""
import numpy as np


def offdiag_slack(ref, G_ref, lam, s_diag):
    """Per-entry slack in gradient units (diagonal entries: +inf)."""
    nz = ref != 0
    slack = np.where(nz, np.abs(ref) * np.asarray(s_diag)[None, :], lam - np.abs(G_ref))
    np.fill_diagonal(slack, np.inf)
    return slack


def unexplained_mismatches(est, ref, G_ref, lam, *, omega_band=0.0, grad_band=0.0, s_diag=None):
    """Off-diagonal entries whose zero pattern differs between est and ref and
    that no band excuses.  Returns (mask of unexplained entries, number of all
    mismatches, slacks of all mismatches in gradient units or None)."""
    p = ref.shape[0]
    off = ~np.eye(p, dtype=bool)
    diff = ((est != 0) != (ref != 0)) & off
    nz = ref != 0
    excused = (~nz & (lam - np.abs(G_ref) <= grad_band)) | (nz & (np.abs(ref) <= omega_band))
    slacks = None
    if s_diag is not None:
        slack = offdiag_slack(ref, G_ref, lam, s_diag)
        excused |= slack <= grad_band
        slacks = slack[diff]
    return diff & ~excused, int(np.sum(diff)), slacks


def fp64_support_ok(est, ref, G_ref, lam, band=1e-8):
    """The FP64 rule: identical zero pattern except entries with
    |ref_ij| <= band or lam - |G_ij| <= band."""
    bad, _, _ = unexplained_mismatches(est, ref, G_ref, lam, omega_band=band, grad_band=band)
    return int(np.sum(bad)) == 0
