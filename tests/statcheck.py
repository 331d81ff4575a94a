"""Acceptance statistics shared by the oracle pins and the GPU parity tests.

Per point, z = (mean - u_exact) / SE.  The epsilon-shell introduces a bias of
at most eps * max|grad u| (the walk returns g at a boundary point closer than
eps), which is allowed for.  Over n points this is a multiple-comparisons
test: the fraction of points with |z| > 4 may not exceed 1e-4 plus the 99.9%
binomial margin, and mean(z^2) must lie in a band around 1.
"""
import numpy as np
from scipy import stats


def z_scores(err, se, allow):
    """z after removing the shell-bias allowance (never increases |err|)."""
    shrunk = np.sign(err) * np.maximum(np.abs(err) - allow, 0.0)
    return shrunk / np.maximum(se, 1e-300)


def check_z(err, se, allow, zthr=4.0, band=(0.5, 1.8), label="", dof=None):
    """dof: degrees of freedom of the per-point SE (walks - 1) when few
    walks are used; z then follows Student's t and the exceedance rate is
    that of t (doubled for the heavy tails of the walk estimates)."""
    err = np.asarray(err, float)
    se = np.asarray(se, float)
    z = z_scores(err, se, allow)
    n = len(z)
    nbad = int(np.count_nonzero(np.abs(z) > zthr))
    p = 1e-4 if dof is None else max(1e-4, 4.0 * stats.t.sf(zthr, dof))
    limit = int(stats.binom.ppf(0.999, n, p))
    assert nbad <= limit, f"{label}: {nbad} of {n} points beyond {zthr} SE (limit {limit}); worst {np.max(np.abs(z)):.2f}"
    hard = 8.0 if dof is None else 30.0  # few walks: Student-t tails
    assert np.all(np.abs(z) < hard), f"{label}: a point is {np.max(np.abs(z)):.2f} SE away"
    keep = se > 2 * allow  # points whose error is not dominated by the shell bias
    if band is not None and keep.sum() >= 16:
        m = float(np.mean((err[keep] / se[keep]) ** 2))
        assert band[0] < m < band[1], f"{label}: mean z^2 = {m:.3f}"
    return z
