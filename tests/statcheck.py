"""Acceptance statistics shared by the oracle pins and the GPU parity tests.

Per point, z = (mean - u_exact) / SE, SE the standard error from the sample
variance of the point's W walk estimates.  The epsilon-shell introduces a
bias of at most eps * max|grad u| (the walk returns g at a boundary point
closer than eps), which is allowed for.  Over n points this is a
multiple-comparisons test: the fraction of points with |z| > 4 may not
exceed 1e-4 plus the 99.9% binomial margin, and mean(z^2) must lie in its
99.9% band.

The band of mean(z^2).  For normal walk estimates z^2 is chi^2 with one
degree of freedom, and n * mean(z^2) is chi^2_n: the band is its 0.05% and
99.95% quantiles over n.  The walk estimates are heavy-tailed (the 1/pdf of
the Neumann term, Sec. 4.5), which makes the sample variance noisy: with
s^2 / sigma^2 = 1 + delta, Var(delta) = (kappa - 1) / W for per-walk
kurtosis kappa (the fourth standardised moment), and to second order in
delta, E[z^2] = 1 + (kappa - 1) / W and Var(z^2) = 2 + 3 (kappa - 1) / W.
When the per-point kurtosis is given (measured from per-walk estimates),
the band is centred on the mean of the first and its half width is 3.29
(two-sided 99.9%) times sqrt(mean of the second / n).  Points whose SE is
below 8 times the shell allowance are left out of the band (there the bias
could move z^2 by more than 1/64); the bias of the kept points widens the
upper limit by mean((allow / SE)^2).
"""
import numpy as np
from scipy import stats


def z_scores(err, se, allow):
    """z after removing the shell-bias allowance (never increases |err|)."""
    shrunk = np.sign(err) * np.maximum(np.abs(err) - allow, 0.0)
    return shrunk / np.maximum(se, 1e-300)


def kurtosis(per_walk):
    """Per-point kurtosis (fourth standardised moment) of per-walk estimates
    [n, W]; 3 where a point's estimates do not vary."""
    x = np.asarray(per_walk, float)
    d = x - x.mean(1, keepdims=True)
    m2 = np.mean(d**2, 1)
    m4 = np.mean(d**4, 1)
    return np.where(m2 > 0, m4 / np.maximum(m2, 1e-300) ** 2, 3.0)


def z2_band(n, walks=None, kurt=None):
    """99.9% band of mean(z^2) over n points (see the module docstring)."""
    if kurt is None:
        return stats.chi2.ppf(0.0005, n) / n, stats.chi2.ppf(0.9995, n) / n
    k = np.asarray(kurt, float)
    c = 1.0 + np.mean((k - 1.0) / walks)
    v = np.mean(2.0 + 3.0 * (k - 1.0) / walks)
    lo, hi = stats.chi2.ppf(0.0005, n) / n, stats.chi2.ppf(0.9995, n) / n
    w = 3.29 * np.sqrt(v / n)
    return min(lo, c - w), max(hi, c + w)


def check_z(err, se, allow, zthr=4.0, band=True, label="", walks=None, kurt=None):
    """Exceedance of |z| > zthr within the binomial 99.9% limit, no point
    beyond 8 SE, and (band) mean z^2 within its 99.9% band; kurt: per-point
    kurtosis of the walk estimates (same order as err) with walks per point."""
    err = np.asarray(err, float)
    se = np.asarray(se, float)
    z = z_scores(err, se, allow)
    n = len(z)
    nbad = int(np.count_nonzero(np.abs(z) > zthr))
    limit = int(stats.binom.ppf(0.999, n, 1e-4))
    assert nbad <= limit, f"{label}: {nbad} of {n} points beyond {zthr} SE (limit {limit}); worst {np.max(np.abs(z)):.2f}"
    assert np.all(np.abs(z) < 8.0), f"{label}: a point is {np.max(np.abs(z)):.2f} SE away"
    keep = se > 8 * allow
    if band and keep.sum() >= 16:
        m = float(np.mean((err[keep] / se[keep]) ** 2))
        lo, hi = z2_band(int(keep.sum()), walks, None if kurt is None else np.asarray(kurt)[keep])
        hi += float(np.mean((allow / se[keep]) ** 2))
        assert lo < m < hi, f"{label}: mean z^2 = {m:.3f} outside its 99.9% band ({lo:.3f}, {hi:.3f}), n = {keep.sum()}"
    return z
