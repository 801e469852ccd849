"""Same-forest (one-dimensional) correlation.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. (2.4) excludes pixel pairs of the same forest (Section 2.1); the paper
names the one-dimensional correlations as future work of its pipeline
(Section 4).  Readings:

* estimator: Eq. (2.4) over the excluded pairs,
      xi1d_p = sum_{i<j, same forest, in bin p} (w d)_i (w d)_j / sum w_i w_j;
* separation: the line-of-sight distance |d_i - d_j| (the bisector split of
  Section 2.1 at theta = 0, where r_perp = 0);
* bins: n half-open bins of width r_max / n over [0, r_max),
  p = floor(|d_i - d_j| / (r_max / n));
* each unordered pair of distinct pixels counts once (no zero lag).
"""
from __future__ import annotations

import numpy as np


def xi1d_sums(cat, n_bins: int, r_max: float, delta=None):
    """N_p, W_p, xi_p, pair counts and the noise floor sigma_p."""
    delta = np.asarray(cat.delta if delta is None else delta)
    dr = r_max / n_bins
    num, wsum, cnt, sq = np.zeros(n_bins), np.zeros(n_bins), np.zeros(n_bins), np.zeros(n_bins)
    for f in range(cat.n_forests):
        sl = cat.forest(f)
        n = sl.stop - sl.start
        if n < 2:
            continue
        d = np.asarray(cat.dist[sl], dtype=np.float64)
        w = cat.weight[sl].astype(np.float64)
        wd = w * delta[sl].astype(np.float64)
        i, j = np.triu_indices(n, k=1)
        p = np.floor(np.abs(d[j] - d[i]) / dr)
        ok = p < n_bins
        P = p[ok].astype(np.int64)
        tn = wd[i[ok]] * wd[j[ok]]
        num += np.bincount(P, weights=tn, minlength=n_bins)
        wsum += np.bincount(P, weights=w[i[ok]] * w[j[ok]], minlength=n_bins)
        cnt += np.bincount(P, minlength=n_bins)
        sq += np.bincount(P, weights=tn * tn, minlength=n_bins)
    xi = np.divide(num, wsum, out=np.zeros_like(wsum), where=wsum != 0)
    sigma = np.divide(np.sqrt(sq), wsum, out=np.zeros_like(wsum), where=wsum != 0)
    return {"num": num, "wsum": wsum, "xi": xi, "count": cnt, "num_sq": sq, "sigma": sigma}
