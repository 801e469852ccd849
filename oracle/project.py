"""Continuum projection eta, Eq. (2.7) (Section 2.2).

For pixels i, k of the same forest

    eta_ik = delta^K_ik - w_k / sum_l w_l
             - (Lambda_i - Lbar) w_k (Lambda_k - Lbar) / sum_l w_l (Lambda_l - Lbar)^2

with Lambda = log lambda; eta vanishes across forests.

Readings:

* Lbar is the weighted mean sum w Lambda / sum w.  With it eta is an exact
  projector (eta^2 = eta); the paper does not define Lbar;
* a forest with sum_l w_l (Lambda_l - Lbar)^2 = 0 (one pixel, or all weight on
  one wavelength) drops the slope term;
* a forest with sum_l w_l = 0 drops both terms (eta = identity);
* the same weights w enter eta and the estimator;
* the log base is irrelevant: eta is invariant under Lambda -> a Lambda + b.

``project`` applies eta to delta forest by forest (delta' = eta delta).
"""
from __future__ import annotations

import numpy as np


def forest_moments(w: np.ndarray, loglam: np.ndarray):
    """(W, Lbar, S, x) of one forest: W = sum w, Lbar = sum w L / W,
    x = L - Lbar, S = sum w x^2."""
    w = np.asarray(w, dtype=np.float64)
    L = np.asarray(loglam, dtype=np.float64)
    W = float(np.sum(w))
    Lbar = float(np.sum(w * L) / W) if W > 0 else 0.0
    x = L - Lbar
    S = float(np.sum(w * x * x)) if W > 0 else 0.0
    return W, Lbar, S, x


def eta_matrix(w: np.ndarray, loglam: np.ndarray) -> np.ndarray:
    """The n x n matrix eta of one forest, written term by term from Eq. (2.7)."""
    w = np.asarray(w, dtype=np.float64)
    n = w.shape[0]
    W, _, S, x = forest_moments(w, loglam)
    eta = np.eye(n)
    if W > 0:
        eta -= np.ones((n, 1)) * (w / W)[None, :]
        if S > 0:
            eta -= x[:, None] * (w * x)[None, :] / S
    return eta


def project(cat, delta=None) -> np.ndarray:
    """delta' = eta delta for every forest (float64 result)."""
    d = np.asarray(cat.delta if delta is None else delta, dtype=np.float64)
    out = np.empty_like(d)
    for f in range(cat.n_forests):
        sl = cat.forest(f)
        if sl.stop == sl.start:
            continue
        w = cat.weight[sl].astype(np.float64)
        W, _, S, x = forest_moments(w, cat.loglam[sl])
        df = d[sl]
        res = df.copy()
        if W > 0:
            res -= np.sum(w * df) / W
            if S > 0:
                res -= x * (np.sum(w * x * df) / S)
        out[sl] = res
    return out
