"""Pins of the oracle's per-bin means (r_par, r_perp, pair distance) and
pixel-pair counts: hand arithmetic, the bin edges, agreement with the
estimator's W and counts, and an analytic uniform grid."""
import math

import numpy as np
import pytest

from conftest import line_catalog
from oracle import xi as oxi
from paper_2507_00129_gb300 import synth


def test_bin_means_hand_built():
    """Two forests on nearly the same line of sight (theta = 2 asin(1e-4)):
    forest a at 1000, 1003; forest b at 1001, 1010.  Bins of 4 (r_par) x 4 (r_perp):
    pairs (1000,1001) r_par = 1 c, (1003,1001) 2 c -> bin (0,0); (1000,1010) 10 c -> (2,0);
    (1003,1010) 7 c -> (1,0), c = cos(theta/2).  Weights 1, 2 (a) and 3, 5 (b)."""
    th = 2 * math.asin(1e-4)
    cat = line_catalog([(0.0, math.pi / 2, [1000.0, 1003.0], [8.0, 8.1], [0.1, 0.2], [1.0, 2.0]),
                        (0.0, math.pi / 2 - th, [1001.0, 1010.0], [8.0, 8.1], [0.3, 0.4], [3.0, 5.0])])
    bins = synth.Bins(4, 4, 16.0, 16.0)
    out = oxi.bin_means(cat, bins, (np.array([0]), np.array([1])))
    c = math.sqrt(1 - 1e-8)
    A0, A1, A2 = 0, 4, 8
    assert out["count"][A0] == 2 and out["count"][A1] == 1 and out["count"][A2] == 1
    assert out["wsum"][A0] == pytest.approx(1 * 3 + 2 * 3)
    assert out["rpar_mean"][A0] == pytest.approx((3 * 1 * c + 6 * 2 * c) / 9, rel=1e-12)
    assert out["rpar_mean"][A1] == pytest.approx(7 * c, rel=1e-12)
    assert out["dist_mean"][A0] == pytest.approx((3 * 1000.5 + 6 * 1002.0) / 9, rel=1e-14)
    assert out["rperp_mean"][A2] == pytest.approx(2010 * 1e-4, rel=1e-9)


def test_bin_means_lie_in_their_bins_and_match_xi():
    cat = synth.make(0)
    bins = synth.bins_for(0)
    from oracle import pairs as opairs
    pl = opairs.forest_pairs(cat, bins)
    sub = (pl[0][::40], pl[1][::40])
    out = oxi.bin_means(cat, bins, sub)
    ref = oxi.xi_sums(cat, bins, sub)
    np.testing.assert_allclose(out["wsum"], ref["wsum"], rtol=1e-14)
    np.testing.assert_array_equal(out["count"], ref["count"])
    on = out["wsum"] > 0
    p, t = np.divmod(np.arange(bins.nbins), bins.n_perp)
    dp, dt = bins.r_par_max / bins.n_par, bins.r_perp_max / bins.n_perp
    assert np.all(out["rpar_mean"][on] >= p[on] * dp) and np.all(out["rpar_mean"][on] < (p[on] + 1) * dp)
    assert np.all(out["rperp_mean"][on] >= t[on] * dt) and np.all(out["rperp_mean"][on] < (t[on] + 1) * dt)
    assert np.all((out["dist_mean"][on] > 3000) & (out["dist_mean"][on] < 5000))


def test_bin_means_analytic_uniform_grid():
    """Two copies of a uniform forest (d_k = d0 + 0.73 k, w = 1) at a tiny angle:
    the mean r_par of bin p is the mean of |k - l| h c over the lags in p,
    weighted by their multiplicities 2 (n - m) (n for m = 0)."""
    n, h, th = 40, 0.73, 2 * math.asin(1e-6)
    d = 1000.0 + h * np.arange(n)
    cat = line_catalog([(0.0, math.pi / 2, d, np.linspace(8, 8.1, n), np.zeros(n), np.ones(n)),
                        (0.0, math.pi / 2 - th, d, np.linspace(8, 8.1, n), np.zeros(n), np.ones(n))])
    bins = synth.Bins(6, 2, 24.0, 8.0)
    out = oxi.bin_means(cat, bins, (np.array([0]), np.array([1])))
    c = math.sqrt(1 - 1e-12)
    for p in range(6):
        ms = [m for m in range(n) if math.floor(m * h * c / 4.0) == p]
        mult = [n if m == 0 else 2 * (n - m) for m in ms]
        exp = sum(k * m * h * c for k, m in zip(mult, ms)) / sum(mult)
        assert out["rpar_mean"][p * 2] == pytest.approx(exp, rel=1e-12)
        assert out["count"][p * 2] == sum(mult)


def test_bin_means_edge_counts_bound_rebinning():
    """Rescaling all distances by a factor that moves separations by less than
    eps bin widths changes a bin's count by at most edge_c and its W by at
    most edge_w."""
    from conftest import random_small
    cat = random_small(n_forests=8, max_len=8, patch_deg=0.6, seed=61, spread=30.0)
    bins = synth.Bins(6, 4, 24.0, 24.0)
    from oracle import pairs as opairs
    pl = opairs.all_pairs(cat.n_forests)
    eps = 0.02
    ref = oxi.bin_means(cat, bins, pl, eps_edge=eps)
    changed = False
    # every separation scales by f: |f - 1| r <= 3e-3 x 24 Mpc/h = 0.072 Mpc/h, below eps = 0.02 bin widths
    # (0.08 Mpc/h for r_par, 0.12 for r_perp)
    for f in (1 + 3e-3, 1 - 3e-3):
        moved = synth.Catalog(ra=cat.ra, dec=cat.dec, offsets=cat.offsets, dist=cat.dist * f,
                              loglam=cat.loglam, delta=cat.delta, weight=cat.weight)
        alt = oxi.bin_means(moved, bins, pl)
        assert np.all(np.abs(alt["count"] - ref["count"]) <= ref["edge_c"])
        assert np.all(np.abs(alt["wsum"] - ref["wsum"]) <= ref["edge_w"] + 1e-12)
        changed |= bool(np.any(alt["count"] != ref["count"]))
    assert ref["count"].sum() > 50
    assert changed or ref["edge_c"].sum() == 0


def test_bin_mean_redshift_hand_built_and_linear_identity():
    """Mean redshift of a bin: (a) the hand-built pairs of the first test with
    pixel redshifts 2.0, 2.1 (a) and 2.2, 2.3 (b): bin (0, 0) holds (i0, j0) and
    (i1, j0) with weights 3 and 6, so z = (3 (2.0 + 2.2) / 2 + 6 (2.1 + 2.2) / 2) / 9;
    (b) a pixel redshift linear in distance, z = alpha + beta d, gives exactly
    alpha + beta dist_mean in every bin; (c) a constant z gives that constant."""
    th = 2 * math.asin(1e-4)
    cat = line_catalog([(0.0, math.pi / 2, [1000.0, 1003.0], [8.0, 8.1], [0.1, 0.2], [1.0, 2.0]),
                        (0.0, math.pi / 2 - th, [1001.0, 1010.0], [8.0, 8.1], [0.3, 0.4], [3.0, 5.0])])
    bins = synth.Bins(4, 4, 16.0, 16.0)
    z = np.array([2.0, 2.1, 2.2, 2.3])
    out = oxi.bin_means(cat, bins, (np.array([0]), np.array([1])), z=z)
    assert out["z_mean"][0] == pytest.approx((3 * 2.1 + 6 * 2.15) / 9, rel=1e-14)
    assert out["z_mean"][4] == pytest.approx((2.1 + 2.3) / 2, rel=1e-14)
    big = synth.make(0)
    bb = synth.bins_for(0)
    from oracle import pairs as opairs
    pl = opairs.forest_pairs(big, bb)
    sub = (pl[0][::60], pl[1][::60])
    lin = oxi.bin_means(big, bb, sub, z=1.7 + 2.5e-4 * big.dist)
    on = lin["wsum"] > 0
    np.testing.assert_allclose(lin["z_mean"][on], 1.7 + 2.5e-4 * lin["dist_mean"][on], rtol=1e-13)
    const = oxi.bin_means(big, bb, sub, z=np.full(big.n_pix, 2.4))
    np.testing.assert_allclose(const["z_mean"][on], 2.4, rtol=1e-14)
    assert np.all(const["z_mean"][~on] == 0)
