"""Pins of the projection eta (Eq. 2.7) and of the distortion matrix (Eq. 2.6):
hand arithmetic, invariants that follow from eta being a projector, and the
literal quadruple sum against the expanded form."""
import math

import numpy as np
import pytest

from oracle import project as oproj, dmat as odm, pairs, xi as oxi
from paper_2507_00129_gb300 import synth
from conftest import line_catalog, random_small


# ---------------------------------------------------------------- projection
def test_projection_hand_example():
    # w = (1,2,1), Lambda = (0,1,2): W = 4, Lbar = 1, x = (-1,0,1), S = 2.
    # delta = (1,0,0): sum w delta / W = 1/4, sum w x delta / S = -1/2
    # delta' = delta - 1/4 + x/2 = (1/4, -1/4, 1/4)
    cat = line_catalog([(0.0, 0.0, [1.0, 2.0, 3.0], [0.0, 1.0, 2.0], [1.0, 0.0, 0.0], [1.0, 2.0, 1.0])])
    np.testing.assert_allclose(oproj.project(cat), [0.25, -0.25, 0.25], atol=1e-15)


def test_projection_removes_weighted_mean_and_slope(cat0):
    dp = oproj.project(cat0)
    for f in range(0, cat0.n_forests, 7):
        sl = cat0.forest(f)
        w = cat0.weight[sl].astype(float)
        W, _, S, x = oproj.forest_moments(w, cat0.loglam[sl])
        assert abs(np.sum(w * dp[sl])) <= 1e-12 * np.sum(np.abs(w * cat0.delta[sl]))
        assert abs(np.sum(w * x * dp[sl])) <= 1e-12 * np.sum(np.abs(w * x * cat0.delta[sl])) + 1e-15


def test_projection_kills_linear_in_lambda(cat0):
    rng = np.random.default_rng(2)
    a = rng.normal(size=cat0.n_forests)
    b = rng.normal(size=cat0.n_forests)
    f_of = np.repeat(np.arange(cat0.n_forests), cat0.lengths())
    d = a[f_of] + b[f_of] * cat0.loglam
    dp = oproj.project(cat0, d)
    assert np.max(np.abs(dp)) < 1e-9


def test_projection_idempotent_and_base_invariant(cat0):
    dp = oproj.project(cat0)
    np.testing.assert_allclose(oproj.project(cat0, dp), dp, atol=1e-13)
    c10 = synth.Catalog(**{**cat0.__dict__, "loglam": cat0.loglam / math.log(10) + 3.0})
    np.testing.assert_allclose(oproj.project(c10), dp, atol=1e-11)


def test_eta_matrix_is_projector_and_matches_project():
    rng = np.random.default_rng(4)
    w = rng.uniform(0.2, 3, 9)
    L = np.sort(rng.uniform(8.1, 8.4, 9))
    eta = oproj.eta_matrix(w, L)
    np.testing.assert_allclose(eta @ eta, eta, atol=1e-12)
    d = rng.normal(size=9)
    cat = line_catalog([(0.0, 0.0, np.arange(9.0), L, d, w)])
    np.testing.assert_allclose(eta @ d.astype(np.float32).astype(float), oproj.project(cat), atol=1e-12)
    assert np.allclose(eta @ np.ones(9), 0, atol=1e-12)


def test_projection_degenerate_forests():
    # one pixel: S = 0 drops the slope, the mean removes everything
    one = line_catalog([(0.0, 0.0, [1.0], [8.2], [0.7], [2.0])])
    np.testing.assert_allclose(oproj.project(one), [0.0], atol=1e-15)
    # zero weight: nothing to remove
    zw = line_catalog([(0.0, 0.0, [1.0, 2.0], [8.2, 8.3], [0.7, -0.1], [0.0, 0.0])])
    np.testing.assert_allclose(oproj.project(zw), [0.7, -0.1], atol=1e-7)
    # two pixels at distinct Lambda: mean and slope fit them exactly
    two = line_catalog([(0.0, 0.0, [1.0, 2.0], [8.2, 8.3], [0.7, -0.1], [1.0, 3.0])])
    np.testing.assert_allclose(oproj.project(two), [0.0, 0.0], atol=1e-14)


# ---------------------------------------------------------------- distortion
def _hand_dm_catalog():
    # Forests a, b on one line of sight, 2 pixels each, unit weights, constant
    # Lambda inside each forest (S = 0, slope dropped): eta = I - 11^T/2.
    a = (0.0, 0.0, [100.0, 120.0], [0.0, 0.0], [0.0, 0.0], [1.0, 1.0])
    b = (0.0, 0.0, [101.0, 121.0], [0.0, 0.0], [0.0, 0.0], [1.0, 1.0])
    return line_catalog([a, b]), synth.Bins(10, 1, 40.0, 4.0)


def test_dmat_hand_example():
    """Pixel pairs: (a0,b0) r=1 -> bin 0, (a1,b1) r=1 -> bin 0, (a1,b0) r=19 -> bin 4,
    (a0,b1) r=21 -> bin 5.  eta_ik eta_jl = +-1/4.  Worked by hand:
    Dt[0,0]=1, Dt[0,4]=Dt[0,5]=-1/2, Dt[4,4]=Dt[4,5]=Dt[5,5]=1/4; W = (2,1,1)."""
    cat, bins = _hand_dm_catalog()
    nb = bins.nbins
    Dt = np.zeros((nb, nb))
    Dt[0, 0] = 1.0
    Dt[0, 4] = Dt[4, 0] = -0.5
    Dt[0, 5] = Dt[5, 0] = -0.5
    Dt[4, 4] = Dt[5, 5] = 0.25
    Dt[4, 5] = Dt[5, 4] = 0.25
    W = np.zeros(nb)
    W[0], W[4], W[5] = 2.0, 1.0, 1.0
    for fn in (odm.dmat_literal, odm.dmat):
        out = fn(cat, bins, pairs.all_pairs(2))
        np.testing.assert_allclose(out["dtilde"], Dt, atol=1e-15)
        np.testing.assert_allclose(out["wsum"], W, atol=1e-15)
        assert out["dmat"][0, 0] == pytest.approx(0.5)
        assert out["dmat"][4, 0] == pytest.approx(-0.5)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dmat_expanded_equals_literal(seed):
    cat = random_small(n_forests=7, max_len=7, seed=seed, zero_weight_forest=(seed == 1),
                       single_pixel_forest=(seed == 2))
    bins = synth.Bins(6, 3, 24.0, 6.0)
    pr = pairs.all_pairs(cat.n_forests)
    lit = odm.dmat_literal(cat, bins, pr)
    exp = odm.dmat(cat, bins, pr)
    scale = np.max(np.abs(lit["dtilde"]))
    assert scale > 0
    np.testing.assert_allclose(exp["dtilde"], lit["dtilde"], atol=1e-12 * scale)
    np.testing.assert_allclose(exp["wsum"], lit["wsum"], rtol=1e-13)


def test_dmat_identity_eta_gives_identity(cat0, bins0):
    sub = synth.subset(cat0, np.arange(30))
    out = odm.dmat(sub, bins0, eta_identity=True)
    on = out["wsum"] > 0
    assert on.sum() > 50
    np.testing.assert_array_equal(out["dmat"][np.ix_(on, on)], np.eye(on.sum()))
    small = random_small(n_forests=5, max_len=5, seed=7)
    lit = odm.dmat_literal(small, synth.Bins(6, 3, 24.0, 6.0), pairs.all_pairs(5), eta_identity=True)
    on = lit["wsum"] > 0
    np.testing.assert_allclose(lit["dmat"][np.ix_(on, on)], np.eye(on.sum()), atol=1e-15)


def test_dmat_rows_sum_to_zero_when_all_pairs_in_grid():
    """If every pixel pair of every forest pair is in the grid,
    sum_B sum_{(k,l) in B} eta_ik eta_jl = (eta 1)_i (eta 1)_j = 0."""
    cat = random_small(n_forests=8, max_len=8, seed=11)
    bins = synth.Bins(6, 2, 60.0, 60.0)   # r_par < 30, r_perp < 2: all in grid, 3 r_par bins
    out = odm.dmat(cat, bins, pairs.all_pairs(8))
    assert np.count_nonzero(out["wsum"]) >= 3
    scale = np.max(out["wsum"])
    np.testing.assert_allclose(out["dtilde"].sum(axis=1), 0.0, atol=1e-11 * scale)
    lit = odm.dmat_literal(cat, bins, pairs.all_pairs(8))
    np.testing.assert_allclose(lit["dtilde"].sum(axis=1), 0.0, atol=1e-11 * scale)


def test_dmat_symmetric_weighted(cat0, bins0):
    sub = synth.subset(cat0, np.arange(40))
    out = odm.dmat(sub, bins0)
    dt = out["dtilde"]
    np.testing.assert_allclose(dt, dt.T, atol=1e-10 * np.max(np.abs(dt)))
    W = out["wsum"]
    D = out["dmat"]
    np.testing.assert_allclose(W[:, None] * D, (W[:, None] * D).T, atol=1e-9 * np.max(np.abs(dt)))
    # W of D equals W of xi over the same pairs
    xo = oxi.xi_sums(sub, bins0)
    np.testing.assert_allclose(W, xo["wsum"], rtol=1e-12)


def test_two_pixel_forests_are_annihilated():
    """Mean + slope fit any two pixels with distinct Lambda exactly: eta = 0, D~ = 0."""
    rng = np.random.default_rng(8)
    fs = [(rng.uniform(0, 1e-4), rng.uniform(0, 1e-4), np.sort(1000 + rng.uniform(0, 20, 2)),
           [8.2, 8.3], [0.0, 0.0], rng.uniform(0.5, 2, 2)) for _ in range(4)]
    cat = line_catalog(fs)
    out = odm.dmat(cat, synth.Bins(6, 2, 24.0, 8.0), pairs.all_pairs(4))
    assert np.max(np.abs(out["dtilde"])) < 1e-12
    assert out["wsum"].sum() > 0


def test_dmat_edge_allowance_brackets_shifted_binning(cat0, bins0):
    """Moving every scaled separation by less than eps changes each D~_AB by
    at most edge_d[A, B]; the bound is not vacuous (pairs do move)."""
    sub = synth.subset(cat0, np.arange(25))
    eps = 1e-3
    pr = pairs.forest_pairs(sub, bins0)
    base = odm.dmat(sub, bins0, pr, eps_edge=eps)
    E = base["edge_d"]
    np.testing.assert_allclose(E, E.T, rtol=1e-12)
    moved_any = False
    for scale in [1 + 0.9 * eps / 25, 1 - 0.9 * eps / 25]:
        b2 = synth.Bins(bins0.n_par, bins0.n_perp, bins0.r_par_max / scale, bins0.r_perp_max / scale)
        moved = odm.dmat(sub, b2, pr)
        diff = np.abs(moved["dtilde"] - base["dtilde"])
        moved_any |= bool(np.any(diff > 1e-6 * np.abs(base["dtilde"]).max()))
        assert np.all(diff <= E * (1 + 1e-9) + 1e-9 * np.abs(base["dtilde"]).max())
    assert moved_any
    # the allowance is small where nothing is near an edge: zero without ambiguous pairs
    far = odm.dmat(sub, bins0, pr, eps_edge=1e-12)
    assert far["edge_d"].sum() < 1e-6 * E.sum()


def test_closed_form_work_counts_by_hand():
    """Two forests, all pixel pairs in one bin except one: the column vectors
    touch {0} and {0, 1}, the rows likewise; the pair touches two bins."""
    from conftest import line_catalog
    from oracle import dmat as odm
    f0 = (0.0, 0.0, [1000.0, 1001.0], [8.2, 8.3], [0.1, 0.2], [1.0, 1.0])
    f1 = (1e-6, 0.0, [1000.5, 1005.5], [8.2, 8.3], [0.3, -0.2], [1.0, 2.0])
    cat = line_catalog([f0, f1])
    bins = synth.Bins(4, 4, 16.0, 16.0)   # 4 Mpc/h bins
    # |d_i - d_j|: (0.5, 5.5), (0.5, 4.5) -> bins p = (0, 1), (0, 1)
    w = odm.closed_form_work(cat, bins, (np.array([0]), np.array([1])))
    assert w["pixel_pairs"] == 4
    # columns: j=0 -> {p0}, j=1 -> {p1}; rows: i=0 -> {p0, p1}, i=1 -> {p0, p1}
    assert w["sum_vec_support_sq"] == 1 + 1 + 4 + 4
    assert w["sum_pair_support_sq"] == 4
    assert w["flops"] == 20 * 4 + 4 * 10 + 8 * 4
