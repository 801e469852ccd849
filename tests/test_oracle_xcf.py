"""Pins of the oracle's forest x quasar cross-correlation, its distortion
matrix and the same-forest (1D) correlation: hand arithmetic, 3-D vector
geometry, the auto-correlation oracle folded over the sign of r_par, Eq. (2.5)
on a bin-constant field, and the projector identities of Eq. (2.7)."""
import math

import numpy as np

from conftest import line_catalog, random_small
from oracle import xcf as ox, xi1d as o1, xi as oxi, project as oproj
from paper_2507_00129_gb300 import synth


def _qso(ra, dec, dist, w):
    z = np.zeros(len(ra))
    return synth.Quasars(ra=np.asarray(ra, float), dec=np.asarray(dec, float), dist=np.asarray(dist, float),
                         weight=np.asarray(w, np.float32), z=z)


def _axis_forest(d, delta, w):
    return (0.0, math.pi / 2, d, np.log(3600.0 + np.arange(len(d))), delta, w)


def test_hand_built_pair_signed_r_par():
    """Forest on the z axis, pixels at 1000, 1004, 1010 (w = 1, 2, 3; delta = 0.5, -1, 2).
    Quasar at angle theta = 2 asin(0.01) from the axis, d_q = 1006, w_q = 1.5:
    r_perp = (d + 1006) 0.01 = 20.06, 20.10, 20.16 -> t = 2 (width 10);
    r_par = (d - 1006) cos(theta/2) = -5.9997, -1.9999, 3.9998 -> with
    [-20, 20) in 10 bins of 4: x = 3.50008, 4.50003, 5.99995 -> p = 3, 4, 5."""
    cat = line_catalog([_axis_forest([1000.0, 1004.0, 1010.0], [0.5, -1.0, 2.0], [1.0, 2.0, 3.0])])
    theta = 2 * math.asin(0.01)
    q = _qso([0.0, 1.0], [math.pi / 2 - theta, math.pi / 2], [1006.0, 1200.0], [1.5, 7.0])
    bins = synth.Bins(10, 5, 20.0, 50.0)
    out = ox.xcf_sums(cat, q, bins, pair_list=(np.array([0]), np.array([0])))
    A = [3 * 5 + 2, 4 * 5 + 2, 5 * 5 + 2]
    np.testing.assert_allclose(out["wsum"][A], [1.5, 3.0, 4.5], rtol=1e-15)
    np.testing.assert_allclose(out["num"][A], [0.75, -3.0, 9.0], rtol=1e-15)
    assert out["count"].sum() == 3
    # the default pair list finds both quasars; quasar 1 is the forest's own and is excluded
    both = ox.forest_quasar_pairs(cat, q, bins)
    own = ox.forest_quasar_pairs(cat, q, bins, forest_qso=np.array([1]))
    assert list(both[1]) == [0, 1] and list(own[1]) == [0]
    np.testing.assert_array_equal(ox.xcf_sums(cat, q, bins, forest_qso=np.array([1]))["wsum"], out["wsum"])


def test_bins_from_3d_vectors():
    """Every (pixel, quasar) bin equals the one found from the 3-D positions:
    r_par = (x_i - x_q) . (n_a + n_q)/|n_a + n_q|, r_perp the rest of |x_i - x_q|."""
    cat = random_small(n_forests=6, max_len=7, patch_deg=0.8, seed=4, spread=40.0)
    rng = np.random.default_rng(5)
    nq = 9
    q = _qso(rng.uniform(0, np.radians(0.8), nq), rng.uniform(0, np.radians(0.8), nq),
             1000.0 + rng.uniform(0, 40.0, nq), rng.uniform(0.5, 2.0, nq))
    bins = synth.Bins(8, 4, 16.0, 16.0)
    out = ox.xcf_sums(cat, q, bins, pair_list=(np.repeat(np.arange(6), nq), np.tile(np.arange(nq), 6)))
    W = np.zeros(bins.nbins)
    N = np.zeros(bins.nbins)
    def unit(ra, dec):
        return np.array([math.cos(dec) * math.cos(ra), math.cos(dec) * math.sin(ra), math.sin(dec)])
    for a in range(6):
        na = unit(cat.ra[a], cat.dec[a])
        for k in range(nq):
            nqv = unit(q.ra[k], q.dec[k])
            u = (na + nqv) / np.linalg.norm(na + nqv)
            for i in range(cat.offsets[a], cat.offsets[a + 1]):
                v = cat.dist[i] * na - q.dist[k] * nqv
                rp = float(v @ u)
                rt = math.sqrt(max(float(v @ v) - rp * rp, 0.0))
                p = math.floor((rp + 16.0) / 4.0)
                t = math.floor(rt / 4.0)
                if 0 <= p < 8 and t < 4:
                    W[p * 4 + t] += float(cat.weight[i]) * float(q.weight[k])
                    N[p * 4 + t] += float(cat.weight[i]) * float(cat.delta[i]) * float(q.weight[k])
    assert W.sum() > 0 and np.count_nonzero(W) > 10
    np.testing.assert_allclose(out["wsum"], W, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(out["num"], N, rtol=1e-9, atol=1e-12)


def test_folds_onto_auto_correlation():
    """A quasar is a one-pixel forest with delta = 1: the auto-correlation
    oracle's sums (|r_par| over n bins) equal the cross sums over 2n bins of
    [-R, R) folded about r_par = 0."""
    cat = random_small(n_forests=5, max_len=8, patch_deg=0.5, seed=11, spread=30.0)
    rng = np.random.default_rng(12)
    nq = 6
    q = _qso(rng.uniform(0, np.radians(0.5), nq), rng.uniform(0, np.radians(0.5), nq),
             1000.0 + rng.uniform(0, 30.0, nq), rng.uniform(0.5, 2.0, nq))
    n_auto = 5
    bx = synth.Bins(2 * n_auto, 4, 20.0, 20.0)
    ba = synth.Bins(n_auto, 4, 20.0, 20.0)
    pl = (np.repeat(np.arange(5), nq), np.tile(np.arange(nq), 5))
    cx = ox.xcf_sums(cat, q, bx, pair_list=pl)
    # the same pairs as forests: catalogue = forests + one-pixel quasar "forests" with delta = 1
    qf = [(q.ra[k], q.dec[k], [q.dist[k]], [8.2], [1.0], [float(q.weight[k])]) for k in range(nq)]
    fs = [(cat.ra[a], cat.dec[a], cat.dist[cat.forest(a)], cat.loglam[cat.forest(a)], cat.delta[cat.forest(a)],
           cat.weight[cat.forest(a)]) for a in range(5)]
    both = line_catalog(fs + qf)
    pa = (np.repeat(np.arange(5), nq), np.tile(np.arange(5, 5 + nq), 5))
    ca = oxi.xi_sums(both, ba, pa)
    for key in ("wsum", "num", "count"):
        X = cx[key].reshape(2 * n_auto, 4)
        folded = X[n_auto:] + X[n_auto - 1::-1]
        np.testing.assert_allclose(folded.ravel(), ca[key], rtol=1e-12, atol=1e-12)
    assert ca["count"].sum() > 20


def _dm_case(seed=21, n_forests=6, nq=7, r_max=200.0):
    cat = random_small(n_forests=n_forests, max_len=7, patch_deg=0.6, seed=seed, spread=30.0)
    rng = np.random.default_rng(seed + 1)
    q = _qso(rng.uniform(0, np.radians(0.6), nq), rng.uniform(0, np.radians(0.6), nq),
             1000.0 + rng.uniform(0, 30.0, nq), rng.uniform(0.5, 2.0, nq))
    bins = synth.Bins(8, 4, r_max, r_max)
    return cat, q, bins


def test_dmat_closed_form_equals_literal():
    cat, q, bins = _dm_case(r_max=24.0)
    pl = ox.forest_quasar_pairs(cat, q, bins)
    lit = ox.xdmat_literal(cat, q, bins, pl)
    cf = ox.xdmat(cat, q, bins, pl)
    assert np.count_nonzero(lit["wsum"]) > 8
    np.testing.assert_allclose(cf["dtilde"], lit["dtilde"], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(cf["wsum"], lit["wsum"], rtol=1e-13)
    # W_A of the distortion matrix is the estimator's weight sum over the same pairs
    np.testing.assert_allclose(cf["wsum"], ox.xcf_sums(cat, q, bins, pl)["wsum"], rtol=1e-13)
    # D~ is symmetric: W_A D_AB = W_B D_BA
    np.testing.assert_allclose(cf["dtilde"], cf["dtilde"].T, rtol=1e-12, atol=1e-13)


def test_dmat_identity_eta_and_zero_rows():
    cat, q, bins = _dm_case(r_max=24.0)
    pl = ox.forest_quasar_pairs(cat, q, bins)
    out = ox.xdmat(cat, q, bins, pl, eta_identity=True)
    on = out["wsum"] > 0
    np.testing.assert_allclose(out["dmat"][np.ix_(on, on)], np.eye(on.sum()), atol=1e-15)
    assert np.all(out["dmat"][~on] == 0)


def test_dmat_row_sums_vanish_when_every_pixel_is_in_grid():
    """With every pixel of every pair in the grid, sum_B alpha_q[B] = W_a and
    sum_B beta_q[B] = sum w x = 0, so every row of D sums to 0 (eta 1 = 0)."""
    cat, q, _ = _dm_case(r_max=500.0)
    bins = synth.Bins(8, 4, 40.0, 500.0)
    pl = ox.forest_quasar_pairs(cat, q, bins)
    assert ox.xcf_sums(cat, q, bins, pl)["count"].sum() == sum(cat.lengths()[a] for a in pl[0])
    out = ox.xdmat(cat, q, bins, pl)
    on = out["wsum"] > 0
    assert on.sum() >= 3
    assert np.max(np.abs(out["dmat"][on].sum(axis=1))) < 1e-12


def test_dmat_maps_bin_constant_field_onto_projected_estimate():
    """Eq. (2.5): with one quasar per forest, every pixel in the grid and
    delta_k = xi_B on the pixels of bin B, the estimator of the projected
    field eta delta equals D xi."""
    cat, q, bins = _dm_case(seed=31, n_forests=6, nq=6, r_max=500.0)
    bins = synth.Bins(8, 4, 40.0, 500.0)
    pl = (np.arange(6), np.arange(6))
    rng = np.random.default_rng(3)
    xi_true = rng.normal(0, 1, bins.nbins)
    A_of = np.zeros(cat.n_pix, dtype=np.int64)
    from oracle.geometry import unit_vectors, half_angle
    nf, nq = unit_vectors(cat.ra, cat.dec), unit_vectors(q.ra, q.dec)
    for a in range(6):
        sl = cat.forest(a)
        c, s = half_angle(nf[a], nq[a])
        A, ok, _, _ = ox.pixel_bins(cat.dist[sl], q.dist[a], c, s, bins)
        assert np.all(ok)
        A_of[sl] = A
    delta = xi_true[A_of]
    est = ox.xcf_sums(cat, q, bins, pl, delta=oproj.project(cat, delta))
    D = ox.xdmat(cat, q, bins, pl)
    on = est["wsum"] > 0
    np.testing.assert_allclose(est["xi"][on], (D["dmat"] @ xi_true)[on], rtol=1e-10, atol=1e-12)


def test_subsample_rule_and_fraction():
    a = np.repeat(np.arange(200), 100)
    k = np.tile(np.arange(100), 200)
    m = ox.keep_xpairs(a, k, 99, 0.25)
    assert 0.23 < m.mean() < 0.27
    np.testing.assert_array_equal(m, ox.keep_xpairs(a, k, 99, 0.25))
    # the pair is ordered: (a, q) and (q, a) are different draws
    assert np.mean(m != ox.keep_xpairs(k, a, 99, 0.25)) > 0.2
    assert ox.keep_xpairs(a, k, 99, 1.0).all() and not ox.keep_xpairs(a, k, 99, 0.0).any()


def test_dmat_edge_allowance_bounds_rebinning():
    """Moving the pixels that lie within eps of an edge to a neighbouring bin
    (here: a shift of every distance by +-eps/2 bin widths) changes D~ by no
    more than edge_d and W by no more than edge_w."""
    cat, q, bins = _dm_case(seed=41, r_max=24.0)
    pl = ox.forest_quasar_pairs(cat, q, bins)
    eps = 0.02
    ref = ox.xdmat(cat, q, bins, pl, eps_edge=eps)
    for shift in (+0.4, -0.4):
        moved = synth.Catalog(ra=cat.ra, dec=cat.dec, offsets=cat.offsets,
                              dist=cat.dist + shift * eps * (2 * bins.r_par_max / bins.n_par),
                              loglam=cat.loglam, delta=cat.delta, weight=cat.weight)
        alt = ox.xdmat(moved, q, bins, pl)
        assert np.all(np.abs(alt["dtilde"] - ref["dtilde"]) <= ref["edge_d"] + 1e-12)
        assert np.all(np.abs(alt["wsum"] - ref["wsum"]) <= ref["edge_w"] + 1e-12)


def test_synthetic_quasars():
    spec = synth.Spec(n_forests=40, seed=3, region="box", box_deg=1.0)
    cat = synth.generate(spec)
    q, own = synth.quasars(spec, cat, extra_fraction=0.5)
    assert q.n == 60 and list(own) == list(range(40))
    np.testing.assert_array_equal(q.ra[:40], cat.ra)
    # a forest's pixels lie in front of its own quasar
    for a in range(40):
        assert cat.dist[cat.offsets[a + 1] - 1] < q.dist[a]
    assert np.all((q.z[40:] >= 1.8) & (q.z[40:] <= 3.5))
    np.testing.assert_allclose(q.weight, ((1 + q.z) / 3.25) ** 0.44, rtol=1e-6)


# -------------------------------------------------------------- 1D correlation
def test_1d_hand_built():
    """Pixels at 1000, 1003, 1009 (bins of 4): separations 3, 9, 6 -> bins 0, 2, 1."""
    cat = line_catalog([_axis_forest([1000.0, 1003.0, 1009.0], [1.0, -2.0, 0.5], [1.0, 2.0, 4.0])])
    out = o1.xi1d_sums(cat, 3, 12.0)
    np.testing.assert_allclose(out["wsum"], [2.0, 8.0, 4.0])
    np.testing.assert_allclose(out["num"], [1.0 * -4.0, -4.0 * 2.0, 1.0 * 2.0])


def test_1d_analytic_weights():
    """d_k = d0 + 0.73 k, w = 1: W_p counts the (n - m) pairs at lag m with
    floor(0.73 m / D) = p (73 m - 400 j is a non-zero integer for m < 400, so
    every lag stays at least 0.01 from an edge)."""
    n, h, D, nb = 60, 0.73, 4.0, 8
    cat = line_catalog([_axis_forest(1000.0 + h * np.arange(n), np.zeros(n), np.ones(n))])
    out = o1.xi1d_sums(cat, nb, nb * D)
    W = np.zeros(nb)
    for m in range(1, n):
        p = math.floor(h * m / D)
        if p < nb:
            W[p] += n - m
    np.testing.assert_array_equal(out["wsum"], W)


def test_1d_equals_auto_of_two_copies():
    """Two copies of one forest on the same line of sight (theta = 0): the auto
    oracle's r_perp bin 0 holds both orders of every same-forest pair plus the
    i = j terms, all at r_par = |d_i - d_j|."""
    cat = random_small(n_forests=1, max_len=40, seed=7, spread=60.0)
    f = (cat.ra[0], cat.dec[0], cat.dist, cat.loglam, cat.delta, cat.weight)
    two = line_catalog([f, f])
    ba = synth.Bins(6, 3, 30.0, 30.0)
    auto = oxi.xi_sums(two, ba, (np.array([0]), np.array([1])))
    one = o1.xi1d_sums(cat, 6, 30.0)
    w = cat.weight.astype(float)
    wd = w * cat.delta.astype(float)
    W0 = auto["wsum"].reshape(6, 3)
    N0 = auto["num"].reshape(6, 3)
    zero = np.zeros(6)
    zero[0] = 1.0
    np.testing.assert_allclose(W0[:, 0], 2 * one["wsum"] + zero * np.sum(w * w), rtol=1e-13)
    np.testing.assert_allclose(N0[:, 0], 2 * one["num"] + zero * np.sum(wd * wd), rtol=1e-12, atol=1e-12)
    assert np.all(W0[:, 1:] == 0)



def test_xcf_edge_masses_bound_rebinning():
    """Shifting every pixel distance by +-0.4 eps bin widths moves only pixels
    within eps of an edge: |dW| <= edge_w and |dN| <= edge_n per bin."""
    cat, q, bins = _dm_case(seed=51, r_max=24.0)
    pl = ox.forest_quasar_pairs(cat, q, bins)
    eps = 0.02
    ref = ox.xcf_sums(cat, q, bins, pl, eps_edge=eps)
    moved_any = False
    for shift in (+0.4, -0.4):
        moved = synth.Catalog(ra=cat.ra, dec=cat.dec, offsets=cat.offsets,
                              dist=cat.dist + shift * eps * (2 * bins.r_par_max / bins.n_par),
                              loglam=cat.loglam, delta=cat.delta, weight=cat.weight)
        alt = ox.xcf_sums(moved, q, bins, pl)
        assert np.all(np.abs(alt["wsum"] - ref["wsum"]) <= ref["edge_w"] + 1e-12)
        assert np.all(np.abs(alt["num"] - ref["num"]) <= ref["edge_n"] + 1e-12)
        moved_any |= bool(np.any(alt["count"] != ref["count"]))
    assert moved_any and ref["edge_w"].sum() > 0


def test_pair_prefilter_drops_nothing():
    """The (forest, quasar) prefilter keeps every pair with an in-grid or
    edge-ambiguous pixel: sums over all pairs equal sums over the kept ones."""
    spec = synth.Spec(n_forests=40, seed=9, region="box", box_deg=1.5, grid="log10")
    cat = synth.generate(spec)
    q, own = synth.quasars(spec, cat, extra_fraction=0.5)
    bins = synth.Bins(20, 10, 40.0, 40.0)
    kept = ox.forest_quasar_pairs(cat, q, bins, own)
    a = np.repeat(np.arange(cat.n_forests), q.n)
    k = np.tile(np.arange(q.n), cat.n_forests)
    m = k != own[a]
    everything = (a[m], k[m])
    assert len(kept[0]) < 0.9 * len(everything[0])
    r1 = ox.xcf_sums(cat, q, bins, kept, eps_edge=1e-3)
    r2 = ox.xcf_sums(cat, q, bins, everything, eps_edge=1e-3)
    for key in ("wsum", "num", "count", "edge_w"):
        np.testing.assert_array_equal(r1[key], r2[key])
    assert r1["count"].sum() > 1000
