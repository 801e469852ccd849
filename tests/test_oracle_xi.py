"""Pins of the oracle's geometry, pair set and xi/W sums (Eq. 2.4, Section 2.1)
against things other than itself: 3-D vector algebra + numpy.histogram2d,
hand arithmetic, closed forms, brute force."""
import math

import numpy as np
import pytest

import oracle
from oracle import geometry, pairs, xi as oxi
from paper_2507_00129_gb300 import synth
from conftest import line_catalog


def test_unit_vectors_known_points():
    n = geometry.unit_vectors(np.array([0.0, math.pi / 2, 1.0]), np.array([0.0, 0.0, math.pi / 2]))
    np.testing.assert_allclose(n[0], [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(n[1], [0, 1, 0], atol=1e-15)
    np.testing.assert_allclose(n[2], [0, 0, 1], atol=1e-15)


def test_half_angle_on_equator():
    # two points on the equator separated by exactly theta
    for theta in [1e-6, 1e-3, 0.05, 1.0, 3.0]:
        n = geometry.unit_vectors(np.array([0.3, 0.3 + theta]), np.zeros(2))
        c, s = geometry.half_angle(n[0], n[1])
        assert abs(s - math.sin(theta / 2)) < 1e-15
        assert abs(c - math.cos(theta / 2)) < 1e-15


def test_separation_split_matches_3d_projection():
    """r_par, r_perp equal the components of x_i - x_j along the bisector of the
    two lines of sight and along n_a - n_b (3-D vector algebra)."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        ra, dec = rng.uniform(0, 2 * np.pi, 2), rng.uniform(-1.2, 1.2, 2)
        n = geometry.unit_vectors(ra, dec)
        da, db = rng.uniform(3500, 4700, 7), rng.uniform(3500, 4700, 5)
        c, s = geometry.half_angle(n[0], n[1])
        rpar, rperp = geometry.separations(da, db, c, s)
        xa = da[:, None, None] * n[0][None, None, :]
        xb = db[None, :, None] * n[1][None, None, :]
        sep = xa - xb
        u = (n[0] + n[1]) / np.linalg.norm(n[0] + n[1])
        v = (n[0] - n[1]) / np.linalg.norm(n[0] - n[1])
        np.testing.assert_allclose(rpar, np.abs(sep @ u), rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(rperp, np.abs(sep @ v), rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(rpar ** 2 + rperp ** 2, np.sum(sep ** 2, -1), rtol=1e-10)


def test_xi_matches_histogram2d_of_3d_separations():
    """Per-bin N and W of one forest pair against numpy.histogram2d of the 3-D
    separation components (bins [p D, (p+1) D) in r_par, r_perp)."""
    cat = synth.make(0)
    bins = synth.bins_for(0)
    a_arr, b_arr = pairs.forest_pairs(cat, bins)
    rng = np.random.default_rng(1)
    nvec = geometry.unit_vectors(cat.ra, cat.dec)
    for k in rng.choice(len(a_arr), 25, replace=False):
        a, b = int(a_arr[k]), int(b_arr[k])
        sa, sb = cat.forest(a), cat.forest(b)
        sep = cat.dist[sa][:, None, None] * nvec[a] - cat.dist[sb][None, :, None] * nvec[b]
        u = (nvec[a] + nvec[b]) / np.linalg.norm(nvec[a] + nvec[b])
        v = (nvec[a] - nvec[b]) / np.linalg.norm(nvec[a] - nvec[b])
        rpar, rperp = np.abs(sep @ u).ravel(), np.abs(sep @ v).ravel()
        w = (cat.weight[sa].astype(float)[:, None] * cat.weight[sb].astype(float)[None, :]).ravel()
        wda = cat.weight[sa].astype(float) * cat.delta[sa].astype(float)
        wdb = cat.weight[sb].astype(float) * cat.delta[sb].astype(float)
        wd = (wda[:, None] * wdb[None, :]).ravel()
        edges_par = np.linspace(0, bins.r_par_max, bins.n_par + 1)
        edges_perp = np.linspace(0, bins.r_perp_max, bins.n_perp + 1)
        Wh, _, _ = np.histogram2d(rpar, rperp, [edges_par, edges_perp], weights=w)
        Nh, _, _ = np.histogram2d(rpar, rperp, [edges_par, edges_perp], weights=wd)
        out = oxi.xi_sums(cat, bins, (np.array([a]), np.array([b])))
        np.testing.assert_allclose(out["wsum"], Wh.ravel(), rtol=1e-12, atol=1e-9)
        np.testing.assert_allclose(out["num"], Nh.ravel(), rtol=1e-10, atol=1e-9)


def test_hand_built_three_forests():
    """Three forests with hand-chosen distances; every pixel pair's bin is worked
    out by hand below.  Bins of 4 Mpc/h, 3 x 3 grid (r_max = 12)."""
    s = 0.003                       # sin(theta/2) of forest C relative to A and B
    th = 2 * math.asin(s)
    A = (0.0, 0.0, [1000.0, 1003.0, 1010.0], [8.2, 8.21, 8.22], [1.0, -2.0, 0.5], [1.0, 2.0, 3.0])
    B = (0.0, 0.0, [1001.0, 1009.0], [8.2, 8.21], [3.0, 1.0], [2.0, 1.0])
    C = (th, 0.0, [1002.0], [8.2], [-1.0], [4.0])
    cat = line_catalog([A, B, C])
    bins = synth.Bins(3, 3, 12.0, 12.0)
    # A-B (theta = 0): r_par = |dA - dB|, r_perp = 0
    #   (1000,1001) 1 -> p0 ; (1000,1009) 9 -> p2 ; (1003,1001) 2 -> p0
    #   (1003,1009) 6 -> p1 ; (1010,1001) 9 -> p2 ; (1010,1009) 1 -> p0
    # A-C: c = sqrt(1-s^2) ~ 0.9999955, r_perp = (dA+1002) * 0.003 ~ 6.006..6.036 -> t1
    #   (1000,1002) r_par 2.0 -> p0 ; (1003,1002) 1.0 -> p0 ; (1010,1002) 8.0 -> p1 (7.99996)
    # B-C: r_perp = (dB + 1002) * 0.003 ~ 6.009, 6.033 -> t1
    #   (1001,1002) 1 -> p0 ; (1009,1002) 7 -> p1
    wA, dA = [1.0, 2.0, 3.0], [1.0, -2.0, 0.5]
    wB, dB = [2.0, 1.0], [3.0, 1.0]
    wC, dC = 4.0, -1.0
    W = np.zeros(9)
    N = np.zeros(9)

    def add(p, t, wi, di, wj, dj):
        W[p * 3 + t] += wi * wj
        N[p * 3 + t] += wi * di * wj * dj

    ab = {(0, 0): 0, (0, 1): 2, (1, 0): 0, (1, 1): 1, (2, 0): 2, (2, 1): 0}
    for (i, j), p in ab.items():
        add(p, 0, wA[i], dA[i], wB[j], dB[j])
    for i, p in enumerate([0, 0, 1]):
        add(p, 1, wA[i], dA[i], wC, dC)
    for j, p in enumerate([0, 1]):
        add(p, 1, wB[j], dB[j], wC, dC)
    out = oxi.xi_sums(cat, bins, pairs.all_pairs(3))
    np.testing.assert_allclose(out["wsum"], W, rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["num"], N, rtol=0, atol=1e-12)
    xi_expect = np.divide(N, W, out=np.zeros(9), where=W != 0)
    np.testing.assert_allclose(out["xi"], xi_expect, atol=1e-12)
    assert out["count"].sum() == 6 + 3 + 2


def test_single_bin_closed_form():
    """One bin covering every pair: W = ((sum_f W_f)^2 - sum_f W_f^2) / 2 and
    N = ((sum_f S_f)^2 - sum_f S_f^2) / 2 with S_f = sum_i w_i delta_i."""
    cat = synth.generate(synth.Spec(n_forests=30, seed=9, region="box", box_deg=2.0))
    bins = synth.Bins(1, 1, 1e5, 1e5)
    out = oxi.xi_sums(cat, bins, pairs.all_pairs(cat.n_forests))
    Wf = np.array([cat.weight[cat.forest(f)].astype(float).sum() for f in range(cat.n_forests)])
    Sf = np.array([(cat.weight[cat.forest(f)].astype(float) * cat.delta[cat.forest(f)].astype(float)).sum()
                   for f in range(cat.n_forests)])
    assert math.isclose(out["wsum"][0], (Wf.sum() ** 2 - (Wf ** 2).sum()) / 2, rel_tol=1e-12)
    assert math.isclose(out["num"][0], (Sf.sum() ** 2 - (Sf ** 2).sum()) / 2, rel_tol=1e-9, abs_tol=1e-6)


def test_analytic_w_on_regular_grid():
    """Two forests on nearly the same line of sight with d_k = d0 + k h
    and unit weights: pixel pairs at index distance m number n at m = 0 and
    2 (n - m) at m > 0; all have r_perp in bin 0.  h = 0.73 keeps m h / 4 at
    least 1/400 away from an integer for every m < 400 (73 m / 400 is never
    an integer), so no pair sits near an edge."""
    n, h, d0 = 120, 0.73, 3800.0
    eps = 1e-7
    d = d0 + h * np.arange(n)
    f = (0.0, 0.0, d, np.zeros(n), np.zeros(n), np.ones(n))
    g = (eps, 0.0, d, np.zeros(n), np.zeros(n), np.ones(n))
    cat = line_catalog([f, g])
    bins = synth.Bins(20, 2, 80.0, 8.0)
    out = oxi.xi_sums(cat, bins, pairs.all_pairs(2))
    c = math.cos(eps / 2)
    expect = np.zeros(bins.nbins)
    for m in range(n):
        mult = n if m == 0 else 2 * (n - m)
        p = int(math.floor(m * h * c / 4.0))
        if p < bins.n_par:
            expect[p * bins.n_perp + 0] += mult
    np.testing.assert_array_equal(out["wsum"], expect)


def test_pair_set_kdtree_equals_brute_force(cat0, bins0):
    a1, b1 = pairs.forest_pairs(cat0, bins0, method="brute")
    a2, b2 = pairs.forest_pairs(cat0, bins0, method="kdtree")
    np.testing.assert_array_equal(a1, a2)
    np.testing.assert_array_equal(b1, b2)
    assert len(a1) > 1000


def test_cut_drops_no_in_grid_pair(cat0, bins0):
    """The angular cut only removes forest pairs with no in-grid pixel pair."""
    sub = synth.subset(cat0, np.arange(60))
    cut = oxi.xi_sums(sub, bins0, pairs.forest_pairs(sub, bins0))
    full = oxi.xi_sums(sub, bins0, pairs.all_pairs(sub.n_forests))
    np.testing.assert_array_equal(cut["count"], full["count"])
    np.testing.assert_allclose(cut["wsum"], full["wsum"], rtol=1e-13)
    np.testing.assert_allclose(cut["num"], full["num"], rtol=1e-11, atol=1e-9)
    assert full["pairs"] > cut["pairs"]


def test_forest_permutation_invariance(cat0, bins0):
    """xi does not depend on forest order or on which forest of a pair comes first."""
    sub = synth.subset(cat0, np.arange(50))
    perm = np.random.default_rng(3).permutation(50)
    sub2 = synth.subset(sub, perm)
    o1 = oxi.xi_sums(sub, bins0)
    o2 = oxi.xi_sums(sub2, bins0)
    np.testing.assert_allclose(o1["wsum"], o2["wsum"], rtol=1e-12)
    np.testing.assert_allclose(o1["num"], o2["num"], rtol=1e-9, atol=1e-8)
    a, b = pairs.forest_pairs(sub, bins0)
    o3 = oxi.xi_sums(sub, bins0, (b, a))
    np.testing.assert_allclose(o1["wsum"], o3["wsum"], rtol=1e-12)


def test_edge_mass_brackets_shifted_binning(cat0, bins0):
    """Moving every scaled separation by less than eps changes each W_A by at
    most the edge mass E_A computed with eps."""
    sub = synth.subset(cat0, np.arange(40))
    eps = 1e-3
    base = oxi.xi_sums(sub, bins0, eps_edge=eps)
    pr = pairs.forest_pairs(sub, bins0)
    for scale in [1 + 0.9 * eps / 50, 1 - 0.9 * eps / 50]:
        b2 = synth.Bins(bins0.n_par, bins0.n_perp, bins0.r_par_max / scale, bins0.r_perp_max / scale)
        moved = oxi.xi_sums(sub, b2, pr)
        assert np.all(np.abs(moved["wsum"] - base["wsum"]) <= base["edge_w"] * (1 + 1e-12) + 1e-9)
        assert np.all(np.abs(moved["num"] - base["num"]) <= base["edge_n"] * (1 + 1e-12) + 1e-9)
