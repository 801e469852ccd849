"""Pins of the gradient oracle (central finite differences; exact in delta
because xi is quadratic in delta) and of the SplitMix64 subsample rule
(published first outputs of SplitMix64 seeded with 0)."""
import numpy as np
import pytest

from oracle import adjoint, pairs, subsample
from paper_2507_00129_gb300 import synth


@pytest.fixture(scope="module")
def small():
    cat = synth.subset(synth.make(0), np.arange(25))
    bins = synth.bins_for(0)
    pr = pairs.forest_pairs(cat, bins)
    c = np.random.default_rng(303).normal(size=bins.nbins)
    return cat, bins, pr, c


def test_grad_delta_central_difference_exact(small):
    cat, bins, pr, c = small
    d0 = cat.delta.astype(np.float64)
    gd, gw, _ = adjoint.xi_grad(cat, bins, c, pr, delta=d0)
    rng = np.random.default_rng(304)
    for i in rng.choice(cat.n_pix, 12, replace=False):
        h = 0.37  # any step: L is quadratic in each delta_i with no delta_i^2 term
        dp, dm = d0.copy(), d0.copy()
        dp[i] += h
        dm[i] -= h
        fd = (adjoint.loss(cat, bins, c, pr, delta=dp) - adjoint.loss(cat, bins, c, pr, delta=dm)) / (2 * h)
        assert fd == pytest.approx(gd[i], rel=1e-9, abs=1e-12)


def test_grad_weight_central_difference(small):
    cat, bins, pr, c = small
    w0 = cat.weight.astype(np.float64)
    gd, gw, _ = adjoint.xi_grad(cat, bins, c, pr)
    rng = np.random.default_rng(305)
    for i in rng.choice(cat.n_pix, 12, replace=False):
        h = 1e-3 * w0[i]
        wp, wm = w0.copy(), w0.copy()
        wp[i] += h
        wm[i] -= h
        fd = (adjoint.loss(cat, bins, c, pr, weight=wp) - adjoint.loss(cat, bins, c, pr, weight=wm)) / (2 * h)
        assert fd == pytest.approx(gw[i], rel=1e-5, abs=1e-9 * max(1.0, abs(gw).max()))


def test_grad_weight_with_weight_sum_term_central_difference(small):
    """L = sum c_A xi_A + sum e_A W_A: the W term adds sum_j e_A w_j to dL/dw_i
    and nothing to dL/d delta_i (W does not depend on delta)."""
    cat, bins, pr, c = small
    e = np.random.default_rng(306).normal(size=bins.nbins) * 1e-3
    w0 = cat.weight.astype(np.float64)
    gd0, _, _ = adjoint.xi_grad(cat, bins, c, pr)
    gd, gw, _ = adjoint.xi_grad(cat, bins, c, pr, grad_wsum=e)
    np.testing.assert_array_equal(gd, gd0)
    rng = np.random.default_rng(307)
    for i in rng.choice(cat.n_pix, 12, replace=False):
        h = 1e-3 * w0[i]
        wp, wm = w0.copy(), w0.copy()
        wp[i] += h
        wm[i] -= h
        fd = (adjoint.loss(cat, bins, c, pr, weight=wp, grad_wsum=e)
              - adjoint.loss(cat, bins, c, pr, weight=wm, grad_wsum=e)) / (2 * h)
        assert fd == pytest.approx(gw[i], rel=1e-5, abs=1e-9 * max(1.0, abs(gw).max()))
    # with c = 0 the gradient is exactly dW/dw contracted with e: sum over partners j of e_A w_j,
    # which FD gets up to the rounding of the two losses (W is linear in each w_i)
    z = np.zeros(bins.nbins)
    _, gw_e, _ = adjoint.xi_grad(cat, bins, z, pr, grad_wsum=e)
    for i in rng.choice(cat.n_pix, 6, replace=False):
        wp, wm = w0.copy(), w0.copy()
        wp[i] += 0.5
        wm[i] -= 0.5
        fd = adjoint.loss(cat, bins, z, pr, weight=wp, grad_wsum=e) - adjoint.loss(cat, bins, z, pr, weight=wm,
                                                                                      grad_wsum=e)
        assert fd == pytest.approx(gw_e[i], rel=1e-7, abs=1e-15)


def test_grad_zero_for_pixels_without_pairs():
    # forest 0 far from the others: no in-grid pair, zero gradient
    from conftest import line_catalog
    f0 = (0.0, 0.0, [1000.0, 1001.0], [8.2, 8.3], [0.1, 0.2], [1.0, 1.0])
    f1 = (0.5, 0.0, [1000.0, 1001.0], [8.2, 8.3], [0.1, 0.2], [1.0, 1.0])
    f2 = (0.5, 1e-5, [1000.5, 1003.0], [8.2, 8.3], [0.3, -0.2], [1.0, 2.0])
    cat = line_catalog([f0, f1, f2])
    bins = synth.Bins(4, 4, 16.0, 16.0)
    gd, gw, _ = adjoint.xi_grad(cat, bins, np.ones(16), pairs.all_pairs(3))
    assert np.all(gd[:2] == 0) and np.all(gw[:2] == 0)
    assert np.any(gd[2:] != 0)


def test_splitmix64_published_first_outputs():
    # SplitMix64 seeded with 0: the first four outputs
    expect = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    golden = 0x9E3779B97F4A7C15
    states = np.array([(k * golden) % 2 ** 64 for k in range(4)], dtype=np.uint64)
    got = subsample.splitmix64(states)
    assert [int(g) for g in got] == expect


def test_subsample_rule():
    rng = np.random.default_rng(0)
    a = rng.integers(0, 10 ** 6, 200_000)
    b = a + rng.integers(1, 10 ** 5, 200_000)
    for p in [0.02, 0.05, 0.5]:
        m = subsample.keep_pairs(a, b, seed=42, p=p)
        n = len(a)
        assert abs(m.mean() - p) < 5 * np.sqrt(p * (1 - p) / n)
        np.testing.assert_array_equal(m, subsample.keep_pairs(b, a, seed=42, p=p))
        assert not np.array_equal(m, subsample.keep_pairs(a, b, seed=43, p=p))
    assert subsample.keep_pairs(a, b, 1, 1.0).all()
    assert not subsample.keep_pairs(a, b, 1, 0.0).any()
    assert subsample.threshold(0.5) == 2 ** 63
