"""Forest x quasar cross-correlation (lya_xcf), its distortion matrix
(lya_xdmat) and the 1D same-forest correlation (lya_xi1d) against the oracle.

Tolerances:
* xcf: |dW_A| <= 1e-6 W_A + E^W_A and |dN_A| <= 1e-5 sqrt(sum t^2) + E^N_A,
  E the oracle's edge mass for eps = 6e-5 bin units.  The library bins in FP32:
  x = fma(x_i, c/D_par, X0) with |x_i| <= 1100 Mpc/h (half-ulp 6.1e-5 Mpc/h,
  1.5e-5 bin units at D_par = 4), |x_i c/D_par| <= 275 (rounding of c/D_par:
  1.6e-5), |X0| <= 325 (1.9e-5) and the final rounding (4e-6): below 6e-5.
* xdmat: |dD_AB| <= 1e-5 max_B |D_AB| + 3 E^W_A / W_A of that maximum +
  edge_d[A, B] / W_A, as for the auto-correlation's D.
* 1D: bins are decided with the definition's FP64 division, so only the
  summation order differs: 1e-12 relative.
"""
import numpy as np
import pytest
import torch

from oracle import xcf as ox, xi1d as o1
from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu

EPS_EDGE = 6e-5


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_00129_gb300 import build, api as _api
    build.build()
    return _api


@pytest.fixture(scope="module")
def handle(api):
    h = api.Handle()
    yield h
    h.close()


def _np(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def small():
    spec = synth.Spec(n_forests=150, seed=5, region="box", box_deg=2.0, grid="log10", delta_sigma=0.2)
    cat = synth.generate(spec)
    q, own = synth.quasars(spec, cat, extra_fraction=0.5)
    bins = synth.Bins(40, 20, 80.0, 80.0)
    pl = ox.forest_quasar_pairs(cat, q, bins, own)
    return cat, q, own, bins, pl


def _check_xcf(num, wsum, ref):
    W, N = _np(wsum), _np(num)
    assert np.all(np.abs(W - ref["wsum"]) <= 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9)
    assert np.all(np.abs(N - ref["num"]) <= 1e-5 * np.sqrt(ref["num_sq"]) + ref["edge_n"] + 1e-12)


def test_xcf_matches_oracle(api, handle, small):
    cat, q, own, bins, pl = small
    num, wsum, xi = api.lya_xcf(handle, api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q), bins,
                                forest_qso=own)
    api.lya_sync_status(handle)
    ref = ox.xcf_sums(cat, q, bins, pl, eps_edge=EPS_EDGE)
    assert ref["count"].sum() > 1e5 and np.count_nonzero(ref["wsum"]) > 0.9 * bins.nbins
    _check_xcf(num, wsum, ref)
    on = ref["wsum"] > 0
    np.testing.assert_allclose(_np(xi)[on], _np(num)[on] / _np(wsum)[on], rtol=1e-15)
    np.testing.assert_array_equal(_np(xi)[~on], 0.0)


def test_xcf_own_quasar_excluded_or_not(api, handle, small):
    cat, q, own, bins, _ = small
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    num, wsum, _ = api.lya_xcf(handle, dc, dq, bins, forest_qso=None)
    ref = ox.xcf_sums(cat, q, bins, ox.forest_quasar_pairs(cat, q, bins, None), eps_edge=EPS_EDGE)
    _check_xcf(num, wsum, ref)
    # the own quasars sit on the line of sight (r_perp = 0, r_par < 0): only the first r_perp column changes
    _, w_own, _ = api.lya_xcf(handle, dc, dq, bins, forest_qso=own)
    # (the FP64 atomics add in a run-dependent order: equal up to 1e-12 relative)
    W2 = _np(wsum).reshape(bins.n_par, bins.n_perp)
    diff = W2 - _np(w_own).reshape(bins.n_par, bins.n_perp)
    same = np.abs(diff) <= 1e-12 * W2 + 1e-12
    assert np.all(same[:, 1:]) and np.all(same[bins.n_par // 2:, 0])
    assert np.all(diff[: bins.n_par // 2, 0] >= -1e-12 * W2[: bins.n_par // 2, 0])
    assert diff[: bins.n_par // 2, 0].sum() > 1e-6 * W2[: bins.n_par // 2, 0].sum()


def test_pair_list_cache_follows_the_inputs(api, small):
    """The (forest, quasar) list is reused only for the same pointers, sizes,
    bins and geometry: in-place changes of the own-quasar indices or of the
    quasar positions rebuild it."""
    cat, q, own, bins, _ = small
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    own_d = torch.from_numpy(own).cuda()
    h, fresh = api.Handle(), api.Handle()
    try:
        _, w_own, _ = api.lya_xcf(h, dc, dq, bins, forest_qso=own_d)
        _, w_none, _ = api.lya_xcf(fresh, dc, dq, bins, forest_qso=None)
        own_d.fill_(-1)                      # same tensor, no own quasar any more
        _, w2, _ = api.lya_xcf(h, dc, dq, bins, forest_qso=own_d)
        np.testing.assert_allclose(_np(w2), _np(w_none), rtol=1e-12, atol=1e-12)
        assert not np.allclose(_np(w2), _np(w_own), rtol=1e-9, atol=0)
        dq.ra.add_(2e-3)                     # move every quasar in place
        _, w3, _ = api.lya_xcf(h, dc, dq, bins, forest_qso=own_d)
        _, w4, _ = api.lya_xcf(fresh, dc, dq, bins, forest_qso=own_d)
        np.testing.assert_allclose(_np(w3), _np(w4), rtol=1e-12, atol=1e-12)
        assert not np.allclose(_np(w3), _np(w2), rtol=1e-9, atol=0)
    finally:
        h.close()
        fresh.close()


def test_xdmat_matches_oracle(api, handle, small):
    cat, q, own, bins, pl = small
    seed, p = 4321, 0.05
    D, Wd = api.lya_xdmat(handle, api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q), bins, p, seed,
                          forest_qso=own)
    api.lya_sync_status(handle)
    m = ox.keep_xpairs(pl[0], pl[1], seed, p)
    sub = (pl[0][m], pl[1][m])
    assert 0.03 * len(pl[0]) < len(sub[0]) < 0.07 * len(pl[0])
    ref = ox.xdmat(cat, q, bins, sub, eps_edge=EPS_EDGE)
    W = ref["wsum"]
    rowmax = np.abs(ref["dmat"]).max(axis=1)
    rel = np.divide(ref["edge_w"], W, out=np.zeros_like(W), where=W > 0)
    col = np.divide(ref["edge_d"], W[:, None], out=np.zeros_like(ref["edge_d"]), where=W[:, None] > 0)
    tol = (1e-5 + 3 * rel)[:, None] * rowmax[:, None] + col
    assert np.all(np.abs(_np(D) - ref["dmat"]) <= tol + 1e-12)
    assert np.all(np.abs(_np(Wd) - W) <= 1e-6 * W + ref["edge_w"] + 1e-9)
    assert np.count_nonzero(W) > 0.5 * bins.nbins


def test_xdmat_identity_eta_and_empty_subsample(api, handle, small):
    cat, q, own, bins, _ = small
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    D, Wd = api.lya_xdmat(handle, dc, dq, bins, 0.05, 7, forest_qso=own, eta="identity")
    Dg, W = _np(D), _np(Wd)
    on = W > 0
    np.testing.assert_allclose(Dg[np.ix_(on, on)], np.eye(on.sum()), atol=1e-12)
    assert np.all(Dg[~on] == 0)
    D0, W0 = api.lya_xdmat(handle, dc, dq, bins, 0.0, 7, forest_qso=own)
    assert np.all(_np(D0) == 0) and np.all(_np(W0) == 0)


def test_xcf_full_size_sampled(api, handle):
    """60,000 SDSS-like forests and 90,000 quasars: the GPU sums over the first
    120 forests (with every quasar) against the oracle, and the full catalogue
    runs with finite output."""
    spec = synth.spec_for(1)
    cat = synth.generate(spec)
    q, own = synth.quasars(spec, cat, extra_fraction=0.5)
    bins = synth.Bins(100, 50, 200.0, 200.0)
    dq = api.DeviceQuasars.from_host(q)
    num, wsum, xi = api.lya_xcf(handle, api.DeviceCatalog.from_host(cat), dq, bins, forest_qso=own)
    api.lya_sync_status(handle)
    W = _np(wsum)
    assert np.all(np.isfinite(_np(xi))) and np.mean(W > 0) > 0.99
    sub = synth.subset(cat, np.arange(120))
    n2, w2, _ = api.lya_xcf(handle, api.DeviceCatalog.from_host(sub), dq, bins, forest_qso=own[:120])
    ref = ox.xcf_sums(sub, q, bins, ox.forest_quasar_pairs(sub, q, bins, own[:120]), eps_edge=EPS_EDGE)
    assert ref["count"].sum() > 1e6
    _check_xcf(n2, w2, ref)


def test_xi1d_matches_oracle(api, handle):
    cat = synth.make(0)
    for n_bins, r_max in ((25, 100.0), (37, 150.0)):
        num, wsum, xi = api.lya_xi1d(handle, api.DeviceCatalog.from_host(cat), n_bins, r_max)
        ref = o1.xi1d_sums(cat, n_bins, r_max)
        assert ref["count"].sum() > 1e5
        np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-12)
        assert np.all(np.abs(_np(num) - ref["num"]) <= 1e-12 * np.sqrt(ref["num_sq"]) * 1e3 + 1e-12)
        on = ref["wsum"] > 0
        np.testing.assert_allclose(_np(xi)[on], ref["xi"][on], rtol=1e-9, atol=1e-12 * ref["sigma"][on].max())


def test_xi1d_full_size_sampled(api, handle):
    """DESI-like forests (100-600 pixels, 0.57 Mpc/h spacing): the GPU on 3,000
    forests against the oracle on the same forests."""
    cat = synth.make(3, n_forests=3000)
    num, wsum, _ = api.lya_xi1d(handle, api.DeviceCatalog.from_host(cat), 50, 200.0)
    ref = o1.xi1d_sums(cat, 50, 200.0)
    np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-12)
    assert np.all(np.abs(_np(num) - ref["num"]) <= 1e-9 * np.sqrt(ref["num_sq"]) + 1e-12)


def test_errors(api, handle, small):
    cat, q, own, bins, _ = small
    dc, dq = api.DeviceCatalog.from_host(cat), api.DeviceQuasars.from_host(q)
    from paper_2507_00129_gb300._lib import LyaError
    with pytest.raises(LyaError):
        api.lya_xcf(handle, dc, dq, synth.Bins(0, 20, 80.0, 80.0))
    with pytest.raises(LyaError):
        api.lya_xcf(handle, dc, dq, synth.Bins(200, 200, 80.0, 80.0))   # 40,000 bins: above the histogram
    with pytest.raises(LyaError):
        api.lya_xi1d(handle, dc, 0, 100.0)
    with pytest.raises(LyaError):
        api.lya_xdmat(handle, dc, dq, bins, 1.5, 0)
    bad = api.DeviceQuasars(dq.ra, dq.dec, dq.dist.clone(), dq.weight)
    bad.dist[3] = float("nan")
    with pytest.raises(LyaError):
        api.lya_xcf(handle, dc, bad, bins)
    # the handle stays usable
    num, wsum, _ = api.lya_xcf(handle, dc, dq, bins, forest_qso=own)
    assert float(wsum.sum()) > 0
