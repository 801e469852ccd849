"""Per-bin means and pixel-pair counts (lya_xi_bin_means) against the oracle
(oracle.xi.bin_means).

Tolerances: the bins are the mixed path's FP32 ones, so pairs within eps =
6e-5 bin widths of an edge may sit in a neighbouring bin (E^W_A their weight,
E^C_A their number, from the oracle).  Such a pair moves a bin's mean by at
most (its weight / W_A) times its distance to the mean: below one bin width
for r_par and r_perp and below the bin's spread of pair distances for
dist_mean, so the allowance is 2 E^W_A / W_A of that range.  Beyond it: FP32
run sums (1e-6 relative).  Counts: |dN_A| <= E^C_A.  W is held to the W bar
of the pair kernel, 1e-6 W + E^W."""
import numpy as np
import pytest
import torch

import oracle
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


def test_bin_means_match_oracle(api, handle):
    cat = synth.make(0)
    bins = synth.bins_for(0)
    pr = oracle.pairs.forest_pairs(cat, bins)
    out = api.lya_xi_bin_means(handle, api.DeviceCatalog.from_host(cat), bins)
    api.lya_sync_status(handle)
    ref = oracle.xi.bin_means(cat, bins, pr, eps_edge=EPS_EDGE)
    on = _check_means(out, ref, bins)
    assert on.sum() > 0.9 * bins.nbins
    assert np.all(_np(out["rpar_mean"])[~on] == 0) and np.all(_np(out["count"])[~on] == 0)


def _check_means(out, ref, bins):
    W = ref["wsum"]
    on = W > 0
    frac = np.divide(ref["edge_w"], W, out=np.zeros_like(W), where=on)
    assert np.all(np.abs(_np(out["wsum"]) - W) <= 1e-6 * W + ref["edge_w"] + 1e-9)
    assert np.all(np.abs(_np(out["count"]) - ref["count"]) <= ref["edge_c"])
    dp, dt = bins.r_par_max / bins.n_par, bins.r_perp_max / bins.n_perp
    for key, rng in (("rpar_mean", dp), ("rperp_mean", dt)):
        g, r = _np(out[key])[on], ref[key][on]
        assert np.all(np.abs(g - r) <= 1e-6 * np.abs(r) + 2 * frac[on] * rng + 1e-9), key
    spread = 1500.0
    g, r = _np(out["dist_mean"])[on], ref["dist_mean"][on]
    assert np.all(np.abs(g - r) <= 1e-6 * r + 2 * frac[on] * spread)
    return on


def test_bin_mean_redshift_matches_oracle(api, handle):
    """Per-bin mean redshift with pixel redshifts z = lambda / 1215.67 - 1 from
    the catalogue's log wavelengths (200-forest catalogue).  A pixel pair
    within eps of an edge moves the mean by at most its weight fraction times
    the bin's spread of redshifts (below 2); FP32 redshifts and run sums add
    1e-6 relative."""
    cat = synth.make(0)
    bins = synth.bins_for(0)
    pr = oracle.pairs.forest_pairs(cat, bins)
    z = np.exp(cat.loglam) / 1215.67 - 1.0
    out = api.lya_xi_bin_means(handle, api.DeviceCatalog.from_host(cat), bins, z_pix=torch.from_numpy(z).cuda())
    api.lya_sync_status(handle)
    ref = oracle.xi.bin_means(cat, bins, pr, eps_edge=EPS_EDGE, z=z)
    on = _check_means(out, ref, bins)
    W = ref["wsum"]
    frac = np.divide(ref["edge_w"], W, out=np.zeros_like(W), where=on)
    g, r = _np(out["z_mean"])[on], ref["z_mean"][on]
    assert np.all(np.abs(g - r) <= 1e-6 * r + 2 * frac[on] * 2.0)
    assert np.all(_np(out["z_mean"])[~on] == 0)
    assert np.all((r > 1.9) & (r < 3.6))


def test_bin_means_sdss_density_against_oracle(api, handle):
    """The 450 forests nearest the cap centre of the 60,000-forest SDSS-like
    catalogue (its sky density, grid and 50 x 50 bins to 200 Mpc/h) against the
    oracle at the W bar, 1e-6 W + E^W."""
    cat = synth.make(1)
    bins = synth.bins_for(1)
    sub = synth.subset(cat, np.argsort(-cat.dec)[:450])
    pr = oracle.pairs.forest_pairs(sub, bins)
    assert len(pr[0]) > 2e4
    out = api.lya_xi_bin_means(handle, api.DeviceCatalog.from_host(sub), bins)
    api.lya_sync_status(handle)
    ref = oracle.xi.bin_means(sub, bins, pr, eps_edge=EPS_EDGE, processes=0)
    on = _check_means(out, ref, bins)
    assert on.sum() > 0.5 * bins.nbins


def test_bin_means_full_size_properties(api, handle):
    """60,000 SDSS-like forests: the counts equal the exact in-grid pixel-pair
    count of the pair kernel's binning up to edge flips, and every mean lies in
    its bin."""
    cat = synth.make(1)
    bins = synth.bins_for(1)
    dc = api.DeviceCatalog.from_host(cat)
    out = api.lya_xi_bin_means(handle, dc, bins)
    stats = api.lya_pair_stats(handle, dc, bins)
    api.lya_sync_status(handle)
    n = float(_np(out["count"]).sum())
    assert n > 1e11
    assert abs(n - stats["pixel_pairs"]) <= 1e-5 * n
    W = _np(out["wsum"])
    on = W > 0
    assert on.sum() > 0.9 * bins.nbins
    p, t = np.divmod(np.arange(bins.nbins), bins.n_perp)
    dp, dt = bins.r_par_max / bins.n_par, bins.r_perp_max / bins.n_perp
    rp, rt = _np(out["rpar_mean"])[on], _np(out["rperp_mean"])[on]
    assert np.all(rp >= p[on] * dp - 1e-3) and np.all(rp <= (p[on] + 1) * dp + 1e-3)
    assert np.all(rt >= t[on] * dt - 1e-3) and np.all(rt <= (t[on] + 1) * dt + 1e-3)
    dm = _np(out["dist_mean"])[on]
    assert np.all((dm > 3400) & (dm < 4800))
