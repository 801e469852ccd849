"""Errors of the CUDA path against the CPU FP64 oracle, per workload and
output, as numbers (and held to the parity bars):

* W:  max |dW_A| / W_A, raw and net of the edge mass E^W_A (the weight of pixel
  pairs within eps = 6e-5 bin widths of an edge, which FP32 separations may bin
  either way);
* xi: max |dxi_A| / max(|xi_A|, sigma_A), raw and net of (E^N_A + |xi_A| E^W_A)
  / (W_A - E^W_A) (xi = N / W: flips move it by (dN - xi dW) / (W + dW)); also
  the plain relative error over bins with |xi_A| > 10 sigma_A;
* D:  max |dD_AB| / max_B' |D_AB'|, raw and net of the edge allowance
  (E^D_AB + |D_AB| E^W_A) / (W_A - E^W_A); also the plain relative error over
  entries above 1e-3 of their row's maximum.

Workloads: the 200-forest catalogue in full (xi, W and D, both precisions);
seeded forest-pair samples of the 60,000-forest SDSS-DR16-like catalogue and
of a 60,000-forest patch at the DESI-Y5-like density and grid (xi, W; D on a
smaller sample); four 400-forest patches of the mock-batch workload through
the batched kernel, in full (per-mock xi).  With LYA_ERROR_TABLE=<path> the
table is written there as JSON.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2507_00129_gb300 import synth

pytestmark = pytest.mark.gpu

EPS = 6e-5
TABLE = {}


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
    path = os.environ.get("LYA_ERROR_TABLE")
    if path and TABLE:
        with open(path, "w") as f:
            json.dump(TABLE, f, indent=1, sort_keys=True)


def _np(t):
    return t.detach().cpu().numpy()


def w_errors(W, ref):
    on = ref["wsum"] > 0
    Wr, E = ref["wsum"][on], ref["edge_w"][on]
    dW = np.abs(W[on] - Wr)
    out = {"W_raw": float(np.max(dW / Wr)), "W_net": float(np.max(np.maximum(dW - E, 0) / Wr))}
    assert out["W_net"] <= 1e-6
    return out


def xi_errors(W, N, X, ref):
    on = ref["wsum"] > 0
    Wr, E, En = ref["wsum"][on], ref["edge_w"][on], ref["edge_n"][on]
    xr, sg = ref["xi"][on], ref["sigma"][on]
    dW = np.abs(W[on] - Wr)
    dx = np.abs(X[on] - xr)
    scale = np.maximum(np.abs(xr), sg)
    strong = np.abs(xr) > 10 * sg
    out = {"bins": int(on.sum()),
           "W_raw": float(np.max(dW / Wr)), "W_net": float(np.max(np.maximum(dW - E, 0) / Wr)),
           "xi_raw": float(np.max(dx / scale)),
           "xi_net": float(np.max(np.maximum(dx - np.divide(En + np.abs(xr) * E, Wr - E, out=np.full_like(Wr, np.inf),
                                                            where=Wr > E), 0) / scale)),
           "xi_plain_rel_strong_bins": float(np.max(dx[strong] / np.abs(xr[strong]))) if strong.any() else None,
           "strong_bins": int(strong.sum())}
    # the parity bars
    assert out["W_net"] <= 1e-6
    assert out["xi_net"] <= 1e-5
    assert np.all(X[~on] == 0)
    return out


def d_errors(D, ref_d, ref_x):
    W, E, Dr = ref_x["wsum"], ref_x["edge_w"], ref_d["dmat"]
    on = W > 0
    rowmax = np.abs(Dr).max(axis=1)
    den = (W - E)[:, None]
    allow = np.divide(ref_d["edge_d"] + np.abs(Dr) * E[:, None], den, out=np.zeros_like(Dr), where=den > 0)
    dd = np.abs(D - Dr)
    rm = np.where(rowmax > 0, rowmax, 1.0)[:, None]
    big = (np.abs(Dr) > 1e-3 * rowmax[:, None]) & on[:, None]
    out = {"D_raw": float(np.max((dd / rm)[on])), "D_net": float(np.max((np.maximum(dd - allow, 0) / rm)[on])),
           "D_plain_rel_large_entries": float(np.max(dd[big] / np.abs(Dr[big]))),
           "D_plain_rel_large_entries_net": float(np.max(np.maximum(dd[big] - allow[big], 0) / np.abs(Dr[big])))}
    assert out["D_net"] <= 1e-5
    return out


def test_error_table_tiny_full(api, handle):
    cat = synth.make(0)
    bins = synth.bins_for(0)
    pr = oracle.pairs.forest_pairs(cat, bins)
    ref = oracle.xi.xi_sums(cat, bins, pr, eps_edge=EPS, processes=0)
    dc = api.DeviceCatalog.from_host(cat)
    row = {}
    for prec in ("mixed", "fp64"):
        n, w, x = api.lya_xi(handle, dc, bins, prec)
        api.lya_sync_status(handle)
        row[prec] = xi_errors(_np(w), _np(n), _np(x), ref)
    assert row["fp64"]["W_raw"] <= 1e-6 and row["fp64"]["xi_raw"] <= 1e-5
    D, Wd = api.lya_dmat(handle, dc, bins, 1.0, 0)
    api.lya_sync_status(handle)
    rd = oracle.dmat.dmat(cat, bins, pr, processes=0, eps_edge=EPS)
    row["dmat"] = d_errors(_np(D), rd, ref)
    row["dmat"].update(w_errors(_np(Wd), ref))
    TABLE["tiny_200_full"] = row


def _sampled(api, handle, cat, bins, n_pairs, seed, dm_pairs=0, name=""):
    pr = oracle.pairs.forest_pairs(cat, bins)
    rng = np.random.default_rng(seed)
    k = np.sort(rng.choice(len(pr[0]), min(n_pairs, len(pr[0])), replace=False))
    a, b = pr[0][k], pr[1][k]
    dc = api.DeviceCatalog.from_host(cat)
    n, w, x = api.lya_xi_pairs(handle, dc, bins, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), "mixed")
    ref = oracle.xi.xi_sums(cat, bins, (a, b), eps_edge=EPS, processes=0)
    row = {"forest_pairs": int(len(a)), "mixed": xi_errors(_np(w), _np(n), _np(x), ref)}
    if dm_pairs:
        # D of lya_dmat over its own subsample rule: choose p so that about dm_pairs pairs are kept
        p = dm_pairs / len(pr[0])
        D, Wd = api.lya_dmat(handle, dc, bins, p, seed)
        api.lya_sync_status(handle)
        sub = oracle.subsample.subsample(pr, seed, p)
        rd = oracle.dmat.dmat(cat, bins, sub, processes=0, eps_edge=EPS)
        rx = oracle.xi.xi_sums(cat, bins, sub, eps_edge=EPS, processes=0)
        row["dmat"] = d_errors(_np(D), rd, rx)
        row["dmat"].update(w_errors(_np(Wd), rx))
        row["dmat"]["forest_pairs"] = int(len(sub[0]))
    TABLE[name] = row


def test_error_table_sdss_sampled(api, handle):
    _sampled(api, handle, synth.make(1), synth.bins_for(1), 2000, 31, dm_pairs=600, name="sdss_dr16_like_60k_sampled")


def test_error_table_desi_density_sampled(api, handle):
    spec = synth.spec_for(2, seed=2)
    spec.area_deg2 = spec.area_deg2 * 60000 / spec.n_forests
    spec.n_forests = 60000
    _sampled(api, handle, synth.generate(spec), synth.bins_for(2), 1500, 32, dm_pairs=300,
             name="desi_y5_like_density_60k_patch_sampled")


def test_error_table_mock_batch_per_mock(api, handle):
    bins = synth.bins_for(4)
    mocks = []
    for m in range(4):
        c = synth.make(4, seed=m)
        mocks.append(synth.subset(c, np.argsort(-c.dec)[:400]))
    dms = [api.DeviceCatalog.from_host(m) for m in mocks]
    num, wsum, xi = api.lya_xi_batched(handle, dms, bins, "mixed")
    api.lya_sync_status(handle)
    rows = []
    for m in range(4):
        ref = oracle.xi.xi_sums(mocks[m], bins, eps_edge=EPS, processes=0)
        r = xi_errors(_np(wsum[m]), _np(num[m]), _np(xi[m]), ref)
        r["mock"] = m
        rows.append(r)
    TABLE["mock_batch_400_forest_patches_per_mock"] = rows
