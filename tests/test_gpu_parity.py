"""CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances (from the workload's 1e-6 / 1e-5 bars and the FP32 error bound of
the mixed path's scaled separations):
* FP64 path: |dW_A| <= 1e-6 W_A, |dxi_A| <= 1e-5 max(|xi_A|, sigma_A).
* Mixed path: the same plus the oracle's edge mass for eps = 6e-5 bin units,
  the bound on the FP32 error of the scaled separations: E^W for W, E^N for
  N, and for xi = N / W the quotient's (E^N + |xi| E^W) / (W - E^W).
* D = D~ / W^DM: with |dD~_AB| <= E^D_AB (the oracle's edge_d: what pixel
  pairs within eps of an edge can move into or out of row A or column B) and
  |dW_A| <= E^W_A, D_AB + dD_AB = (D~_AB + dD~_AB) / (W_A + dW_A) gives
  |dD_AB| <= (E^D_AB + |D_AB| E^W_A) / (W_A - E^W_A); beyond it the FP32
  products, 1e-5 max_B |D_AB|.  W^DM is held to the W bar, 1e-6 W + E^W.
* Gradients: |dg_i| <= 1e-5 sum_j |term_ij| + the oracle's edge allowance.
"""
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


@pytest.fixture(scope="module")
def c0():
    cat = synth.make(0)
    bins = synth.bins_for(0)
    pr = oracle.pairs.forest_pairs(cat, bins)
    return cat, bins, pr


@pytest.fixture(scope="module")
def ref0(c0):
    cat, bins, pr = c0
    return oracle.xi.xi_sums(cat, bins, pr, eps_edge=EPS_EDGE, processes=0)


def _np(t):
    return t.detach().cpu().numpy()


def _xi_allowance(ref):
    """Mixed-path bound on |dxi_A|: 1e-5 max(|xi_A|, sigma_A), plus what the
    edge pixel pairs can move.  xi = N / W, so flips that change N by dN and W
    by dW change xi by (dN - xi dW) / (W + dW); with |dN| <= E^N, |dW| <= E^W
    that is at most (E^N + |xi| E^W) / (W - E^W), unbounded where every pair
    of the bin is an edge pair."""
    den = ref["wsum"] - ref["edge_w"]
    edge = np.divide(ref["edge_n"] + np.abs(ref["xi"]) * ref["edge_w"], den, out=np.full_like(den, np.inf),
                     where=den > 0)
    return 1e-5 * np.maximum(np.abs(ref["xi"]), ref["sigma"]) + edge


# ------------------------------------------------------------------ pair list
def test_pair_list_equals_oracle(api, handle, c0):
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    n = api.lya_pairs_build(handle, dc, bins)
    a, b = api.lya_pairs_get(handle, n)
    got = np.stack([_np(a), _np(b)], 1).astype(np.int64)
    assert np.all(got[:, 0] < got[:, 1])
    got = got[np.lexsort((got[:, 1], got[:, 0]))]
    exp = np.stack(pr, 1)
    np.testing.assert_array_equal(got, exp)


# ------------------------------------------------------------------ xi, W
def test_xi_fp64_matches_oracle(api, handle, c0, ref0):
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    num, wsum, xi = api.lya_xi(handle, dc, bins, "fp64")
    api.lya_sync_status(handle)
    W, N, X = _np(wsum), _np(num), _np(xi)
    assert np.all(np.abs(W - ref0["wsum"]) <= 1e-6 * ref0["wsum"] + 1e-12)
    assert np.all(np.abs(X - ref0["xi"]) <= 1e-5 * np.maximum(np.abs(ref0["xi"]), ref0["sigma"]) + 1e-15)
    assert np.all(np.abs(N - ref0["num"]) <= 1e-5 * np.sqrt(ref0["num_sq"]) + 1e-12)
    assert ref0["count"].sum() > 5e7


def test_xi_mixed_matches_oracle_within_edge_allowance(api, handle, c0, ref0):
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    num, wsum, xi = api.lya_xi(handle, dc, bins, "mixed")
    api.lya_sync_status(handle)
    W, N, X = _np(wsum), _np(num), _np(xi)
    dW = np.abs(W - ref0["wsum"])
    assert np.all(dW <= 1e-6 * ref0["wsum"] + ref0["edge_w"] + 1e-9)
    assert np.all(np.abs(N - ref0["num"]) <= 1e-5 * np.sqrt(ref0["num_sq"]) + ref0["edge_n"] + 1e-9)
    on = ref0["wsum"] > 0
    allow = _xi_allowance(ref0)
    assert np.all(np.abs(X - ref0["xi"])[on] <= allow[on] + 1e-15)
    # the flips are rare: the total moved weight is far below the allowance
    assert dW.sum() <= 0.05 * ref0["edge_w"].sum() + 1e-6 * ref0["wsum"].sum()


def test_xi_wide_bands_in_windows_match_oracle(api, handle, c0):
    """r_perp bins of 1/3 Mpc/h: a forest pair's r_perp band then spans more rows than the pair kernels hold at
    once (14 rows of 25 r_par bins in the mixed kernel, 10 in the FP64 one), so they take such pairs in windows
    of rows, each window a pass over the pair.  Here r_perp / D_perp reaches 300, so three of the FP32 roundings in
    the scaled r_perp are of values up to 300 (1.5e-5 each) and the rounding of s / D_perp adds 1.8e-5: the bound
    on its error is ~6.6e-5 bin units, and the edge mass is taken at eps = 1e-4."""
    cat, _, _ = c0
    bins = synth.Bins(25, 300, 100.0, 100.0)
    pr = oracle.pairs.forest_pairs(cat, bins)
    # band rows of each pair, from its forests' extreme distances (r_perp grows with both distances)
    from oracle.geometry import unit_vectors
    nv = unit_vectors(cat.ra, cat.dec)
    a, b = pr
    s = 0.5 * np.linalg.norm(nv[a] - nv[b], axis=1) / (bins.r_perp_max / bins.n_perp)
    lo = np.floor((cat.dist[cat.offsets[a]] + cat.dist[cat.offsets[b]]) * s)
    hi = np.minimum(np.floor((cat.dist[cat.offsets[a + 1] - 1] + cat.dist[cat.offsets[b + 1] - 1]) * s),
                    bins.n_perp - 1)
    rows = (hi - lo + 1)[lo < bins.n_perp]
    assert np.mean(rows > 14) > 0.5 and np.mean(rows > 10) > 0.7
    ref = oracle.xi.xi_sums(cat, bins, pr, eps_edge=1e-4, processes=0)
    dc = api.DeviceCatalog.from_host(cat)
    on = ref["wsum"] > 0
    num, wsum, xi = api.lya_xi(handle, dc, bins, "fp64")
    api.lya_sync_status(handle)
    W, N, X = _np(wsum), _np(num), _np(xi)
    assert np.all(np.abs(W - ref["wsum"]) <= 1e-6 * ref["wsum"] + 1e-12)
    assert np.all(np.abs(X - ref["xi"]) <= 1e-5 * np.maximum(np.abs(ref["xi"]), ref["sigma"]) + 1e-15)
    num, wsum, xi = api.lya_xi(handle, dc, bins, "mixed")
    api.lya_sync_status(handle)
    W, N, X = _np(wsum), _np(num), _np(xi)
    assert np.all(np.abs(W - ref["wsum"]) <= 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9)
    assert np.all(np.abs(N - ref["num"]) <= 1e-5 * np.sqrt(ref["num_sq"]) + ref["edge_n"] + 1e-9)
    allow = _xi_allowance(ref)
    assert np.all(np.abs(X - ref["xi"])[on] <= allow[on] + 1e-15)
    assert np.all(X[~on] == 0)


def test_flip_tally_is_bounded_by_edge_mass(api, handle, c0, ref0):
    """The pixel pairs whose FP32 bin differs from their FP64 bin carry at most
    the oracle's edge mass for eps = 6e-5; the FP64 in-grid count is the
    oracle's, and the mixed and FP64 weights differ by at most the flipped
    weight moved out of one bin and into another."""
    cat, bins, _ = c0
    dc = api.DeviceCatalog.from_host(cat)
    t = api.lya_flip_tally(handle, dc, bins, 1.0)
    n_ref = float(ref0["count"].sum())
    assert abs(t["pixel_pairs"] - n_ref) <= 1e-6 * n_ref
    np.testing.assert_allclose(t["weight"], ref0["wsum"].sum(), rtol=1e-6)
    assert 0 <= t["flipped_weight"] <= ref0["edge_w"].sum() + 1e-9
    assert t["flipped"] <= 1e-3 * t["pixel_pairs"]
    _, w_mixed, _ = api.lya_xi(handle, dc, bins, "mixed")
    _, w_fp64, _ = api.lya_xi(handle, dc, bins, "fp64")
    moved = float(np.abs(_np(w_mixed) - _np(w_fp64)).sum())
    assert moved <= 2 * t["flipped_weight"] + 1e-9 * float(_np(w_fp64).sum())


def test_xi_pairs_subset_equals_oracle(api, handle, c0):
    cat, bins, pr = c0
    rng = np.random.default_rng(11)
    k = rng.choice(len(pr[0]), 700, replace=False)
    a, b = pr[0][k], pr[1][k]
    # give half of the pairs in reversed order: the estimator is symmetric
    a2 = np.where(np.arange(700) % 2 == 0, a, b)
    b2 = np.where(np.arange(700) % 2 == 0, b, a)
    dc = api.DeviceCatalog.from_host(cat)
    num, wsum, xi = api.lya_xi_pairs(handle, dc, bins, torch.from_numpy(a2).cuda(),
                                     torch.from_numpy(b2).cuda(), "fp64")
    ref = oracle.xi.xi_sums(cat, bins, (a, b))
    np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-6, atol=1e-9)


def test_xi_is_invariant_to_forest_order(api, handle, c0):
    cat, bins, _ = c0
    perm = np.random.default_rng(5).permutation(cat.n_forests)
    cat2 = synth.subset(cat, perm)
    _, w1, x1 = api.lya_xi(handle, api.DeviceCatalog.from_host(cat), bins, "fp64")
    _, w2, x2 = api.lya_xi(handle, api.DeviceCatalog.from_host(cat2), bins, "fp64")
    np.testing.assert_allclose(_np(w2), _np(w1), rtol=1e-12)
    np.testing.assert_allclose(_np(x2), _np(x1), rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------ projection
def test_projection_matches_oracle(api, handle):
    cat = synth.make(2, n_forests=400)
    dc = api.DeviceCatalog.from_host(cat)
    out = api.lya_project(handle, dc)
    api.lya_sync_status(handle)
    ref = oracle.project.project(cat)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(_np(out), ref, atol=2e-6 * scale + 1e-7)
    # in place
    d2 = dc.delta.clone()
    api.lya_project(handle, dc.with_(delta=d2), out=d2)
    np.testing.assert_array_equal(_np(d2), _np(out))


# ------------------------------------------------------------------ distortion matrix
def _d_allowance(ref_xi, ref_d):
    """1e-5 of the row maximum, plus the effect of pixel pairs within the FP32
    separation error of an edge on the quotient D~_AB / W_A (module docstring):
    (E^D_AB + |D_AB| E^W_A) / (W_A - E^W_A)."""
    W = ref_xi["wsum"]
    E = ref_xi["edge_w"]
    D = ref_d["dmat"]
    rowmax = np.abs(D).max(axis=1)
    den = (W - E)[:, None]
    edge = np.divide(ref_d["edge_d"] + np.abs(D) * E[:, None], den, out=np.zeros_like(D), where=den > 0)
    return 1e-5 * rowmax[:, None] + edge


def test_dmat_matches_oracle(api, handle, c0, ref0):
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    D, Wd = api.lya_dmat(handle, dc, bins, 1.0, 0)
    api.lya_sync_status(handle)
    ref = oracle.dmat.dmat(cat, bins, pr, processes=0, eps_edge=EPS_EDGE)
    Dg = _np(D)
    assert np.all(np.abs(Dg - ref["dmat"]) <= _d_allowance(ref0, ref) + 1e-12)
    assert np.all(np.abs(_np(Wd) - ref0["wsum"]) <= 1e-6 * ref0["wsum"] + ref0["edge_w"] + 1e-9)


def test_dmat_tensor_core_tiles_match_oracle(api, c0, ref0):
    """The TF32x3 tensor-core form of the rank-1 tiles meets the same bars as
    the FP32 form: D against the oracle, W^DM at the W bar."""
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    with api.Handle() as h:
        api.lya_set_dmat_tiles(h, "tf32x3")
        D, Wd = api.lya_dmat(h, dc, bins, 1.0, 0)
        api.lya_sync_status(h)
        api.lya_set_dmat_tiles(h, "fp32")
        D32, _ = api.lya_dmat(h, dc, bins, 1.0, 0)
    ref = oracle.dmat.dmat(cat, bins, pr, processes=0, eps_edge=EPS_EDGE)
    assert np.all(np.abs(_np(D) - ref["dmat"]) <= _d_allowance(ref0, ref) + 1e-12)
    assert np.all(np.abs(_np(Wd) - ref0["wsum"]) <= 1e-6 * ref0["wsum"] + ref0["edge_w"] + 1e-9)
    # the two tile forms differ only by rounding: both lie within the oracle's allowance
    assert np.all(np.abs(_np(D32) - ref["dmat"]) <= _d_allowance(ref0, ref) + 1e-12)
    assert np.all(np.abs(_np(D) - _np(D32)) <= 2 * _d_allowance(ref0, ref) + 1e-12)


def test_dmat_identity_eta(api, handle, c0):
    cat, bins, pr = c0
    dc = api.DeviceCatalog.from_host(cat)
    D, Wd = api.lya_dmat(handle, dc, bins, 1.0, 0, eta="identity")
    Dg, W = _np(D), _np(Wd)
    on = W > 0
    np.testing.assert_allclose(Dg[np.ix_(on, on)], np.eye(on.sum()), atol=2e-6)
    assert np.all(Dg[~on] == 0)


def test_dmat_subsample_matches_oracle(api, handle, c0):
    cat, bins, pr = c0
    seed, p = 12345, 0.3
    dc = api.DeviceCatalog.from_host(cat)
    D, Wd = api.lya_dmat(handle, dc, bins, p, seed)
    sub = oracle.subsample.subsample(pr, seed, p)
    assert 0.2 * len(pr[0]) < len(sub[0]) < 0.4 * len(pr[0])
    ref = oracle.dmat.dmat(cat, bins, sub, processes=0, eps_edge=EPS_EDGE)
    rx = oracle.xi.xi_sums(cat, bins, sub, eps_edge=EPS_EDGE)
    assert np.all(np.abs(_np(D) - ref["dmat"]) <= _d_allowance(rx, ref) + 1e-12)
    assert np.all(np.abs(_np(Wd) - rx["wsum"]) <= 1e-6 * rx["wsum"] + rx["edge_w"] + 1e-9)


def test_dmat_work_counts_match_oracle(api, handle, c0):
    """The closed form's work counts (the D roofline's flops) against the
    oracle's, on a seeded 30% subsample: in-grid pixel pairs up to the rare FP32
    edge flips, and the sums of squared supports to 1e-3."""
    cat, bins, pr = c0
    seed, p = 12345, 0.3
    got = api.lya_dmat_work(handle, api.DeviceCatalog.from_host(cat), bins, p, seed)
    sub = oracle.subsample.subsample(pr, seed, p)
    ref = oracle.dmat.closed_form_work(cat, bins, sub)
    assert abs(got["pixel_pairs"] - ref["pixel_pairs"]) <= 1e-4 * ref["pixel_pairs"]
    for k in ("sum_vec_support_sq", "sum_pair_support_sq", "flops"):
        assert got[k] == pytest.approx(ref[k], rel=1e-3), k


def test_dmat_zero_fraction(api, handle, c0):
    cat, bins, _ = c0
    D, W = api.lya_dmat(handle, api.DeviceCatalog.from_host(cat), bins, 0.0, 1)
    assert float(D.abs().max()) == 0.0 and float(W.abs().max()) == 0.0


# ------------------------------------------------------------------ adjoint
@pytest.fixture(scope="module")
def small3():
    cat = synth.make(3, n_forests=600)
    bins = synth.bins_for(3)
    return cat, bins, oracle.pairs.forest_pairs(cat, bins)


def test_backward_matches_oracle(api, handle, small3):
    cat, bins, pr = small3
    c = np.random.default_rng(303).normal(size=bins.nbins)
    fwd = oracle.xi.xi_sums(cat, bins, pr)
    gd_ref, gw_ref, info = oracle.adjoint.xi_grad(cat, bins, c, pr, absolute=True, eps_edge=EPS_EDGE,
                                                  fwd=fwd)
    dc = api.DeviceCatalog.from_host(cat)
    # feed the oracle's forward sums so that only the backward binning differs
    gd, gw = api.lya_xi_backward(handle, dc, bins, torch.from_numpy(c).cuda(),
                                 torch.from_numpy(fwd["xi"]).cuda(), torch.from_numpy(fwd["wsum"]).cuda())
    api.lya_sync_status(handle)
    e1 = np.abs(_np(gd) - gd_ref)
    e2 = np.abs(_np(gw) - gw_ref)
    assert np.all(e1 <= 1e-5 * info["grad_delta_abs"] + info["grad_delta_edge"] + 1e-12)
    assert np.all(e2 <= 1e-5 * info["grad_weight_abs"] + info["grad_weight_edge"] + 1e-12)
    assert np.abs(gd_ref).max() > 0


def test_autograd_function_and_fd(api, handle, small3):
    """torch.autograd through XiFunction; central differences of the GPU FP64
    forward on 16 pixels against the backward."""
    cat, bins, pr = small3
    dc = api.DeviceCatalog.from_host(cat)
    c = torch.from_numpy(np.random.default_rng(303).normal(size=bins.nbins)).cuda()
    d = dc.delta.clone().requires_grad_(True)
    w = dc.weight.clone().requires_grad_(True)
    x, W = api.xi(dc, bins, handle, delta=d, weight=w)
    (x * c).sum().backward()
    fwd = oracle.xi.xi_sums(cat, bins, pr)
    _, _, info = oracle.adjoint.xi_grad(cat, bins, c.cpu().numpy(), pr, absolute=True,
                                        eps_edge=EPS_EDGE, fwd=fwd)
    rng = np.random.default_rng(304)
    for i in rng.choice(cat.n_pix, 16, replace=False):
        h = 0.37
        vals = []
        for sgn in (1, -1):
            dd = dc.delta.clone()
            dd[i] += sgn * h
            _, _, xx = api.lya_xi(handle, dc.with_(delta=dd), bins, "fp64")
            vals.append(float((xx * c).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        g = float(d.grad[i])
        assert abs(fd - g) <= 1e-4 * info["grad_delta_abs"][i] + 3 * info["grad_delta_edge"][i] + 1e-9


def test_autograd_weight_sum_gradient_matches_oracle(api, handle, small3):
    """A loss that uses both outputs, L = sum c_A xi_A + sum e_A W_A, through
    XiFunction: dL/dw carries the weight sum's own term sum_j e_A w_j (the
    oracle's gradient, pinned by central differences)."""
    cat, bins, pr = small3
    dc = api.DeviceCatalog.from_host(cat)
    c = np.random.default_rng(303).normal(size=bins.nbins)
    e = np.random.default_rng(306).normal(size=bins.nbins) * 1e-4
    d = dc.delta.clone().requires_grad_(True)
    w = dc.weight.clone().requires_grad_(True)
    x, W = api.xi(dc, bins, handle, delta=d, weight=w)
    ((x * torch.from_numpy(c).cuda()).sum() + (W * torch.from_numpy(e).cuda()).sum()).backward()
    fwd = oracle.xi.xi_sums(cat, bins, pr)
    gd_ref, gw_ref, info = oracle.adjoint.xi_grad(cat, bins, c, pr, absolute=True, eps_edge=EPS_EDGE,
                                                  fwd=fwd, grad_wsum=e)
    # the forward W of the mixed path differs from the oracle's only by edge
    # flips; the backward is checked with the oracle's gamma / rho inputs
    gd2, gw2 = api.lya_xi_backward_full(handle, dc, bins, torch.from_numpy(c).cuda(), torch.from_numpy(e).cuda(),
                                        torch.from_numpy(fwd["xi"]).cuda(), torch.from_numpy(fwd["wsum"]).cuda())
    api.lya_sync_status(handle)
    assert np.all(np.abs(_np(gd2) - gd_ref) <= 1e-5 * info["grad_delta_abs"] + info["grad_delta_edge"] + 1e-12)
    assert np.all(np.abs(_np(gw2) - gw_ref) <= 1e-5 * info["grad_weight_abs"] + info["grad_weight_edge"] + 1e-12)
    # autograd runs the same entry point on its own forward outputs
    gd3, gw3 = api.lya_xi_backward_full(handle, dc, bins, torch.from_numpy(c).cuda(), torch.from_numpy(e).cuda(),
                                        x.detach(), W.detach())
    np.testing.assert_array_equal(_np(w.grad), _np(gw3))
    np.testing.assert_array_equal(_np(d.grad), _np(gd3))
    # and the W term is really there
    _, gw0 = api.lya_xi_backward(handle, dc, bins, torch.from_numpy(c).cuda(), x.detach(), W.detach())
    assert np.abs(_np(gw3) - _np(gw0)).max() > 1e-3 * np.abs(_np(gw0)).max()


# ------------------------------------------------------------------ batching
def test_batched_equals_single(api, handle):
    bins = synth.bins_for(4)
    mocks = [synth.make(4, seed=m, n_forests=300) for m in range(3)]
    dms = [api.DeviceCatalog.from_host(m) for m in mocks]
    num, wsum, xi = api.lya_xi_batched(handle, dms, bins, "mixed")
    for m in range(3):
        n1, w1, x1 = api.lya_xi(handle, dms[m], bins, "mixed")
        np.testing.assert_allclose(_np(wsum[m]), _np(w1), rtol=1e-12, atol=1e-9)
        ref = oracle.xi.xi_sums(mocks[m], bins, eps_edge=EPS_EDGE)
        dw = np.abs(_np(wsum[m]) - ref["wsum"])
        allow = 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9
        bad = np.nonzero(dw > allow)[0]
        assert len(bad) == 0, [(int(k), float(dw[k]), float(ref["wsum"][k]), float(ref["edge_w"][k]))
                               for k in bad[:10]]


def test_dmat_batched_equals_single(api, handle):
    """D of three mocks in one launch equals D of each mock alone (same seed;
    the subsample rule uses mock-local forest indices), to the FP32 chunk sums'
    rounding; W^DM likewise, at the W bar.  One mock against the oracle."""
    bins = synth.bins_for(4)
    mocks = [synth.make(4, seed=m, n_forests=250) for m in range(3)]
    dms = [api.DeviceCatalog.from_host(m) for m in mocks]
    p, seed = 0.3, 77
    D, W = api.lya_dmat_batched(handle, dms, bins, p, seed)
    api.lya_sync_status(handle)
    Db, Wb = _np(D).copy(), _np(W).copy()
    for m in range(3):
        D1, W1 = api.lya_dmat(handle, dms[m], bins, p, seed)
        d1 = _np(D1)
        np.testing.assert_allclose(Wb[m], _np(W1), rtol=1e-6, atol=1e-9)
        assert np.all(np.abs(Db[m] - d1) <= 1e-5 * np.abs(d1).max(axis=1, keepdims=True) + 1e-12)
        assert np.abs(d1).max() > 0.5
    assert not np.allclose(Db[0], Db[1])
    pr = oracle.pairs.forest_pairs(mocks[2], bins)
    sub = oracle.subsample.subsample(pr, seed, p)
    ref = oracle.dmat.dmat(mocks[2], bins, sub, processes=0, eps_edge=EPS_EDGE)
    rx = oracle.xi.xi_sums(mocks[2], bins, sub, eps_edge=EPS_EDGE)
    assert np.all(np.abs(Db[2] - ref["dmat"]) <= _d_allowance(rx, ref) + 1e-12)
    assert np.all(np.abs(Wb[2] - rx["wsum"]) <= 1e-6 * rx["wsum"] + rx["edge_w"] + 1e-9)


# ------------------------------------------------------------------ edge cases and errors
def test_degenerate_catalogues(api, handle):
    from conftest import line_catalog
    bins = synth.Bins(4, 4, 16.0, 16.0)
    # single-pixel forests, a zero-weight forest, an empty forest, an isolated forest
    fs = [(0.0, 0.0, [1000.0], [8.2], [0.5], [1.0]),
          (1e-4, 0.0, [1001.0], [8.2], [-0.5], [2.0]),
          (2e-4, 0.0, [1000.5, 1002.0], [8.2, 8.3], [0.1, 0.2], [0.0, 0.0]),
          (3e-4, 0.0, [], [], [], []),
          (1.0, 0.5, [1000.0, 1003.0], [8.2, 8.3], [0.3, 0.1], [1.0, 1.0])]
    cat = line_catalog(fs)
    dc = api.DeviceCatalog.from_host(cat)
    ref = oracle.xi.xi_sums(cat, bins, oracle.pairs.all_pairs(cat.n_forests))
    for prec in ("fp64", "mixed"):
        num, wsum, xi = api.lya_xi(handle, dc, bins, prec)
        api.lya_sync_status(handle)
        np.testing.assert_allclose(_np(wsum), ref["wsum"], rtol=1e-6, atol=1e-12)
        np.testing.assert_allclose(_np(xi), ref["xi"], rtol=1e-5, atol=1e-12)


def test_empty_catalogue(api, handle):
    from conftest import line_catalog
    bins = synth.Bins(4, 4, 16.0, 16.0)
    cat = line_catalog([(0.0, 0.0, [1000.0, 1001.0], [8.2, 8.3], [0.5, 0.1], [1.0, 1.0])])
    num, wsum, xi = api.lya_xi(handle, api.DeviceCatalog.from_host(cat), bins, "mixed")
    assert float(wsum.abs().sum()) == 0.0 and float(xi.abs().sum()) == 0.0


def test_input_errors_are_reported(api, handle, c0):
    from paper_2507_00129_gb300._lib import LyaError
    cat, bins, _ = c0
    sub = synth.subset(cat, np.arange(20))
    bad = synth.Catalog(**{**sub.__dict__, "dist": sub.dist.copy()})
    bad.dist[5], bad.dist[6] = bad.dist[6], bad.dist[5]
    with pytest.raises(LyaError) as e:
        api.lya_pairs_build(handle, api.DeviceCatalog.from_host(bad), bins)
    assert e.value.code == -2
    nan = synth.Catalog(**{**sub.__dict__, "delta": sub.delta.copy()})
    nan.delta[3] = np.nan
    with pytest.raises(LyaError) as e:
        api.lya_pairs_build(handle, api.DeviceCatalog.from_host(nan), bins)
    assert e.value.code == -3
    off = synth.Catalog(**{**sub.__dict__, "offsets": sub.offsets.copy()})
    off.offsets[-1] += 5
    with pytest.raises(LyaError) as e:
        api.lya_pairs_build(handle, api.DeviceCatalog.from_host(off), bins)
    assert e.value.code == -7
    with pytest.raises(LyaError) as e:
        api.lya_xi(handle, api.DeviceCatalog.from_host(sub), synth.Bins(1000, 4, 10.0, 10.0))
    assert e.value.code == -8
    # within the C-ABI grid limits but beyond the pair kernels' shared-memory layout
    for prec, n_par in (("mixed", 204), ("fp64", 257)):
        with pytest.raises(LyaError) as e:
            api.lya_xi(handle, api.DeviceCatalog.from_host(sub), synth.Bins(n_par, 4, 10.0, 10.0), prec)
        assert e.value.code == -8
    dc = api.DeviceCatalog.from_host(sub)
    api.lya_xi_pairs(handle, dc, bins, torch.tensor([0, 3, 25], dtype=torch.int32).cuda(),
                     torch.tensor([0, 5, 1], dtype=torch.int32).cuda())
    with pytest.raises(LyaError) as e:
        api.lya_sync_status(handle)
    assert e.value.code == -7
    # the handle stays usable
    n = api.lya_pairs_build(handle, dc, bins)
    assert n > 0
