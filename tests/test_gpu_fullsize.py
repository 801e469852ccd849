"""The CUDA path at the full workload sizes, checked on sampled outputs.

The oracle cannot evaluate a 60,000- or 600,000-forest catalogue in a test,
so these tests run the library on the full catalogues, in the launch
configuration the bench times (autotuned pair kernel, cached pair list), and
check:

* outputs the oracle computes one by one: the neighbour set of sampled
  forests, xi/W over sampled forest pairs, the gradient at sampled pixels, D
  over a sparse seeded subsample of the full pair list;
* properties that hold at any size: additivity of the pair sums over a split
  of the pair list, D = I for eta = I, the batched launch equal to one launch
  per mock, central differences of L = sum_A c_A xi_A equal to the adjoint,
  the projection removing the continuum tilt (Eq. 2.7) exactly.

Tolerances as in test_gpu_parity (edge allowance eps = 6e-5 bin units for the
FP32 separations of the mixed path).
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


def _np(t):
    return t.detach().cpu().numpy()


def _gpu_pairs(api, handle, dc, bins):
    n = api.lya_pairs_build(handle, dc, bins)
    a, b = api.lya_pairs_get(handle, n)
    return a.long(), b.long()


def _pairs_touching(a, b, forests, n_forests):
    """Rows of the (a, b) list with a or b in `forests` (torch, on device; a
    per-forest flag table, read in slices of 1e8 rows)."""
    flag = torch.zeros(n_forests, dtype=torch.bool, device=a.device)
    flag[torch.as_tensor(np.asarray(forests), device=a.device)] = True
    outa, outb = [], []
    for s in range(0, len(a), 100_000_000):
        aa, bb = a[s:s + 100_000_000], b[s:s + 100_000_000]
        m = flag[aa] | flag[bb]
        outa.append(aa[m])
        outb.append(bb[m])
    return torch.cat(outa), torch.cat(outb)


def _as_set(a, b):
    a = np.asarray(a, dtype=np.int64)
    b = np.asarray(b, dtype=np.int64)
    return set((a << 32 | b).tolist())


def _check_w_sampled(api, handle, dc, cat, bins, a, b):
    """xi/W of the library (mixed path) over explicit pairs against the oracle."""
    num, wsum, xi = api.lya_xi_pairs(handle, dc, bins, torch.from_numpy(a).cuda(),
                                     torch.from_numpy(b).cuda(), "mixed")
    api.lya_sync_status(handle)
    ref = oracle.xi.xi_sums(cat, bins, (a, b), eps_edge=EPS_EDGE)
    dW = np.abs(_np(wsum) - ref["wsum"])
    assert np.all(dW <= 1e-6 * ref["wsum"] + ref["edge_w"] + 1e-9)
    dN = np.abs(_np(num) - ref["num"])
    assert np.all(dN <= 1e-5 * np.sqrt(ref["num_sq"]) + ref["edge_n"] + 1e-9)
    assert ref["count"].sum() > 1e6
    return ref


# --------------------------------------------------------------- SDSS-DR16-like, 60,000 forests
@pytest.fixture(scope="module")
def sdss(api):
    cat = synth.make(1)
    bins = synth.bins_for(1)
    return cat, bins, api.DeviceCatalog.from_host(cat)


@pytest.fixture(scope="module")
def sdss_pairs(sdss):
    cat, bins, _ = sdss
    return oracle.pairs.forest_pairs(cat, bins)


def test_sdss_full_pair_list_equals_oracle(api, handle, sdss, sdss_pairs):
    cat, bins, dc = sdss
    a, b = _gpu_pairs(api, handle, dc, bins)
    ra, rb = sdss_pairs
    assert len(a) == len(ra) > 1e7
    ga = np.minimum(_np(a), _np(b))
    gb = np.maximum(_np(a), _np(b))
    order = np.lexsort((gb, ga))
    np.testing.assert_array_equal(ga[order], ra)
    np.testing.assert_array_equal(gb[order], rb)


def test_sdss_full_xi_sampled_pairs_and_additivity(api, handle, sdss, sdss_pairs):
    cat, bins, dc = sdss
    api.lya_autotune(handle, dc, bins)
    num, wsum, xi = api.lya_xi(handle, dc, bins, "mixed")
    api.lya_sync_status(handle)
    # sampled forest pairs against the oracle
    ra, rb = sdss_pairs
    k = np.random.default_rng(21).choice(len(ra), 3000, replace=False)
    _check_w_sampled(api, handle, dc, cat, bins, ra[k], rb[k])
    # the full sums are additive over a split of the pair list
    a, b = _gpu_pairs(api, handle, dc, bins)
    part = torch.from_numpy(np.random.default_rng(22).integers(0, 3, len(a))).cuda()
    tot_n = torch.zeros_like(num)
    tot_w = torch.zeros_like(wsum)
    for q in range(3):
        m = part == q
        n_q, w_q, _ = api.lya_xi_pairs(handle, dc, bins, a[m], b[m], "mixed")
        tot_n += n_q
        tot_w += w_q
    api.lya_sync_status(handle)
    np.testing.assert_allclose(_np(tot_w), _np(wsum), rtol=1e-9, atol=1e-6)
    scale = np.sqrt(np.maximum(_np(wsum), 1.0)) * 1e-9 * float(np.abs(_np(num)).max() + 1)
    assert np.all(np.abs(_np(tot_n) - _np(num)) <= 1e-9 * np.abs(_np(num)) + scale)
    # xi is finite and zero exactly where W is
    x = _np(xi)
    assert np.all(np.isfinite(x)) and np.all(x[_np(wsum) == 0] == 0)


def test_sdss_full_dmat(api, handle, sdss, sdss_pairs):
    cat, bins, dc = sdss
    # eta = I on the bench's 5% subsample: D = I on the filled bins
    D, Wd = api.lya_dmat(handle, dc, bins, 0.05, 1234, eta="identity")
    Dn, Wn = _np(D), _np(Wd)
    on = Wn > 0
    assert on.sum() > 0.9 * bins.nbins
    assert np.abs(Dn[np.ix_(on, on)] - np.eye(on.sum())).max() <= 2e-6
    del D
    # W of D on the 5% subsample equals the xi weights of the same forest pairs
    ra, rb = sdss_pairs
    sa, sb = oracle.subsample.subsample((ra, rb), 1234, 0.05)
    _, wsub, _ = api.lya_xi_pairs(handle, dc, bins, torch.from_numpy(sa).cuda(), torch.from_numpy(sb).cuda(),
                                  "mixed")
    _, Wd2 = api.lya_dmat(handle, dc, bins, 0.05, 1234)
    # same FP32 binning on both sides: only the summation differs (W bar, 1e-6)
    np.testing.assert_allclose(_np(Wd2), _np(wsub), rtol=1e-6, atol=1e-6)
    # a sparse subsample of the full list against the oracle's closed form
    p, seed = 5e-5, 77
    D, Wd = api.lya_dmat(handle, dc, bins, p, seed)
    api.lya_sync_status(handle)
    sub = oracle.subsample.subsample((ra, rb), seed, p)
    assert 500 < len(sub[0]) < 2000
    ref = oracle.dmat.dmat(cat, bins, sub, processes=0, eps_edge=EPS_EDGE)
    rx = oracle.xi.xi_sums(cat, bins, sub, eps_edge=EPS_EDGE)
    W, E, Dr = rx["wsum"], rx["edge_w"], ref["dmat"]
    rowmax = np.abs(Dr).max(axis=1)
    # |dD_AB| <= (E^D_AB + |D_AB| E^W_A) / (W_A - E^W_A) + 1e-5 max_B |D_AB| (test_gpu_parity)
    den = (W - E)[:, None]
    allow = 1e-5 * rowmax[:, None] + np.divide(ref["edge_d"] + np.abs(Dr) * E[:, None], den,
                                               out=np.zeros_like(Dr), where=den > 0)
    on = W > 0
    Dg, Wg = _np(D), _np(Wd)
    assert np.all((np.abs(Dg - ref["dmat"]) <= allow + 1e-12)[on])
    # a bin the oracle leaves empty can only hold pairs within eps of its edges
    assert np.all(Wg[~on] <= rx["edge_w"][~on] + 1e-9)


# --------------------------------------------------------------- differentiable, 20,000 forests
def test_differentiable_full_backward_sampled_pixels(api, handle):
    cat = synth.make(3)
    bins = synth.bins_for(3)
    dc = api.DeviceCatalog.from_host(cat)
    nb = bins.nbins
    c = np.random.default_rng(303).normal(size=nb)
    # the adjoint's inputs xi and W are given, not recomputed: seeded values
    g = np.random.default_rng(305)
    W = g.uniform(1e5, 1e6, nb)
    X = g.normal(0.0, 1e-2, nb)
    gd, gw = api.lya_xi_backward(handle, dc, bins, torch.from_numpy(c).cuda(), torch.from_numpy(X).cuda(),
                                 torch.from_numpy(W).cuda())
    api.lya_sync_status(handle)
    gd, gw = _np(gd), _np(gw)
    # 64 pixels: 16 in each of 4 forests (the oracle's cost is per forest pair)
    rng = np.random.default_rng(304)
    forests = rng.choice(cat.n_forests, 4, replace=False)
    pix = np.concatenate([cat.offsets[f] + rng.choice(cat.lengths()[f], 16, replace=False) for f in forests])
    ra, rb = oracle.pairs.forest_pairs(cat, bins)
    m = np.isin(ra, forests) | np.isin(rb, forests)
    sub = (ra[m], rb[m])
    fwd = {"num": X * W, "wsum": W, "xi": X}
    gd_ref, gw_ref, info = oracle.adjoint.xi_grad(cat, bins, c, sub, absolute=True, eps_edge=EPS_EDGE, fwd=fwd)
    e1 = np.abs(gd[pix] - gd_ref[pix])
    e2 = np.abs(gw[pix] - gw_ref[pix])
    assert np.all(e1 <= 1e-5 * info["grad_delta_abs"][pix] + info["grad_delta_edge"][pix] + 1e-12)
    assert np.all(e2 <= 1e-5 * info["grad_weight_abs"][pix] + info["grad_weight_edge"][pix] + 1e-12)
    assert np.abs(gd_ref[pix]).max() > 0
    # central differences, h = 1e-3: delta_i only enters the numerators of the
    # pairs of its own forest, so L(+h) - L(-h) = sum_A c_A (N+_A - N-_A) / W_A
    # over those pairs (W does not depend on delta)
    h = 1e-3
    for f, base in zip(forests, range(0, 64, 16)):
        fa = torch.from_numpy(sub[0][(sub[0] == f) | (sub[1] == f)]).cuda()
        fb = torch.from_numpy(sub[1][(sub[0] == f) | (sub[1] == f)]).cuda()
        for i in pix[base:base + 16]:
            vals = []
            for sgn in (1.0, -1.0):
                d = dc.delta.clone()
                d[int(i)] += sgn * h
                n_, _, _ = api.lya_xi_pairs(handle, dc.with_(delta=d), bins, fa, fb, "mixed")
                vals.append(_np(n_))
            fd = float(np.dot(c / W, (vals[0] - vals[1]) / (2 * h)))
            assert abs(fd - gd[i]) <= 1e-4 * info["grad_delta_abs"][i] + 1e-9, (i, fd, gd[i])


# --------------------------------------------------------------- mock batch, 15,000 forests per mock
def test_mock_batch_full_mocks(api, handle):
    bins = synth.bins_for(4)
    mocks = [synth.make(4, seed=m) for m in range(6)]
    dms = [api.DeviceCatalog.from_host(m) for m in mocks]
    num, wsum, xi = api.lya_xi_batched(handle, dms, bins, "mixed")
    api.lya_sync_status(handle)
    Wb = _np(wsum).copy()
    Nb = _np(num).copy()
    for m in (0, 5):
        n1, w1, _ = api.lya_xi(handle, dms[m], bins, "mixed")
        np.testing.assert_allclose(Wb[m], _np(w1), rtol=1e-9, atol=1e-6)
        np.testing.assert_allclose(Nb[m], _np(n1), rtol=1e-7, atol=1e-6 * np.abs(Nb[m]).max())
        ra, rb = oracle.pairs.forest_pairs(mocks[m], bins)
        k = np.random.default_rng(40 + m).choice(len(ra), 800, replace=False)
        _check_w_sampled(api, handle, dms[m], mocks[m], bins, ra[k], rb[k])
    # independent mocks differ
    assert not np.allclose(Nb[0], Nb[1])


# --------------------------------------------------------------- DESI-Y5-like, 600,000 forests
def test_desi_full_neighbours_projection_and_sampled_pairs(api, handle):
    spec = synth.spec_for(2)
    cat = synth.generate(spec, name="desi")
    bins = synth.bins_for(2)
    dc = api.DeviceCatalog.from_host(cat)
    rng = np.random.default_rng(60)
    # projection of the whole catalogue; sampled forests against the oracle
    dp = api.lya_project(handle, dc)
    api.lya_sync_status(handle)
    fs = np.sort(rng.choice(cat.n_forests, 2000, replace=False))
    sub = synth.subset(cat, fs)
    idx = np.concatenate([np.arange(cat.offsets[f], cat.offsets[f + 1]) for f in fs])
    ref = oracle.project.project(sub)
    got = _np(dp)[idx]
    np.testing.assert_allclose(got, ref, atol=2e-6 * np.abs(ref).max() + 1e-7)
    # the continuum tilt is removed exactly: the untilted draw projects to the same deltas
    spec0 = synth.spec_for(2)
    spec0.tilt = False
    flat = synth.generate(spec0, name="desi-flat")
    dp0 = api.lya_project(handle, dc.with_(delta=torch.from_numpy(flat.delta).cuda()))
    api.lya_sync_status(handle)
    assert float((dp - dp0).abs().max()) <= 2e-5 * float(dp.abs().max())
    del flat, dp0
    # neighbour sets of sampled forests against a k-d tree query of the oracle
    dcp = dc.with_(delta=dp)
    a, b = _gpu_pairs(api, handle, dcp, bins)
    assert len(a) > 1e8
    q = np.sort(rng.choice(cat.n_forests, 300, replace=False))
    sa, sb = _pairs_touching(a, b, q, cat.n_forests)
    got = _as_set(np.minimum(_np(sa), _np(sb)), np.maximum(_np(sa), _np(sb)))
    from scipy.spatial import cKDTree
    nvec = oracle.geometry.unit_vectors(cat.ra, cat.dec)
    th = oracle.pairs.theta_max(cat, bins)
    tree = cKDTree(nvec)
    cand = tree.query_ball_point(nvec[q], 2.0 * np.sin(0.5 * th) * (1 + 1e-9))
    ea, eb = [], []
    for f, nbrs in zip(q, cand):
        nbrs = np.asarray([x for x in nbrs if x != f], dtype=np.int64)
        ea.append(np.minimum(f, nbrs))
        eb.append(np.maximum(f, nbrs))
    ea, eb = np.concatenate(ea), np.concatenate(eb)
    keep = oracle.pairs._exact_keep(nvec[ea], nvec[eb], oracle.pairs.forest_dmin(cat)[ea],
                                    oracle.pairs.forest_dmin(cat)[eb], bins.r_perp_max)
    exp = _as_set(ea[keep], eb[keep])
    assert got == exp
    # xi/W over 1500 sampled pairs of those forests, on the projected deltas
    lst = np.array(sorted(exp), dtype=np.int64)
    k = rng.choice(len(lst), 1500, replace=False)
    pa, pb = (lst[k] >> 32), (lst[k] & 0xFFFFFFFF)
    catp = synth.Catalog(**{**cat.__dict__, "delta": _np(dp)})
    _check_w_sampled(api, handle, dcp, catp, bins, pa, pb)
