"""Python face of liblya.so: device catalogues, a handle, one function per C
entry point (same names), and a torch.autograd.Function for xi.

PyTorch provides device memory and the current stream; every computation
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from ._lib import LyaBins, LyaCatalog, check

PREC = {"mixed": _lib.LYA_PREC_MIXED, "fp64": _lib.LYA_PREC_FP64}


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class DeviceCatalog:
    """A forest catalogue resident on the GPU (layout of ``lya_catalog``)."""

    def __init__(self, offsets, ra, dec, dist, loglam, delta, weight):
        self.offsets = offsets.contiguous()
        self.ra = ra.contiguous()
        self.dec = dec.contiguous()
        self.dist = dist.contiguous()
        self.loglam = loglam.contiguous()
        self.delta = delta.contiguous()
        self.weight = weight.contiguous()
        assert self.offsets.dtype == torch.int64
        for t in (self.ra, self.dec, self.dist, self.loglam):
            assert t.dtype == torch.float64
        for t in (self.delta, self.weight):
            assert t.dtype == torch.float32

    @property
    def n_forests(self) -> int:
        return int(self.ra.shape[0])

    @property
    def n_pix(self) -> int:
        return int(self.dist.shape[0])

    @classmethod
    def from_host(cls, cat, device="cuda", pin: bool = False) -> "DeviceCatalog":
        def t(a, dt):
            x = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
            if pin:
                x = x.pin_memory()
            return x.to(device, non_blocking=pin)
        return cls(t(cat.offsets, torch.int64), t(cat.ra, torch.float64), t(cat.dec, torch.float64),
                   t(cat.dist, torch.float64), t(cat.loglam, torch.float64), t(cat.delta, torch.float32),
                   t(cat.weight, torch.float32))

    def with_(self, delta=None, weight=None) -> "DeviceCatalog":
        return DeviceCatalog(self.offsets, self.ra, self.dec, self.dist, self.loglam,
                             self.delta if delta is None else delta,
                             self.weight if weight is None else weight)

    def c(self) -> LyaCatalog:
        return LyaCatalog(self.n_forests, self.n_pix, self.offsets.data_ptr(), self.ra.data_ptr(),
                          self.dec.data_ptr(), self.dist.data_ptr(), self.loglam.data_ptr(),
                          self.delta.data_ptr(), self.weight.data_ptr())


def c_bins(bins) -> LyaBins:
    return LyaBins(int(bins.n_par), int(bins.n_perp), float(bins.r_par_max), float(bins.r_perp_max))


class Handle:
    """Owns an ``lya_handle`` (scratch memory, cached pair list)."""

    def __init__(self):
        lib = _lib.load()
        h = ctypes.c_void_p()
        rc = lib.lya_create(ctypes.byref(h))
        if rc != 0:
            raise _lib.LyaError(rc, "lya_create failed (no CUDA device?)")
        self._h = h

    @property
    def h(self):
        return self._h

    def close(self):
        if self._h:
            _lib.load().lya_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---------------------------------------------------------------------------
# one function per C entry point (same names); tensors are CUDA tensors
# ---------------------------------------------------------------------------
def lya_sync_status(handle: Handle, stream=None):
    check(handle.h, _lib.load().lya_sync_status(handle.h, _stream(stream)))


def lya_pairs_build(handle: Handle, cat: DeviceCatalog, bins, stream=None) -> int:
    n = ctypes.c_int64(0)
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_pairs_build(handle.h, ctypes.byref(c), ctypes.byref(b),
                                                ctypes.byref(n), _stream(stream)))
    return int(n.value)


def lya_pairs_get(handle: Handle, n_pairs: int, stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
    a = torch.empty(max(n_pairs, 1), dtype=torch.int32, device="cuda")
    b = torch.empty(max(n_pairs, 1), dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(0)
    check(handle.h, _lib.load().lya_pairs_get(handle.h, _ptr(a), _ptr(b), n_pairs, ctypes.byref(n),
                                              _stream(stream)))
    return a[: n.value], b[: n.value]


def lya_project(handle: Handle, cat: DeviceCatalog, out: Optional[torch.Tensor] = None, stream=None):
    out = torch.empty_like(cat.delta) if out is None else out
    c = cat.c()
    check(handle.h, _lib.load().lya_project(handle.h, ctypes.byref(c), _ptr(out), _stream(stream)))
    return out


def lya_xi(handle: Handle, cat: DeviceCatalog, bins, precision: str = "mixed", num=None, wsum=None,
           xi=None, stream=None):
    nb = bins.n_par * bins.n_perp
    num = torch.empty(nb, dtype=torch.float64, device="cuda") if num is None else num
    wsum = torch.empty(nb, dtype=torch.float64, device="cuda") if wsum is None else wsum
    xi = torch.empty(nb, dtype=torch.float64, device="cuda") if xi is None else xi
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xi(handle.h, ctypes.byref(c), ctypes.byref(b), PREC[precision],
                                       _ptr(num), _ptr(wsum), _ptr(xi), _stream(stream)))
    return num, wsum, xi


def lya_xi_pairs(handle: Handle, cat: DeviceCatalog, bins, pair_a: torch.Tensor, pair_b: torch.Tensor,
                 precision: str = "mixed", stream=None):
    nb = bins.n_par * bins.n_perp
    num = torch.empty(nb, dtype=torch.float64, device="cuda")
    wsum = torch.empty(nb, dtype=torch.float64, device="cuda")
    xi = torch.empty(nb, dtype=torch.float64, device="cuda")
    pa = pair_a.to(torch.int32).contiguous()
    pb = pair_b.to(torch.int32).contiguous()
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xi_pairs(handle.h, ctypes.byref(c), ctypes.byref(b), PREC[precision],
                                             _ptr(pa), _ptr(pb), int(pa.numel()), _ptr(num), _ptr(wsum),
                                             _ptr(xi), _stream(stream)))
    return num, wsum, xi


def lya_xi_pairs_static(cat: DeviceCatalog, bins, pair_a: torch.Tensor, pair_b: torch.Tensor, stream=None):
    """xi/W over explicit pairs using only the library's fixed device array
    (no device allocation inside the library call; no handle)."""
    nb = bins.n_par * bins.n_perp
    num = torch.empty(nb, dtype=torch.float64, device="cuda")
    wsum = torch.empty(nb, dtype=torch.float64, device="cuda")
    xi = torch.empty(nb, dtype=torch.float64, device="cuda")
    pa = pair_a.to(torch.int32).contiguous()
    pb = pair_b.to(torch.int32).contiguous()
    c, b = cat.c(), c_bins(bins)
    check(None, _lib.load().lya_xi_pairs_static(ctypes.byref(c), ctypes.byref(b), _ptr(pa), _ptr(pb),
                                                int(pa.numel()), _ptr(num), _ptr(wsum), _ptr(xi),
                                                _stream(stream)))
    return num, wsum, xi


def lya_dmat(handle: Handle, cat: DeviceCatalog, bins, p_subsample: float, seed: int,
             eta: str = "mean_slope", stream=None, D=None, W=None):
    nb = bins.n_par * bins.n_perp
    D = torch.empty((nb, nb), dtype=torch.float64, device="cuda") if D is None else D
    W = torch.empty(nb, dtype=torch.float64, device="cuda") if W is None else W
    e = _lib.LYA_ETA_MEAN_SLOPE if eta == "mean_slope" else _lib.LYA_ETA_IDENTITY
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_dmat(handle.h, ctypes.byref(c), ctypes.byref(b), e, float(p_subsample),
                                         ctypes.c_uint64(seed), _ptr(D), _ptr(W), _stream(stream)))
    return D, W


def lya_dmat_batched(handle: Handle, mocks: Sequence[DeviceCatalog], bins, p_subsample: float, seed: int,
                     eta: str = "mean_slope", stream=None, D=None, W=None):
    nb = bins.n_par * bins.n_perp
    m = len(mocks)
    D = torch.empty((m, nb, nb), dtype=torch.float64, device="cuda") if D is None else D
    W = torch.empty((m, nb), dtype=torch.float64, device="cuda") if W is None else W
    e = _lib.LYA_ETA_MEAN_SLOPE if eta == "mean_slope" else _lib.LYA_ETA_IDENTITY
    arr = (LyaCatalog * m)(*[c.c() for c in mocks])
    b = c_bins(bins)
    check(handle.h, _lib.load().lya_dmat_batched(handle.h, arr, m, ctypes.byref(b), e, float(p_subsample),
                                                 ctypes.c_uint64(seed), _ptr(D), _ptr(W), _stream(stream)))
    return D, W


def lya_xi_backward(handle: Handle, cat: DeviceCatalog, bins, grad_xi: torch.Tensor, xi: torch.Tensor,
                    wsum: torch.Tensor, stream=None, grad_delta=None, grad_weight=None):
    gd = torch.empty_like(cat.delta) if grad_delta is None else grad_delta
    gw = torch.empty_like(cat.weight) if grad_weight is None else grad_weight
    g = grad_xi.to(torch.float64).contiguous()
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xi_backward(handle.h, ctypes.byref(c), ctypes.byref(b), _ptr(g),
                                                _ptr(xi.contiguous()), _ptr(wsum.contiguous()), _ptr(gd),
                                                _ptr(gw), _stream(stream)))
    return gd, gw


def lya_xi_backward_full(handle: Handle, cat: DeviceCatalog, bins, grad_xi: torch.Tensor,
                         grad_wsum: Optional[torch.Tensor], xi: torch.Tensor, wsum: torch.Tensor, stream=None,
                         grad_delta=None, grad_weight=None):
    """Gradient of sum grad_xi * xi + sum grad_wsum * W (grad_wsum may be None)."""
    gd = torch.empty_like(cat.delta) if grad_delta is None else grad_delta
    gw = torch.empty_like(cat.weight) if grad_weight is None else grad_weight
    g = grad_xi.to(torch.float64).contiguous()
    e = None if grad_wsum is None else grad_wsum.to(torch.float64).contiguous()
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xi_backward_full(handle.h, ctypes.byref(c), ctypes.byref(b), _ptr(g), _ptr(e),
                                                     _ptr(xi.contiguous()), _ptr(wsum.contiguous()), _ptr(gd),
                                                     _ptr(gw), _stream(stream)))
    return gd, gw


def lya_xi_batched(handle: Handle, mocks: Sequence[DeviceCatalog], bins, precision: str = "mixed",
                   stream=None, num=None, wsum=None, xi=None):
    nb = bins.n_par * bins.n_perp
    m = len(mocks)
    num = torch.empty(m * nb, dtype=torch.float64, device="cuda") if num is None else num
    wsum = torch.empty(m * nb, dtype=torch.float64, device="cuda") if wsum is None else wsum
    xi = torch.empty(m * nb, dtype=torch.float64, device="cuda") if xi is None else xi
    arr = (LyaCatalog * m)(*[c.c() for c in mocks])
    b = c_bins(bins)
    check(handle.h, _lib.load().lya_xi_batched(handle.h, arr, m, ctypes.byref(b), PREC[precision], _ptr(num),
                                               _ptr(wsum), _ptr(xi), _stream(stream)))
    return num.view(m, nb), wsum.view(m, nb), xi.view(m, nb)


def lya_autotune(handle: Handle, cat: DeviceCatalog, bins, stream=None) -> int:
    ch = ctypes.c_int32(-1)
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_autotune(handle.h, ctypes.byref(c), ctypes.byref(b), ctypes.byref(ch),
                                             _stream(stream)))
    return int(ch.value)


def lya_last_launch(handle: Handle):
    n, g, bl, sm = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    check(handle.h, _lib.load().lya_last_launch(handle.h, ctypes.byref(n), ctypes.byref(g), ctypes.byref(bl),
                                                ctypes.byref(sm)))
    return {"pairs": n.value, "grid": g.value, "block": bl.value, "smem": sm.value}


def lya_pair_stats(handle: Handle, cat: DeviceCatalog, bins, p_subsample: float = 1.0, seed: int = 0,
                   stream=None):
    n, pix, sq = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_pair_stats(handle.h, ctypes.byref(c), ctypes.byref(b), float(p_subsample),
                                               ctypes.c_uint64(seed), ctypes.byref(n), ctypes.byref(pix),
                                               ctypes.byref(sq), _stream(stream)))
    return {"forest_pairs": n.value, "pixel_pairs": pix.value, "pixel_pairs_sq": sq.value}


def lya_set_dmat_tiles(handle: Handle, mode: str):
    """Rank-1 tiles of the distortion-matrix kernel: "fp32" (FMA) or "tf32x3" (tensor cores)."""
    check(handle.h, _lib.load().lya_set_dmat_tiles(handle.h, {"fp32": 0, "tf32x3": 1}[mode]))


def lya_dmat_work(handle: Handle, cat: DeviceCatalog, bins, p_subsample: float, seed: int, stream=None) -> dict:
    """Work counts of the closed-form distortion matrix and its algorithmic flops
    (20 per in-grid pixel pair + 4 sum |S_v|^2 + 8 sum |S_pair|^2)."""
    n, pix = ctypes.c_int64(0), ctypes.c_int64(0)
    sv2, sp2 = ctypes.c_double(0), ctypes.c_double(0)
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_dmat_work(handle.h, ctypes.byref(c), ctypes.byref(b), float(p_subsample),
                                              int(seed), ctypes.byref(n), ctypes.byref(pix), ctypes.byref(sv2),
                                              ctypes.byref(sp2), _stream(stream)))
    return {"forest_pairs": n.value, "pixel_pairs": pix.value, "sum_vec_support_sq": sv2.value,
            "sum_pair_support_sq": sp2.value,
            "flops": 20.0 * pix.value + 4.0 * sv2.value + 8.0 * sp2.value}


def lya_xi_subsamples(handle: Handle, cat: DeviceCatalog, bins, nside: int, stream=None):
    """Per sub-sample (nested HEALPix pixel of the first forest) num, wsum, xi
    as [12 nside^2, nb] tensors, and each forest's sub-sample."""
    nb = bins.n_par * bins.n_perp
    ns = 12 * nside * nside
    num = torch.empty((ns, nb), dtype=torch.float64, device="cuda")
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)
    sub = torch.empty(max(cat.n_forests, 1), dtype=torch.int32, device="cuda")
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xi_subsamples(handle.h, ctypes.byref(c), ctypes.byref(b), int(nside), _ptr(num),
                                                  _ptr(wsum), _ptr(xi), _ptr(sub), _stream(stream)))
    return num, wsum, xi, sub[: cat.n_forests]


def lya_xi_covariance(handle: Handle, num_sub: torch.Tensor, wsum_sub: torch.Tensor, stream=None):
    """Weighted sub-sample covariance [nb, nb] and the full-sample xi [nb]."""
    ns, nb = num_sub.shape
    cov = torch.empty((nb, nb), dtype=torch.float64, device="cuda")
    xi = torch.empty(nb, dtype=torch.float64, device="cuda")
    n = num_sub.to(torch.float64).contiguous()
    w = wsum_sub.to(torch.float64).contiguous()
    check(handle.h, _lib.load().lya_xi_covariance(handle.h, _ptr(n), _ptr(w), int(ns), int(nb), _ptr(cov), _ptr(xi),
                                                  _stream(stream)))
    return cov, xi


def lya_xi3(handle: Handle, cat: DeviceCatalog, grid, stream=None):
    """Three-point estimator on grid (n_r, n_theta, n_alpha, r_max): num, wsum, xi
    as flat [n_r^2 n_alpha n_theta^2] tensors."""
    nbins = grid.n_r * grid.n_r * grid.n_alpha * grid.n_theta * grid.n_theta
    num = torch.empty(nbins, dtype=torch.float64, device="cuda")
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)
    c = cat.c()
    b = _lib.LyaBins3(int(grid.n_r), int(grid.n_theta), int(grid.n_alpha), float(grid.r_max))
    check(handle.h, _lib.load().lya_xi3(handle.h, ctypes.byref(c), ctypes.byref(b), _ptr(num), _ptr(wsum), _ptr(xi),
                                        _stream(stream)))
    return num, wsum, xi


def lya_xi_bin_means(handle: Handle, cat: DeviceCatalog, bins, stream=None, z_pix: Optional[torch.Tensor] = None):
    """Per-bin weighted mean r_par, r_perp and pair distance, W and pixel-pair
    counts (and, with per-pixel redshifts z_pix, the mean redshift "z_mean"):
    dict of [n_par n_perp] tensors."""
    nb = bins.n_par * bins.n_perp
    keys = ("wsum", "rpar_mean", "rperp_mean", "dist_mean") + (("z_mean",) if z_pix is not None else ())
    out = {k: torch.empty(nb, dtype=torch.float64, device="cuda") for k in keys}
    out["count"] = torch.empty(nb, dtype=torch.int64, device="cuda")
    c, b = cat.c(), c_bins(bins)
    if z_pix is None:
        check(handle.h, _lib.load().lya_xi_bin_means(handle.h, ctypes.byref(c), ctypes.byref(b), _ptr(out["wsum"]),
                                                     _ptr(out["rpar_mean"]), _ptr(out["rperp_mean"]),
                                                     _ptr(out["dist_mean"]), _ptr(out["count"]), _stream(stream)))
    else:
        z = z_pix.to(torch.float64).contiguous()
        check(handle.h, _lib.load().lya_xi_bin_means_z(handle.h, ctypes.byref(c), ctypes.byref(b), _ptr(z),
                                                       _ptr(out["wsum"]), _ptr(out["rpar_mean"]),
                                                       _ptr(out["rperp_mean"]), _ptr(out["dist_mean"]),
                                                       _ptr(out["z_mean"]), _ptr(out["count"]), _stream(stream)))
    return out


class DeviceQuasars:
    """Quasars resident on the GPU (layout of ``lya_quasars``)."""

    def __init__(self, ra, dec, dist, weight):
        self.ra = ra.contiguous()
        self.dec = dec.contiguous()
        self.dist = dist.contiguous()
        self.weight = weight.contiguous()
        for t in (self.ra, self.dec, self.dist):
            assert t.dtype == torch.float64
        assert self.weight.dtype == torch.float32

    @property
    def n(self) -> int:
        return int(self.ra.shape[0])

    @classmethod
    def from_host(cls, q, device="cuda") -> "DeviceQuasars":
        def t(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dt).to(device)
        return cls(t(q.ra, torch.float64), t(q.dec, torch.float64), t(q.dist, torch.float64),
                   t(q.weight, torch.float32))

    def c(self) -> "_lib.LyaQuasars":
        return _lib.LyaQuasars(self.n, self.ra.data_ptr(), self.dec.data_ptr(), self.dist.data_ptr(),
                               self.weight.data_ptr())


def _own(forest_qso):
    if forest_qso is None:
        return None, None
    t = forest_qso if isinstance(forest_qso, torch.Tensor) else torch.as_tensor(np.asarray(forest_qso))
    t = t.to(device="cuda", dtype=torch.int64).contiguous()
    return t, t.data_ptr()


def lya_xcf(handle: Handle, cat: DeviceCatalog, qso: DeviceQuasars, bins, forest_qso=None, stream=None):
    """Forest x quasar cross-correlation: num, wsum, xi as flat [n_par n_perp]
    tensors, r_par over [-r_par_max, r_par_max)."""
    nb = bins.n_par * bins.n_perp
    num = torch.empty(nb, dtype=torch.float64, device="cuda")
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)
    keep, own = _own(forest_qso)
    c, q, b = cat.c(), qso.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_xcf(handle.h, ctypes.byref(c), ctypes.byref(q), own, ctypes.byref(b),
                                        _ptr(num), _ptr(wsum), _ptr(xi), _stream(stream)))
    return num, wsum, xi


def lya_xdmat(handle: Handle, cat: DeviceCatalog, qso: DeviceQuasars, bins, p_subsample: float, seed: int,
              forest_qso=None, eta: str = "mean_slope", stream=None):
    """Distortion matrix of the cross-correlation: D [nb, nb] and W_A [nb]."""
    nb = bins.n_par * bins.n_perp
    D = torch.empty((nb, nb), dtype=torch.float64, device="cuda")
    W = torch.empty(nb, dtype=torch.float64, device="cuda")
    keep, own = _own(forest_qso)
    c, q, b = cat.c(), qso.c(), c_bins(bins)
    e = _lib.LYA_ETA_IDENTITY if eta == "identity" else _lib.LYA_ETA_MEAN_SLOPE
    check(handle.h, _lib.load().lya_xdmat(handle.h, ctypes.byref(c), ctypes.byref(q), own, ctypes.byref(b), e,
                                          float(p_subsample), ctypes.c_uint64(seed), _ptr(D), _ptr(W),
                                          _stream(stream)))
    return D, W


def lya_xi1d(handle: Handle, cat: DeviceCatalog, n_bins: int, r_max: float, stream=None):
    """Same-forest correlation: num, wsum, xi as [n_bins] tensors."""
    num = torch.empty(int(n_bins), dtype=torch.float64, device="cuda")
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)
    c = cat.c()
    check(handle.h, _lib.load().lya_xi1d(handle.h, ctypes.byref(c), int(n_bins), float(r_max), _ptr(num),
                                         _ptr(wsum), _ptr(xi), _stream(stream)))
    return num, wsum, xi


def lya_flip_tally(handle: Handle, cat: DeviceCatalog, bins, p_subsample: float = 1.0, seed: int = 0,
                   stream=None):
    n, f = ctypes.c_int64(), ctypes.c_int64()
    w, wf = ctypes.c_double(), ctypes.c_double()
    c, b = cat.c(), c_bins(bins)
    check(handle.h, _lib.load().lya_flip_tally(handle.h, ctypes.byref(c), ctypes.byref(b), float(p_subsample),
                                               ctypes.c_uint64(seed), ctypes.byref(n), ctypes.byref(f),
                                               ctypes.byref(w), ctypes.byref(wf), _stream(stream)))
    return {"pixel_pairs": n.value, "flipped": f.value, "weight": w.value, "flipped_weight": wf.value}


STAGES = {"xi": 0, "dmat": 1, "adjoint": 2, "pairs": 3}


def lya_stage_ms(handle: Handle, stage: str) -> float:
    ms = ctypes.c_float()
    check(handle.h, _lib.load().lya_stage_ms(handle.h, STAGES[stage], ctypes.byref(ms)))
    return float(ms.value)


def lya_kernel_launches() -> int:
    return int(_lib.load().lya_kernel_launches())


class Graph:
    """A captured launch sequence (``lya_graph``); ``launch`` replays it.
    Keeps its handle alive (the graph reads and writes the handle's buffers)."""

    def __init__(self, ptr, handle: Handle):
        self._g = ptr
        self._handle = handle

    def launch(self, stream=None):
        check(self._handle.h, _lib.load().lya_graph_launch(self._g, _stream(stream)))

    def close(self):
        if self._g:
            _lib.load().lya_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lya_capture_begin(handle: Handle, stream):
    """Start recording the calls made on ``handle`` with ``stream`` (a
    non-default torch.cuda.Stream).  Every output must be preallocated."""
    check(handle.h, _lib.load().lya_capture_begin(handle.h, _stream(stream)))


def lya_capture_end(handle: Handle) -> Graph:
    g = ctypes.c_void_p()
    check(handle.h, _lib.load().lya_capture_end(handle.h, ctypes.byref(g)))
    return Graph(g, handle)


# ---------------------------------------------------------------------------
# autograd
# ---------------------------------------------------------------------------
class XiFunction(torch.autograd.Function):
    """(xi, W) = estimator of Eq. (2.4) as a differentiable function of (delta, w).
    Both outputs are differentiable: W_A = sum w_i w_j depends on w."""

    @staticmethod
    def forward(ctx, delta, weight, handle, cat, bins):
        c = cat.with_(delta=delta.detach().contiguous(), weight=weight.detach().contiguous())
        num, wsum, xi = lya_xi(handle, c, bins, "mixed")
        ctx.handle, ctx.cat, ctx.bins = handle, c, bins
        ctx.save_for_backward(xi, wsum)
        return xi, wsum

    @staticmethod
    def backward(ctx, grad_xi, grad_wsum):
        xi, wsum = ctx.saved_tensors
        if grad_xi is None and grad_wsum is None:
            return None, None, None, None, None
        if grad_xi is None:
            grad_xi = torch.zeros_like(xi)
        gd, gw = lya_xi_backward_full(ctx.handle, ctx.cat, ctx.bins, grad_xi, grad_wsum, xi, wsum)
        return gd, gw, None, None, None


def xi(cat: DeviceCatalog, bins, handle: Optional[Handle] = None, delta=None, weight=None):
    """Differentiable (xi, W) for the catalogue (delta / weight may be leaf tensors)."""
    handle = handle or Handle()
    d = cat.delta if delta is None else delta
    w = cat.weight if weight is None else weight
    return XiFunction.apply(d, w, handle, cat, bins)
