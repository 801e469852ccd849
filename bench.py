#!/usr/bin/env python
"""Throughput of the Lyman-alpha pixel-pair hot path on GB300.

Default workload: the DESI-Y5-like catalogue, 600,000 forests over
10,000 deg^2 on a linear 0.8 A grid (100-600 pixels per forest, a continuum
tilt projected out), 50 x 50 bins of 4 Mpc/h.  One step = continuum
projection + pair-list build + xi/W (mixed precision) over the whole
catalogue.  `value` is in-grid pixel pairs of the xi/W sum per second of step
time.  Beside it: the plain-FP64 path on a seeded 0.5% sample of the forest
pairs, the xi kernel's roofline, the end-to-end rate through the C ABI from
host buffers, the CPU FP64 oracle on a slice of the same catalogue, a
graph-replay comparison, and (extra key `sdss_60k_step`) the SDSS-DR16-like
step with the distortion matrix and the adjoint.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own independent mock (seed + rank): the
forest pairs of different catalogues share nothing, so there is no data-path
collective ("scaling": "weak"); ranks only meet at barriers for timing.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = {"workload": "sdss_dr16_like_60k", "forests": 60000, "area_deg2": 2500,
            "bins": "50x50 of 4 Mpc/h", "dm_subsample": 0.05, "grid": "log10 step 3e-4"}
WORKLOAD_DESI = {"workload": "desi_y5_like_600k", "forests": 600000, "area_deg2": 10000,
                 "bins": "50x50 of 4 Mpc/h", "grid": "linear 0.8 A, 100-600 px, continuum tilt projected out"}
METRIC = "pixel pairs/s (xi+W) and DM pair-pairs/s at 1 GB300; fraction of FP32 roofline"
DM_P, DM_SEED = 0.05, 1234
FLOPS_PER_PAIR = 8  # 4 for the two scaled separations, 2 products, 2 accumulations


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of xi_mixed_kernel per in-grid pixel pair, from
# one ncu capture of a smaller catalogue of the same kind (summarised in profiles/), keyed by the workload and a
# hash of the kernel's sources: a launch's traffic is this times its in-grid pixel pairs, reported only while the
# sources are unchanged.  Traffic grows with the pairs: every forest pair reads its two forests' pixels (from L2
# when they are resident) and its pair-list entry.
XI_TRAFFIC = {
    # 5.3883 GB read + 15.9 MB written by one launch on a 20,000-forest catalogue of the DESI-Y5-like kind
    # (5.7033e11 in-grid pixel pairs), profiles/xi_kernel_desi_y5_like_20000.md
    "desi_y5_like": {"sha256": "2fd3b5e1b9a72de5422dc0054a2f6a7abd1ec3bbda877a3b632a6c97c59fd24e",
                     "bytes_per_pixel_pair": (5388336000 + 15879168) / 570330594405},
}


# FP64 fused multiply-adds per SM per clock measured on this GB300 (a DFMA throughput
# microbenchmark at 1.9 GHz); the plain-FP64 path's roofline uses it.
FP64_DFMA_PER_SM_CLK = 1.7


def xi_source_hash() -> str:
    import hashlib
    hsh = hashlib.sha256()
    for f in ("xi.cu", "lya_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2507_00129_gb300", "csrc", f), "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def xi_traffic(workload: str, pixel_pairs: float):
    t = XI_TRAFFIC.get(workload)
    if not t or xi_source_hash() != t["sha256"]:
        return None
    return t["bytes_per_pixel_pair"] * pixel_pairs


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples go to a file named by LYA_CLOCK_LOG_DIR (default: the system temp
        # directory); the JSON line carries their summary
        log_dir = os.environ.get("LYA_CLOCK_LOG_DIR") or tempfile.gettempdir()
        self.path = os.path.join(log_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                   "reasons": sorted(reasons), "samples": len(sm)}
        return out


def dist_setup():
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def rank_seed(rank: int) -> int:
    """Catalogue seed of a rank: each rank runs its own independent mock."""
    return 1 + rank


def aggregate(ms_local: float, units_local: float, world: int):
    """Whole-job timing over ranks: (max ms per step, total units, units/s)."""
    ms = max_over_ranks(ms_local, world)
    total = sum_over_ranks(units_local, world)
    return ms, total, total / (ms / 1e3)


# ----------------------------------------------------------------------------
# CPU oracle timing (the reported baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(cat, bins, target_pixel_pairs: float):
    """Forests inside a small cap around the catalogue centre, grown until the
    oracle's pair set holds about `target_pixel_pairs` candidate pixel pairs."""
    import oracle
    from paper_2507_00129_gb300 import synth
    n = oracle.geometry.unit_vectors(cat.ra, cat.dec)
    centre = np.array([0.0, 0.0, 1.0])
    ang = np.arccos(np.clip(n @ centre, -1, 1))
    order = np.argsort(ang)
    lens = cat.lengths()
    k = 64
    while True:
        sub = synth.subset(cat, np.sort(order[:k]))
        a, b = oracle.pairs.forest_pairs(sub, bins)
        L = sub.lengths()
        cand = float(np.sum(L[a].astype(float) * L[b]))
        if cand >= target_pixel_pairs or k >= len(order):
            return sub, (a, b), cand
        k = int(k * 1.4) + 1
    del lens


def time_oracle(cat, bins, target_pixel_pairs: float, processes: int = 0):
    import oracle
    sub, pr, cand = oracle_sample(cat, bins, target_pixel_pairs)
    procs = processes if processes > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    out = oracle.xi.xi_sums(sub, bins, pr, processes=procs)
    dt = time.perf_counter() - t0
    pix = float(out["count"].sum())
    return {"value": pix / dt, "unit": "pixel pairs/s", "cores": procs, "kind": "oracle",
            "sample": f"xi/W of {len(pr[0])} forest pairs among the {sub.n_forests} forests nearest "
                      f"the cap centre ({pix:.3g} in-grid of {cand:.3g} candidate pixel pairs), "
                      f"{dt:.1f} s on {procs} processes"}


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_slice(cat, bins, target_candidates: float):
    """The forest pairs of the catalogue that have a forest inside a small cap
    around the catalogue centre (the pole), every partner included, each pair
    once.  The cap is grown until the slice holds about `target_candidates`
    candidate pixel pairs.  Returns (sub-catalogue, local pairs, candidates,
    cap radius in degrees, forests in the cap)."""
    import oracle
    from paper_2507_00129_gb300 import synth
    n = oracle.geometry.unit_vectors(cat.ra, cat.dec)
    ang = np.degrees(np.arccos(np.clip(n[:, 2], -1.0, 1.0)))
    order = np.argsort(ang)
    dmin = float(cat.dist.min())
    th_max = np.degrees(2.0 * np.arcsin(min(1.0, bins.r_perp_max / (2.0 * dmin))))
    k = 8
    while True:
        rad = float(ang[order[k - 1]])
        near = np.nonzero(ang <= rad + th_max + 1e-9)[0]
        sub = synth.subset(cat, near)
        a, b = oracle.pairs.forest_pairs(sub, bins)
        inside = ang[near] <= rad
        keep = inside[a] | inside[b]
        a, b = a[keep], b[keep]
        L = sub.lengths()
        cand = float(np.sum(L[a].astype(float) * L[b]))
        if cand >= target_candidates or k >= len(order):
            return sub, (a, b), cand, rad, int(inside.sum())
        k = int(k * 1.3) + 1


def time_oracle_slice(cat, bins, target_candidates: float, total_pixel_pairs: float, processes: int = 0):
    """The CPU FP64 oracle on a slice of the catalogue (oracle_slice), on all
    host cores: in-grid pixel pairs per second, and the full catalogue's time
    extrapolated from that rate."""
    import oracle
    sub, pr, cand, rad, n_in = oracle_slice(cat, bins, target_candidates)
    procs = processes if processes > 0 else (os.cpu_count() or 1)
    t0 = time.perf_counter()
    out = oracle.xi.xi_sums(sub, bins, pr, processes=procs)
    dt = time.perf_counter() - t0
    pix = float(out["count"].sum())
    rate = pix / dt
    return {"value": rate, "unit": "pixel pairs/s", "cores": procs, "kind": "oracle", "cpu_model": cpu_model(),
            "sample": f"xi/W of the {len(pr[0])} forest pairs with a forest within {rad:.2f} deg of the "
                      f"catalogue centre ({n_in} forests), all partners: {pix:.3g} in-grid of {cand:.3g} "
                      f"candidate pixel pairs, {dt:.1f} s on {procs} processes",
            "extrapolated_full_catalogue_s": total_pixel_pairs / rate,
            "extrapolated": "full-catalogue time = its in-grid pixel pairs / the slice's rate"}


def run_reference(args, rank, world):
    """The reference arm of this tier: the CPU FP64 oracle on the default
    workload's catalogue, each step a bounded slice of it (oracle_slice)."""
    if rank != 0:
        return
    from paper_2507_00129_gb300 import synth
    spec = synth.spec_for(2, seed=2)
    if args.forests:
        spec.area_deg2 = spec.area_deg2 * args.forests / spec.n_forests
        spec.n_forests = args.forests
    cat = synth.generate(spec, name="desi_like")
    bins = synth.bins_for(2)
    vals = []
    info = None
    for k in range(args.warmup + args.steps):
        r = time_oracle_slice(cat, bins, 2e9, float("nan"))
        if k >= args.warmup:
            vals.append(r["value"])
            info = r
    v = float(np.median(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "pixel pairs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(WORKLOAD_DESI, **({"forests": args.forests} if args.forests else {}),
                           impl="CPU FP64 oracle (bounded slice per step)"),
            "cpu_baseline": {"value": v, "unit": "pixel pairs/s", "cores": info["cores"], "kind": "oracle",
                             "cpu_model": info["cpu_model"], "sample": info["sample"]},
            "e2e": {"value": v, "unit": "pixel pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------
def sdss_step(args, rank, world, local, steps: int, warmup: int, full: bool = True):
    """The SDSS-DR16-like step (60,000 forests, 50 x 50 bins to 200 Mpc/h):
    project + pair list + xi/W (mixed) + D (5%) + adjoint.  Returns the JSON
    line's fields; with full=False (the default workload's extra key) the
    end-to-end, plain-FP64, CPU and graph measurements are left out."""
    import torch
    from paper_2507_00129_gb300 import synth, build
    build.build()
    from paper_2507_00129_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = synth.spec_for(1, seed=rank_seed(rank))
    if args.forests:
        # smaller catalogue at the same sky density (profiling captures)
        spec.area_deg2 = spec.area_deg2 * args.forests / spec.n_forests
        spec.n_forests = args.forests
    cat = synth.generate(spec, name="sdss_like")
    bins = synth.bins_for(1)
    nb = bins.nbins
    dc = api.DeviceCatalog.from_host(cat, device=dev)
    h = api.Handle()
    g = torch.from_numpy(np.random.default_rng(303).normal(size=nb)).to(dev)
    delta_p = torch.empty_like(dc.delta)
    dcp = dc.with_(delta=delta_p)
    num = torch.empty(nb, dtype=torch.float64, device=dev)
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)

    # untimed: work counts and launch tuning
    api.lya_project(h, dc, out=delta_p)
    st = api.lya_pair_stats(h, dcp, bins, 1.0)
    dm = api.lya_pair_stats(h, dcp, bins, DM_P, DM_SEED)
    dmw = api.lya_dmat_work(h, dcp, bins, DM_P, DM_SEED)
    tune = api.lya_autotune(h, dcp, bins)

    def step():
        api.lya_project(h, dc, out=delta_p)
        api.lya_pairs_build(h, dcp, bins)
        api.lya_xi(h, dcp, bins, "mixed", num, wsum, xi)
        D, Wd = api.lya_dmat(h, dcp, bins, DM_P, DM_SEED)
        gd, gw = api.lya_xi_backward(h, dcp, bins, g, xi, wsum)
        return D, gd, gw

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    stage = {"xi": [], "dmat": [], "adjoint": [], "pairs": []}
    launches0 = api.lya_kernel_launches()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            step()
            for k in stage:
                stage[k].append(api.lya_stage_ms(h, k))
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
    launches = api.lya_kernel_launches() - launches0
    ms_local = e0.elapsed_time(e1) / steps
    ms, pix_total, value = aggregate(ms_local, float(st["pixel_pairs"]), world)
    med = {k: float(np.median(v)) for k, v in stage.items()}
    pk, how = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_fp32 = n_sm * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s at the maximum SM clock
    ach = FLOPS_PER_PAIR * st["pixel_pairs"] / (med["xi"] / 1e3) / 1e12
    ach_dm = dmw["flops"] / (med["dmat"] / 1e3) / 1e12
    dm_line = {"pair_pairs_per_s": dm["pixel_pairs_sq"] / (med["dmat"] / 1e3),
               "pair_pairs": dm["pixel_pairs_sq"], "forest_pairs": dm["forest_pairs"],
               "pixel_pairs": dm["pixel_pairs"],
               "closed_form_flops": dmw["flops"], "sum_vec_support_sq": dmw["sum_vec_support_sq"],
               "sum_pair_support_sq": dmw["sum_pair_support_sq"],
               "roofline_dm": {"bound": "alu", "kernel": "dm_kernel", "achieved": ach_dm, "peak": peak_fp32,
                               "unit": "TFLOP/s", "frac": ach_dm / peak_fp32,
                               "flops_note": "20 per in-grid pixel pair + 4 sum |S_v|^2 + 8 sum |S_pair|^2 "
                                             "(lya_dmat_work), over the D stage's device time"}}
    # the same D stage with the rank-1 tiles on the tensor cores (TF32x3) instead of FP32 FMA
    tiles = {"fp32_fma_ms": med["dmat"]}
    try:
        api.lya_set_dmat_tiles(h, "tf32x3")
        api.lya_dmat(h, dcp, bins, DM_P, DM_SEED)
        tt = []
        for _ in range(2):
            api.lya_dmat(h, dcp, bins, DM_P, DM_SEED)
            tt.append(api.lya_stage_ms(h, "dmat"))
        tiles["tf32x3_tensor_ms"] = float(np.median(tt))
    finally:
        api.lya_set_dmat_tiles(h, "fp32")
    dm_line["rank1_tiles"] = tiles
    if not full:
        flips = api.lya_flip_tally(h, dcp, bins, 0.01, 99)
        flips["fraction_of_weight"] = flips["flipped_weight"] / max(flips["weight"], 1e-300)
        h.close()
        return {"workload": "sdss_dr16_like_60k", "step": "project + pair list + xi/W mixed + D (5%) + adjoint",
                "value": value, "unit": "pixel pairs/s", "ms_per_step": ms, "steps": steps, "warmup": warmup,
                "stages_ms": med, "dominant_stage": max(med, key=med.get),
                "xi_kernel": {"pixel_pairs_per_s": st["pixel_pairs"] / (med["xi"] / 1e3),
                              "pixel_pairs": st["pixel_pairs"], "forest_pairs": st["forest_pairs"],
                              "roofline": {"bound": "alu", "achieved": ach, "peak": peak_fp32, "unit": "TFLOP/s",
                                           "frac": ach / peak_fp32}},
                "dm": dm_line,
                "adjoint": {"ms": med["adjoint"],
                            "pixel_pair_visits_per_s": 2 * st["pixel_pairs"] / (med["adjoint"] / 1e3)},
                "edge_flips": flips, "gpu_launches": int(launches), "clocks": clk.summary()}

    # end to end through the public API from pinned host memory
    host = {k: getattr(dc, k).cpu().pin_memory() for k in
            ("offsets", "ra", "dec", "dist", "loglam", "delta", "weight")}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    e2e_steps = max(1, min(steps, 3))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        devt = {k: v.to(dev, non_blocking=True) for k, v in host.items()}
        dce = api.DeviceCatalog(**devt)
        dpe = torch.empty_like(dce.delta)
        api.lya_project(h, dce, out=dpe)
        dcep = dce.with_(delta=dpe)
        api.lya_pairs_build(h, dcep, bins)
        n_, w_, x_ = api.lya_xi(h, dcep, bins, "mixed")
        D, Wd = api.lya_dmat(h, dcep, bins, DM_P, DM_SEED)
        gd, gw = api.lya_xi_backward(h, dcep, bins, g, x_, w_)
        outs = [x_.cpu(), w_.cpu(), D.cpu(), gd.cpu(), gw.cpu()]
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    d2h = sum(t.numel() * t.element_size() for t in outs)

    # plain-FP64 path on the same workload (one timed call, after a warm-up)
    fp64 = None
    if not args.no_fp64:
        api.lya_xi(h, dcp, bins, "fp64", num, wsum, xi)
        torch.cuda.synchronize()
        f0 = time.perf_counter()
        api.lya_xi(h, dcp, bins, "fp64", num, wsum, xi)
        torch.cuda.synchronize()
        fms = api.lya_stage_ms(h, "xi")
        fp64 = {"pixel_pairs_per_s": st["pixel_pairs"] / (fms / 1e3), "kernel_ms": fms,
                "call_ms": (time.perf_counter() - f0) * 1e3}

    if fp64 is not None:
        # the plain-FP64 path against an FP64 peak from the DFMA rate measured on this part
        # (1.7 DFMA per SM per clock in a microbenchmark), same 8 algorithmic flops per pair
        peak_fp64 = n_sm * FP64_DFMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
        a64 = FLOPS_PER_PAIR * fp64["pixel_pairs_per_s"] / 1e12
        fp64["roofline"] = {"bound": "fp64", "achieved": a64, "peak": peak_fp64, "unit": "TFLOP/s",
                            "frac": a64 / peak_fp64,
                            "peak_note": f"{n_sm} SMs x {FP64_DFMA_PER_SM_CLK} DFMA x 2 flops x {sm_max:.0f} MHz "
                                         "(DFMA rate measured on this GB300)"}
    dominant = max(med, key=med.get)
    # FP32-vs-FP64 bin-edge flips of the mixed path on a seeded 1% of the forest pairs
    flips = api.lya_flip_tally(h, dcp, bins, 0.01, 99)
    flips["fraction_of_pixel_pairs"] = flips["flipped"] / max(flips["pixel_pairs"], 1)
    flips["fraction_of_weight"] = flips["flipped_weight"] / max(flips["weight"], 1e-300)
    flips["sample"] = "forest pairs kept by the subsample rule with p = 0.01, seed 99"
    # covariance from HEALPix sub-samples (nside 8, the data split of the paper's inputs)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    n_s, w_s, _, _ = api.lya_xi_subsamples(h, dcp, bins, 8)
    ev[1].record()
    cov, _ = api.lya_xi_covariance(h, n_s, w_s)
    ev[2].record()
    torch.cuda.synchronize()
    covariance = {"nside": 8, "subsamples_with_pairs": int((w_s.sum(dim=1) > 0).sum()),
                  "subsample_xi_ms": ev[0].elapsed_time(ev[1]), "covariance_ms": ev[1].elapsed_time(ev[2])}
    del n_s, w_s, cov
    graph = None if args.no_graph else graph_replay(api, synth, dev)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(cat, bins, 6e9)
    line = {
        "metric": METRIC, "value": value, "unit": "pixel pairs/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD, **({"forests": args.forests} if args.forests else {}),
                       l2="inputs larger than L2 (catalogue 450 MB; packed pixels 180 MB)",
                       step="project + pair list + xi/W mixed + D (5%) + adjoint",
                       seeds=f"catalogue seed 1+rank, DM seed {DM_SEED}"),
        "roofline": {"bound": "alu", "kernel": "xi_mixed_kernel", "achieved": ach, "peak": peak_fp32,
                     "unit": "TFLOP/s", "frac": ach / peak_fp32,
                     "traffic": xi_traffic("sdss_dr16_like", st["pixel_pairs"]),
                     "peak_note": f"FP32 FMA peak {n_sm} SMs x 128 lanes x 2 flops x {sm_max:.0f} MHz "
                                  f"(sm_max of {how} peaks); {FLOPS_PER_PAIR} algorithmic flops per "
                                  "in-grid pixel pair; traffic = ncu DRAM bytes of one full-size launch "
                                  "(bytes), null if the kernel changed since"},
        "stages_ms": med, "dominant_stage": dominant,
        "xi_kernel": {"pixel_pairs_per_s": st["pixel_pairs"] / (med["xi"] / 1e3),
                      "pixel_pairs": st["pixel_pairs"], "forest_pairs": st["forest_pairs"]},
        "dm": dm_line,
        "fp64_path": fp64,
        "edge_flips": flips,
        "covariance": covariance,
        "graph_replay": graph,
        "autotune_choice": tune,
        "e2e": {"value": pix_total / e2e_s, "unit": "pixel pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
    }
    h.close()
    return line


def run_sdss(args, rank, world, local):
    line = sdss_step(args, rank, world, local, args.steps, args.warmup, full=True)
    if rank == 0:
        print(json.dumps(line), flush=True)


def graph_replay(api, synth, dev, iters: int = 20):
    """Eager calls vs a captured CUDA graph for the tiny workload (200 forests,
    25 x 25 bins): project + xi/W + adjoint + D, per iteration, on one stream."""
    import torch
    cat = synth.make(0)
    bins = synth.bins_for(0)
    nb = bins.nbins
    dc = api.DeviceCatalog.from_host(cat, device=dev)
    h = api.Handle()
    o = {"dp": torch.empty_like(dc.delta), "num": torch.empty(nb, dtype=torch.float64, device=dev),
         "wsum": torch.empty(nb, dtype=torch.float64, device=dev), "xi": torch.empty(nb, dtype=torch.float64, device=dev),
         "gd": torch.empty_like(dc.delta), "gw": torch.empty_like(dc.weight),
         "D": torch.empty((nb, nb), dtype=torch.float64, device=dev), "Wd": torch.empty(nb, dtype=torch.float64, device=dev)}
    g = torch.from_numpy(np.random.default_rng(303).normal(size=nb)).to(dev)
    s = torch.cuda.Stream(device=dev)

    def calls():
        dcp = dc.with_(delta=o["dp"])
        api.lya_project(h, dc, out=o["dp"], stream=s)
        api.lya_xi(h, dcp, bins, "mixed", o["num"], o["wsum"], o["xi"], stream=s)
        api.lya_xi_backward(h, dcp, bins, g, o["xi"], o["wsum"], stream=s, grad_delta=o["gd"], grad_weight=o["gw"])
        api.lya_dmat(h, dcp, bins, 1.0, 3, stream=s, D=o["D"], W=o["Wd"])

    with torch.cuda.stream(s):
        for _ in range(3):
            calls()
        api.lya_sync_status(h, s)
        api.lya_capture_begin(h, s)
        calls()
        gr = api.lya_capture_end(h)
        for _ in range(3):
            gr.launch(s)
        s.synchronize()
        k0 = api.lya_kernel_launches()
        t0 = time.perf_counter()
        for _ in range(iters):
            calls()
        s.synchronize()
        eager_ms = (time.perf_counter() - t0) * 1e3 / iters
        k1 = api.lya_kernel_launches()
        t0 = time.perf_counter()
        for _ in range(iters):
            gr.launch(s)
        s.synchronize()
        graph_ms = (time.perf_counter() - t0) * 1e3 / iters
        k2 = api.lya_kernel_launches()
    gr.close()
    h.close()
    return {"workload": "tiny_200_forests", "step": "project + xi/W + adjoint + D (p = 1)",
            "eager_ms_per_iter": eager_ms, "graph_ms_per_iter": graph_ms,
            "kernels_per_iter": (k1 - k0) / iters, "graph_kernels_per_iter": (k2 - k1) / iters,
            "iters": iters}


def run_ours(args, rank, world, local):
    """The default line: the DESI-Y5-like catalogue (600,000 forests), one step
    = project + pair list + xi/W (mixed) over the whole catalogue."""
    import torch
    from paper_2507_00129_gb300 import synth, build
    build.build()
    from paper_2507_00129_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = synth.spec_for(2, seed=2 + rank)
    if args.forests:
        spec.area_deg2 = spec.area_deg2 * args.forests / spec.n_forests
        spec.n_forests = args.forests
    t_gen = time.perf_counter()
    cat = synth.generate(spec, name="desi_like")
    t_gen = time.perf_counter() - t_gen
    bins = synth.bins_for(2)
    nb = bins.nbins
    dc = api.DeviceCatalog.from_host(cat, device=dev)
    h = api.Handle()
    dp = torch.empty_like(dc.delta)
    dcp = dc.with_(delta=dp)
    num = torch.empty(nb, dtype=torch.float64, device=dev)
    wsum = torch.empty_like(num)
    xi = torch.empty_like(num)
    # launch shape tuned on a 30,000-forest catalogue of the same kind (same bins)
    tspec = synth.spec_for(2, seed=1000 + rank, n_forests=30000)
    tspec.area_deg2 = spec.area_deg2 * 30000 / spec.n_forests
    tcat = api.DeviceCatalog.from_host(synth.generate(tspec), device=dev)
    tune = api.lya_autotune(h, tcat, bins)
    del tcat
    api.lya_project(h, dc, out=dp)
    st = api.lya_pair_stats(h, dcp, bins, 1.0)
    max_len = int(cat.lengths().max())

    def step():
        api.lya_project(h, dc, out=dp)
        api.lya_pairs_build(h, dcp, bins)
        api.lya_xi(h, dcp, bins, "mixed", num, wsum, xi)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    stage = {"xi": [], "pairs": []}
    launches0 = api.lya_kernel_launches()
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            step()
            for k in stage:
                stage[k].append(api.lya_stage_ms(h, k))
        e1.record()
        torch.cuda.synchronize()
        barrier(world)
    launches = api.lya_kernel_launches() - launches0
    ms_local = e0.elapsed_time(e1) / args.steps
    ms, pix_total, value = aggregate(ms_local, float(st["pixel_pairs"]), world)
    med = {k: float(np.median(v)) for k, v in stage.items()}

    # end to end through the C ABI: pinned host catalogue -> device, the step,
    # xi and W back to the host
    host = {k: getattr(dc, k).cpu().pin_memory() for k in
            ("offsets", "ra", "dec", "dist", "loglam", "delta", "weight")}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    e2e_steps = max(1, min(args.steps, 2))
    devt = {k: torch.empty_like(getattr(dc, k)) for k in host}
    dce = api.DeviceCatalog(**devt)
    dpe = torch.empty_like(dce.delta)
    dcep = dce.with_(delta=dpe)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for k, v in host.items():
            devt[k].copy_(v, non_blocking=True)
        api.lya_project(h, dce, out=dpe)
        api.lya_pairs_build(h, dcep, bins)
        n_, w_, x_ = api.lya_xi(h, dcep, bins, "mixed")
        outs = [x_.cpu(), w_.cpu()]
    torch.cuda.synchronize()
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps, world)
    d2h = sum(t.numel() * t.element_size() for t in outs)
    del devt, dce, dpe, dcep

    # graph replay of project + xi/W (the pair list is cached between replays)
    graph = None if args.no_graph else graph_replay_large(api, h, dc, dp, dcp, bins, num, wsum, xi, dev)

    # plain FP64 beside mixed on a seeded 0.5% sample of the forest pairs
    fp64 = None
    if not args.no_fp64:
        n = api.lya_pairs_build(h, dcp, bins)
        pa, pb = api.lya_pairs_get(h, n)
        gen = torch.Generator(device=dev)
        gen.manual_seed(7)
        sel = torch.rand(n, generator=gen, device=dev) < 0.005
        sa, sb = pa[sel].contiguous(), pb[sel].contiguous()
        del pa, pb, sel
        sub = {}
        for prec in ("mixed", "fp64"):
            api.lya_xi_pairs(h, dcp, bins, sa, sb, prec)
            torch.cuda.synchronize()
            api.lya_xi_pairs(h, dcp, bins, sa, sb, prec)
            sub[prec] = api.lya_stage_ms(h, "xi")
        # in-grid pixel pairs of the sample (counted with the mixed binning)
        _, wcount, _ = api.lya_xi_pairs(h, dcp.with_(weight=torch.ones_like(dc.weight)), bins, sa, sb, "mixed")
        sample_pix = float(wcount.sum())
        fp64 = {"sample": "seeded 0.5% of the forest pairs (torch generator seed 7)", "forest_pairs": int(sa.numel()),
                "pixel_pairs": sample_pix, "mixed_ms": sub["mixed"], "fp64_ms": sub["fp64"],
                "mixed_pixel_pairs_per_s": sample_pix / (sub["mixed"] / 1e3),
                "fp64_pixel_pairs_per_s": sample_pix / (sub["fp64"] / 1e3)}
        del sa, sb

    pk, how = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_fp32 = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    ach = FLOPS_PER_PAIR * st["pixel_pairs"] / (med["xi"] / 1e3) / 1e12
    if fp64 is not None:
        peak_fp64 = n_sm * FP64_DFMA_PER_SM_CLK * 2 * sm_max * 1e6 / 1e12
        a64 = FLOPS_PER_PAIR * fp64["fp64_pixel_pairs_per_s"] / 1e12
        fp64["roofline"] = {"bound": "fp64", "achieved": a64, "peak": peak_fp64, "unit": "TFLOP/s",
                            "frac": a64 / peak_fp64,
                            "peak_note": f"{n_sm} SMs x {FP64_DFMA_PER_SM_CLK} DFMA x 2 flops x {sm_max:.0f} MHz "
                                         "(DFMA rate measured on this GB300)"}
    h.close()
    del dc, dcp, dp
    torch.cuda.empty_cache()

    # the SDSS-DR16-like step with D and the adjoint (timed extra key)
    sdss = None
    if not args.no_sdss:
        try:
            sdss = sdss_step(args, rank, world, local, steps=3, warmup=2, full=False)
        except Exception as e:  # keep the headline line
            sdss = {"error": f"{type(e).__name__}: {e}"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle_slice(cat, bins, 3e9, float(st["pixel_pairs"]))
    line = {
        "metric": METRIC, "value": value, "unit": "pixel pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(WORKLOAD_DESI, **({"forests": args.forests} if args.forests else {}),
                       l2="inputs larger than L2 (catalogue 4.8 GB; packed pixels and prefix sums 7 GB)",
                       step="project + pair list + xi/W mixed", seeds="catalogue seed 2+rank",
                       fp64_path="plain-FP64 kernel on a seeded 0.5% sample of the forest pairs"),
        "roofline": {"bound": "alu", "kernel": "xi_mixed_kernel", "achieved": ach, "peak": peak_fp32,
                     "unit": "TFLOP/s", "frac": ach / peak_fp32,
                     "traffic": xi_traffic("desi_y5_like", st["pixel_pairs"]),
                     "peak_note": f"FP32 FMA peak {n_sm} SMs x 128 lanes x 2 flops x {sm_max:.0f} MHz "
                                  f"(sm_max of {how} peaks); {FLOPS_PER_PAIR} algorithmic flops per "
                                  "in-grid pixel pair; achieved over the kernel's own device time (CUDA events "
                                  "on its stream); traffic = ncu DRAM bytes per launch scaled from a smaller "
                                  "capture, null if the kernel changed since"},
        "stages_ms": med, "dominant_stage": max(med, key=med.get),
        "xi_kernel": {"pixel_pairs_per_s": st["pixel_pairs"] / (med["xi"] / 1e3),
                      "pixel_pairs": st["pixel_pairs"], "forest_pairs": st["forest_pairs"],
                      "max_forest_pixels": max_len},
        "fp64_path": fp64,
        "graph_replay": graph,
        "sdss_60k_step": sdss,
        "autotune_choice": tune, "generate_s": t_gen,
        "e2e": {"value": pix_total / e2e_s, "unit": "pixel pairs/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "gpu_launches": int(launches), "clocks": clk.summary(), "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def graph_replay_large(api, h, dc, dp, dcp, bins, num, wsum, xi, dev, iters: int = 1):
    """Eager calls vs a replayed CUDA graph of the same calls (project + xi/W
    on the cached pair list) on the default workload, on one side stream."""
    import torch
    s = torch.cuda.Stream(device=dev)

    def calls():
        api.lya_project(h, dc, out=dp, stream=s)
        api.lya_xi(h, dcp, bins, "mixed", num, wsum, xi, stream=s)

    with torch.cuda.stream(s):
        calls()
        api.lya_sync_status(h, s)
        api.lya_capture_begin(h, s)
        calls()
        gr = api.lya_capture_end(h)
        gr.launch(s)
        s.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record(s)
        for _ in range(iters):
            calls()
        ev[1].record(s)
        for _ in range(iters):
            gr.launch(s)
        ev[2].record(s)
        s.synchronize()
    gr.close()
    return {"workload": "desi_y5_like_600k", "step": "project + xi/W (pair list cached)",
            "eager_ms_per_iter": ev[0].elapsed_time(ev[1]) / iters,
            "graph_ms_per_iter": ev[1].elapsed_time(ev[2]) / iters, "iters": iters}


def run_mocks(args, rank, world, local):
    """The mock batch: N independent DESI-like catalogues of 15,000 forests
    (seeds N*rank .. N*rank+N-1); one step = xi/W of all mocks in one launch
    + D on a 2% forest-pair subsample of all mocks in one launch."""
    import torch
    from paper_2507_00129_gb300 import synth, build
    build.build()
    from paper_2507_00129_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    nm = args.mocks
    p_dm, seed_dm = 0.02, 4321
    t_gen = time.perf_counter()
    mocks = [api.DeviceCatalog.from_host(synth.make(4, seed=nm * rank + m), device=dev) for m in range(nm)]
    t_gen = time.perf_counter() - t_gen
    bins = synth.bins_for(4)
    nb = bins.nbins
    h = api.Handle()
    tune = api.lya_autotune(h, mocks[0], bins)
    pix = dmpp = 0.0
    dmpairs = 0
    for m in mocks:
        st = api.lya_pair_stats(h, m, bins, 1.0)
        sd = api.lya_pair_stats(h, m, bins, p_dm, seed_dm)
        pix += st["pixel_pairs"]
        dmpp += sd["pixel_pairs_sq"]
        dmpairs += sd["forest_pairs"]
    D = torch.empty((nm, nb, nb), dtype=torch.float64, device=dev)
    Wd = torch.empty((nm, nb), dtype=torch.float64, device=dev)

    def step():
        n_, w_, x_ = api.lya_xi_batched(h, mocks, bins, "mixed")
        api.lya_dmat_batched(h, mocks, bins, p_dm, seed_dm, D=D, W=Wd)
        return n_, w_, x_

    t0 = time.perf_counter()
    for _ in range(args.warmup):
        n_, w_, x_ = step()
    torch.cuda.synchronize()
    first_s = time.perf_counter() - t0
    barrier(world)
    stage = {"xi": [], "dmat": []}
    with Clocks(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches0 = api.lya_kernel_launches()
        e0.record()
        for _ in range(args.steps):
            n_, w_, x_ = step()
            for k in stage:
                stage[k].append(api.lya_stage_ms(h, k))
        e1.record()
        torch.cuda.synchronize()
        launches = api.lya_kernel_launches() - launches0
        barrier(world)
    ms_local = e0.elapsed_time(e1) / args.steps
    ms, pix_total, value = aggregate(ms_local, pix, world)
    med = {k: float(np.median(v)) for k, v in stage.items()}
    # eager calls against a replayed CUDA graph of the same step (pair lists cached)
    graph = None
    if not args.no_graph:
        s_ = torch.cuda.Stream(device=dev)
        outs = {"n": torch.empty((nm, nb), dtype=torch.float64, device=dev),
                "w": torch.empty((nm, nb), dtype=torch.float64, device=dev),
                "x": torch.empty((nm, nb), dtype=torch.float64, device=dev)}

        def calls():
            api.lya_xi_batched(h, mocks, bins, "mixed", stream=s_, num=outs["n"], wsum=outs["w"], xi=outs["x"])
            api.lya_dmat_batched(h, mocks, bins, p_dm, seed_dm, D=D, W=Wd, stream=s_)

        with torch.cuda.stream(s_):
            calls()
            api.lya_sync_status(h, s_)
            api.lya_capture_begin(h, s_)
            calls()
            gr = api.lya_capture_end(h)
            gr.launch(s_)
            s_.synchronize()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(s_)
            calls()
            ev[1].record(s_)
            gr.launch(s_)
            ev[2].record(s_)
            s_.synchronize()
        gr.close()
        graph = {"workload": f"mock_batch_{nm}x15k", "step": "xi/W batched + D batched (pair lists cached)",
                 "eager_ms_per_iter": ev[0].elapsed_time(ev[1]), "graph_ms_per_iter": ev[1].elapsed_time(ev[2]),
                 "iters": 1}
    # per-mock deviation of the batched mixed path from the plain-FP64 path (two mocks)
    dev_rows = []
    for m in range(min(2, nm)):
        _, w64, x64 = api.lya_xi(h, mocks[m], bins, "fp64")
        W64, X64 = w64.cpu().numpy(), x64.cpu().numpy()
        Wm, Xm = w_[m].cpu().numpy(), x_[m].cpu().numpy()
        on = W64 > 0
        dev_rows.append({"mock": m, "max_rel_dW": float(np.max(np.abs(Wm - W64)[on] / W64[on])),
                         "max_abs_dxi": float(np.max(np.abs(Xm - X64))), "rms_xi": float(np.sqrt(np.mean(X64 ** 2)))})
    pk, how = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_fp32 = n_sm * 128 * 2 * sm_max * 1e6 / 1e12
    ach = FLOPS_PER_PAIR * pix / (med["xi"] / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": "pixel pairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"mock_batch_{nm}x15k", "mocks": nm, "forests_per_mock": 15000, "area_deg2": 600,
                   "bins": "50x50 of 4 Mpc/h", "dm_subsample": p_dm, "grid": "linear 0.8 A, 100-600 px",
                   "step": "xi/W of all mocks in one launch + D (2%) of all mocks in one launch",
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "alu", "kernel": "xi_mixed_kernel", "achieved": ach, "peak": peak_fp32,
                     "unit": "TFLOP/s", "frac": ach / peak_fp32, "traffic": None},
        "stages_ms": med,
        "xi_kernel": {"pixel_pairs_per_s": pix / (med["xi"] / 1e3), "pixel_pairs": pix},
        "dm": {"pair_pairs_per_s": dmpp / (med["dmat"] / 1e3), "pair_pairs": dmpp, "forest_pairs": dmpairs},
        "mixed_vs_fp64_per_mock": dev_rows, "first_call_s": first_s, "generate_s": t_gen, "graph_replay": graph,
        "autotune_choice": tune, "gpu_launches": int(launches), "clocks": clk.summary(),
        "cpu_baseline": None, "e2e": None,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()


def run_xi3(args, rank, world, local):
    """The anisotropic three-point estimator on the SDSS-DR16-like catalogue:
    r_max = 40 Mpc/h (the paper's 3PCF timings) with 4 Mpc/h radial bins,
    10 theta bins and 20 cos(alpha) bins (the figure's bin widths)."""
    import torch
    from paper_2507_00129_gb300 import synth, build
    build.build()
    from paper_2507_00129_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = synth.spec_for(1, seed=rank_seed(rank))
    if args.forests:
        spec.area_deg2 = spec.area_deg2 * args.forests / spec.n_forests
        spec.n_forests = args.forests
    cat = synth.generate(spec, name="sdss_like")
    grid = type("Grid3", (), {"n_r": 10, "n_theta": 10, "n_alpha": 20, "r_max": 40.0})
    dc = api.DeviceCatalog.from_host(cat, device=dev)
    h = api.Handle()
    # records per bin with unit weights (untimed): the work count
    _, cnt, _ = api.lya_xi3(h, dc.with_(weight=torch.ones_like(dc.weight)), grid)
    api.lya_sync_status(h)
    records = float(cnt.sum())
    for _ in range(args.warmup):
        api.lya_xi3(h, dc, grid)
    torch.cuda.synchronize()
    barrier(world)
    ks = []
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches0 = api.lya_kernel_launches()
        e0.record()
        for _ in range(args.steps):
            api.lya_xi3(h, dc, grid)
            ks.append(api.lya_stage_ms(h, "xi"))
        e1.record()
        torch.cuda.synchronize()
        launches = api.lya_kernel_launches() - launches0
    api.lya_sync_status(h)
    ms_local = e0.elapsed_time(e1) / args.steps
    ms, rec_total, value = aggregate(ms_local, records, world)
    line = {
        "metric": "triangle records/s (3PCF)", "value": value, "unit": "records/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "sdss_dr16_like_60k_xi3", "forests": spec.n_forests, "r_max": 40.0, "n_r": 10,
                   "n_theta": 10, "n_alpha": 20, "bins": 200000,
                   "unit": "records = (main vertex, ordered pair of two other pixels) with |r1|, |r2| < r_max"},
        "records": records, "kernel_ms": float(np.median(ks)),
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()


def run_xcf(args, rank, world, local):
    """Forest x quasar cross-correlation on the SDSS-DR16-like catalogue: 60,000
    forests, 90,000 quasars (each forest's own plus 30,000 without a forest),
    r_par in [-200, 200) Mpc/h in 100 bins, r_perp < 200 in 50.  A step is the
    cross-correlation and its distortion matrix (2% of the forest-quasar pairs)
    on the cached (forest, quasar) list, whose build is timed once beside it;
    the 1D same-forest correlation (50 bins to 200 Mpc/h) and the per-bin
    means and counts of the auto-correlation are timed on their own."""
    import time
    import torch
    from paper_2507_00129_gb300 import synth, build
    build.build()
    from paper_2507_00129_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = synth.spec_for(1, seed=rank_seed(rank))
    if args.forests:
        spec.area_deg2 = spec.area_deg2 * args.forests / spec.n_forests
        spec.n_forests = args.forests
    cat = synth.generate(spec, name="sdss_like")
    qso, own = synth.quasars(spec, cat, extra_fraction=0.5)
    bins = synth.Bins(100, 50, 200.0, 200.0)
    p_dm, seed = 0.02, 2024
    dc = api.DeviceCatalog.from_host(cat, device=dev)
    dq = api.DeviceQuasars.from_host(qso, device=dev)
    own_d = torch.from_numpy(own).to(dev)
    h = api.Handle()
    # work counts with unit weights (untimed)
    ones_q = api.DeviceQuasars(dq.ra, dq.dec, dq.dist, torch.ones_like(dq.weight))
    _, cnt, _ = api.lya_xcf(h, dc.with_(weight=torch.ones_like(dc.weight)), ones_q, bins, forest_qso=own_d)
    n_xpairs = int(api.lya_last_launch(h)["pairs"])
    pair_build_ms = api.lya_stage_ms(h, "pairs")   # the list is cached for the timed calls (same geometry)
    _, cnt1, _ = api.lya_xi1d(h, dc.with_(weight=torch.ones_like(dc.weight)), 50, 200.0)
    api.lya_sync_status(h)
    pix_pairs, pix_pairs_1d = float(cnt.sum()), float(cnt1.sum())

    def step():
        api.lya_xcf(h, dc, dq, bins, forest_qso=own_d)
        api.lya_xdmat(h, dc, dq, bins, p_dm, seed, forest_qso=own_d)

    for _ in range(args.warmup):
        step()
        api.lya_xi1d(h, dc, 50, 200.0)
    torch.cuda.synchronize()
    barrier(world)
    st = {"xcf": [], "xdmat": []}
    with Clocks(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        launches0 = api.lya_kernel_launches()
        e0.record()
        for _ in range(args.steps):
            api.lya_xcf(h, dc, dq, bins, forest_qso=own_d)
            st["xcf"].append(api.lya_stage_ms(h, "xi"))
            api.lya_xdmat(h, dc, dq, bins, p_dm, seed, forest_qso=own_d)
            st["xdmat"].append(api.lya_stage_ms(h, "dmat"))
        e1.record()
        torch.cuda.synchronize()
        launches = api.lya_kernel_launches() - launches0
        # 1D correlation, timed on its own
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record()
        for _ in range(args.steps):
            api.lya_xi1d(h, dc, 50, 200.0)
        f1.record()
        torch.cuda.synchronize()
    # per-bin means and counts of the auto-correlation (50 x 50 bins to 200), on its cached pair list
    abins = synth.bins_for(1)
    bm = api.lya_xi_bin_means(h, dc, abins)
    torch.cuda.synchronize()
    m0 = torch.cuda.Event(enable_timing=True)
    m1 = torch.cuda.Event(enable_timing=True)
    m0.record()
    for _ in range(args.steps):
        bm = api.lya_xi_bin_means(h, dc, abins)
    m1.record()
    torch.cuda.synchronize()
    api.lya_sync_status(h)
    ms_local = e0.elapsed_time(e1) / args.steps
    ms1d = f0.elapsed_time(f1) / args.steps
    ms_means = m0.elapsed_time(m1) / args.steps
    n_means = float(bm["count"].sum())
    ms, tot, value = aggregate(ms_local, pix_pairs, world)
    line = {
        "metric": "forest-quasar pixel pairs/s (cross-correlation + its D)", "value": value,
        "unit": "pixel-quasar pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": "sdss_dr16_like_60k_xcf", "forests": spec.n_forests, "quasars": qso.n,
                   "bins": [bins.n_par, bins.n_perp], "r_par": [-200.0, 200.0], "r_perp_max": 200.0,
                   "dm_fraction": p_dm, "l2": "inputs 0.2 GB + 90k quasars; D~ 200 MB > L2",
                   "unit": "in-grid (pixel, quasar) pairs"},
        "pixel_quasar_pairs": pix_pairs, "forest_quasar_pairs": n_xpairs,
        "stages_ms": {k: float(np.median(v)) for k, v in st.items()},
        "pair_build_ms": pair_build_ms,
        "xi1d": {"ms": ms1d, "pixel_pairs": pix_pairs_1d, "pairs_per_s": pix_pairs_1d / (ms1d * 1e-3),
                 "bins": 50, "r_max": 200.0},
        "bin_means": {"ms": ms_means, "pixel_pairs": n_means, "pairs_per_s": n_means / (ms_means * 1e-3),
                      "bins": [abins.n_par, abins.n_perp]},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        nf = min(600, cat.n_forests)
        sub = synth.subset(cat, np.arange(nf))
        t0 = time.perf_counter()
        pl = oracle.xcf.forest_quasar_pairs(sub, qso, bins, own[:nf])
        ref = oracle.xcf.xcf_sums(sub, qso, bins, pl)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": float(ref["count"].sum()) / dt, "unit": "pixel-quasar pairs/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"cross-correlation sums of the first {nf} forests with all quasars "
                                          f"({dt:.1f} s, pair search included; D not included)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--forests", type=int, default=0,
                    help="profiling: use this many forests (same sky density) instead of the workload's")
    ap.add_argument("--workload", default="desi", choices=["sdss", "desi", "mocks", "xi3", "xcf"],
                    help="desi: 600,000-forest DESI-Y5-like xi step (default); sdss: 60,000-forest SDSS-DR16-like "
                         "step with D and the adjoint; "
                         "mocks: batch of 15,000-forest mocks, xi/W + D (2%%) in one launch each; "
                         "xi3: three-point estimator on the 60,000-forest catalogue; "
                         "xcf: forest x quasar cross-correlation, its D and the 1D correlation")
    ap.add_argument("--mocks", type=int, default=128, help="mocks per rank for --workload mocks")
    ap.add_argument("--no-graph", action="store_true", help="skip the graph-replay measurement")
    ap.add_argument("--no-sdss", action="store_true", help="default workload: skip the SDSS-DR16-like extra step")
    args = ap.parse_args()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "sdss":
        run_sdss(args, rank, world, local)
    elif args.workload == "mocks":
        run_mocks(args, rank, world, local)
    elif args.workload == "xi3":
        run_xi3(args, rank, world, local)
    elif args.workload == "xcf":
        run_xcf(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
