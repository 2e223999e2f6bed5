#!/usr/bin/env python
"""Throughput of full-polarisation AW-projection gridding + degridding on GB300.

Workload (default): 4 linear correlations, 16 Mueller A-kernels from an Airy
beam (12 m dish) with 1 % complex leakage, Eq. 6 regularised inverse for
gridding, 32 w planes x 8 parallactic-angle bins x 4 beam-frequency bins
(1024 bins, supports 16..72 cells, oversampling 8), 288 channels of uneven
visibility counts (~64M visibilities), 4096 x 4096 x 4 complex64 grid.
Synthetic ASKAP-shaped geometry (see paper_2206_15117_gb300.synthetic);
visibility values are seeded complex Gaussian noise (the work does not depend
on them).

One step = one Cotton-Schwab major-cycle pass of the hot path: zero the grid,
aw_grid_batched (persistent, graph-captured, autotuned), aw_fft_to_image,
aw_degrid.  Kernel synthesis and the visibility sort run once per dataset
before the timed region and are reported separately.

`--impl reference` times the FP64 CPU oracle instead (see cpu_baseline).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Mvis/s grid+degrid (full-pol AW; FP32 vs mixed vs learned) and % of roofline"
UNIT = "Mvis/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--time-samples", type=int, default=2000, help="scale the workload (2000 = full)")
    ap.add_argument("--no-variants", action="store_true", help="skip the BF16/FP16 table variants")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--subset", action="store_true",
                    help="profiling case: only the visibilities of one (PA, frequency) bin pair, with its "
                         "32 w-plane kernels (same per-bin density and tables, 1/32 of the memory)")
    ap.add_argument("--tune", default=None, help="tile,chunk,ctas_per_sm[,dg_tile[,grid_mode]] (skips the autotuner)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-surrogate comparison")
    ap.add_argument("--no-learned-degrid", action="store_true", help="skip the learned degridding comparison")
    ap.add_argument("--no-learned-full", action="store_true",
                    help="skip the full configuration-5 mosaic (7 fields x 10M visibilities)")
    ap.add_argument("--learned-inline-case", type=int, default=None, metavar="ENGINE",
                    help="only run the small inline-surrogate profiling case on engine 0 (mma.sync) or 1 (tcgen05)")
    ap.add_argument("--wproj-case", type=int, default=None, metavar="REPS",
                    help="only grid and degrid configuration 2 (Stokes-I w-projection, FP32 tables, region schedule "
                         "with planes 0-17) REPS times: the profiling case of that configuration")
    ap.add_argument("--learned-train-case", type=int, default=None, metavar="STEPS",
                    help="only run the small surrogate-training profiling case for STEPS steps")
    ap.add_argument("--no-clean", action="store_true", help="skip the Cotton-Schwab cleaning measurement")
    ap.add_argument("--no-mosaic", action="store_true", help="skip the mosaic measurements")
    ap.add_argument("--no-baselines", action="store_true", help="skip the per-baseline kernel measurement")
    ap.add_argument("--no-wproj", action="store_true", help="skip the configuration 2 / 4 measurement")
    ap.add_argument("--uvmosaic-fraction", type=float, default=0.1,
                    help="fraction of each mosaic field's visibilities in the UV/image-domain comparison")
    ap.add_argument("--clean-major", type=int, default=3, help="major cycles of the cleaning measurement")
    ap.add_argument("--learned-steps", type=int, default=8000)
    ap.add_argument("--learned-fraction", type=float, default=0.1,
                    help="fraction of the mosaic field's visibilities gridded by both kernel paths")
    return ap.parse_args()


# ----------------------------------------------------------------------------- workload
def workload(time_samples: int, subset: bool = False):
    from paper_2206_15117_gb300 import synthetic as sy
    ob = sy.observation(3, time_samples=time_samples)
    if subset:
        a, f = 3, 1
        keep = np.flatnonzero((ob.pa_bin[ob.row_of_vis] == a) & (ob.fbin[ob.chan_of_vis] == f))
        ob = sy.Observation(**{**ob.__dict__, "row_of_vis": ob.row_of_vis[keep], "chan_of_vis": ob.chan_of_vis[keep],
                               "pa_bin": np.zeros_like(ob.pa_bin), "fbin": np.zeros_like(ob.fbin),
                               "pa_centres": ob.pa_centres[a:a + 1], "fbin_freqs": ob.fbin_freqs[f:f + 1]})
    g = sy.grid_geometry(3)
    nw = 32
    kw = sy.config_spec(3, ob)
    assert kw["nw"] == nw and kw["N"] == g["N"]
    return ob, kw


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.path = tempfile.mktemp(prefix="clocks_", suffix=".csv")
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() in ("active", "1", "0x1"):
                    reasons.add(name)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


# ----------------------------------------------------------------------------- CPU oracle sample
# Size of the oracle's sample of the workload: complex MACs of one grid +
# degrid pass (about 16 s on one Grace core, 1 s on 16).  Fixed, so that the
# cpu_baseline leg and the reference arm time the same visibilities.
ORACLE_SAMPLE_MACS = 1.1e10


def oracle_sample(ob, kw, budget_macs: float = ORACLE_SAMPLE_MACS, seed: int = 5):
    """A fixed sample of the workload for the FP64 oracle: every visibility
    of four seeded bins (each capped at a quarter of the MAC budget), with the
    oracle's own kernels for them."""
    from oracle import core as oc
    from paper_2206_15117_gb300 import synthetic as sy
    rng = np.random.default_rng(seed)
    sub = np.sort(rng.choice(ob.nvis, size=min(ob.nvis, 2_000_000), replace=False))
    spec = oc.KernelSpec(**kw)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis[sub], ob.chan_of_vis[sub], ob.freq, ob.pa_bin, ob.fbin)
    ok = co.valid == 1
    bins, counts = np.unique(co.bin[ok], return_counts=True)
    pick = rng.choice(bins, size=min(4, bins.size), replace=False, p=counts / counts.sum())
    sup = np.array(spec.supports)
    per = spec.npa * spec.nfb
    S2_all = float(np.mean(sup[co.bin[ok] // per].astype(np.float64) ** 2))
    # every visibility of the picked bins: the rows/channels of their (PA, frequency)
    # bin pairs, then the oracle's own coordinates
    sel = []
    # grid + degrid cost 2 x 16 S^2 complex MACs per visibility
    for b in pick:
        a_, f_ = (b // spec.nfb) % spec.npa, b % spec.nfb
        cand = np.flatnonzero((ob.pa_bin[ob.row_of_vis] == a_) & (ob.fbin[ob.chan_of_vis] == f_))
        c2 = oc.coords(spec, ob.uvw, ob.row_of_vis[cand], ob.chan_of_vis[cand], ob.freq, ob.pa_bin, ob.fbin)
        idx = cand[(c2.valid == 1) & (c2.bin == b)]
        S = sup[b // per]
        cap = max(16, int(budget_macs / len(pick) / (32.0 * S * S)))
        sel.append(idx[:cap])
    keep = np.sort(np.concatenate(sel))
    rows, chans = ob.row_of_vis[keep], ob.chan_of_vis[keep]
    cos = oc.coords(spec, ob.uvw, rows, chans, ob.freq, ob.pa_bin, ob.fbin)
    kg = oc.make_kernels(oc.KernelSpec(**kw, role=oc.ROLE_GRID), bins=pick)
    kd = oc.make_kernels(oc.KernelSpec(**kw, role=oc.ROLE_DEGRID), bins=pick)
    vis = sy.random_vis(keep.size, 4, seed=seed + 1)
    model = sy.random_grid(4, kw["N"], seed=seed + 2).astype(np.complex128)
    S2_sample = float(np.mean(sup[cos.bin[cos.valid == 1] // (spec.npa * spec.nfb)].astype(np.float64) ** 2))
    return dict(co=cos, kg=kg, kd=kd, vis=vis, model=model, n=int(keep.size), bins=[int(b) for b in pick],
                S2_sample=S2_sample, S2_all=S2_all)


def oracle_step(smp):
    from oracle import core as oc
    t0 = time.perf_counter()
    oc.grid(smp["kg"], smp["co"], smp["vis"])
    oc.degrid(smp["kd"], smp["co"], smp["model"])
    return time.perf_counter() - t0


def oracle_step_parallel(smp, nthreads):
    """The same sample split into `nthreads` shards of visibilities, each gridded
    (into its own grid) and degridded by the unchanged oracle on its own thread
    (the oracle's C loops run without the interpreter lock): the host's cores
    working on the one sample."""
    import dataclasses
    from concurrent.futures import ThreadPoolExecutor
    from oracle import core as oc
    if smp.get("nshard") != nthreads:
        parts = np.array_split(np.arange(smp["n"]), nthreads)
        co = smp["co"]
        smp["shards"] = [(oc.Coords(**{f.name: getattr(co, f.name)[p] for f in dataclasses.fields(co)}),
                          np.ascontiguousarray(smp["vis"][p])) for p in parts if p.size]
        smp["nshard"] = nthreads

    def work(sh):
        oc.grid(smp["kg"], sh[0], sh[1])
        oc.degrid(smp["kd"], sh[0], smp["model"])

    with ThreadPoolExecutor(max_workers=nthreads) as ex:
        t0 = time.perf_counter()
        list(ex.map(work, smp["shards"]))
        return time.perf_counter() - t0


def host_cores():
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def oracle_mvis(smp, seconds):
    # scaled from the sample's mean S^2 to the workload's (the oracle's cost is
    # proportional to the taps per visibility)
    return smp["n"] / seconds / 1e6 * smp["S2_sample"] / smp["S2_all"]


def oracle_mvis_unscaled(smp, seconds):
    return smp["n"] / seconds / 1e6


def sample_text(smp, threads=1):
    return ("fixed sample: %d visibilities of bins %s of the same workload (mean S^2 %.0f vs %.0f for all); "
            "value scaled by that S^2 ratio, value_sample_unscaled the sample's own rate; FP64 C loops, %s" %
            (smp["n"], smp["bins"], smp["S2_sample"], smp["S2_all"],
             "one thread" if threads == 1 else "%d threads on disjoint shards of the sample" % threads))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    from oracle import build as ob_build
    ob_build.build()
    ob, kw = workload(args.time_samples, args.subset)
    nthr = host_cores()
    # the same fixed sample as the cpu_baseline leg of the GPU arm
    smp = oracle_sample(ob, kw)
    for _ in range(args.warmup):
        oracle_step_parallel(smp, nthr)
    ts = [oracle_step_parallel(smp, nthr) for _ in range(args.steps)]
    t = statistics.median(ts)
    val = oracle_mvis(smp, t)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ts) / len(ts),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(ob, kw, None),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": nthr, "kind": "oracle",
                             "sample": sample_text(smp, nthr),
                             "value_sample_unscaled": oracle_mvis_unscaled(smp, t)},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(ob, kw, info):
    cfg = {"workload": "full-pol AW grid+FFT+degrid, 4096^2 x 4 grid, 1024 bins (32 w x 8 PA x 4 freq), "
                       "supports 16-72, OS 8, 288 channels of uneven counts",
           "nvis": int(ob.nvis), "N": kw["N"], "npol": 4, "nbins": 32 * len(kw["pa"]) * len(kw["fbin_freqs"]),
           "OS": kw["OS"], "supports": list(kw["supports"]),
           "l2": "inputs larger than L2 (visibilities 2 GB, kernel tables 33 GB)",
           "weights": "natural: the timed steps pass no weight array (the weighted gridding call is timed "
                      "separately, weighted_grid)"}
    if info is not None:
        cfg.update({"nvalid": int(info.nvalid), "mean_taps": round(info.mean_taps, 1),
                    "tile": info.tile, "chunk": info.chunk})
    return cfg


# ----------------------------------------------------------------------------- configurations 2 and 4
def wproj_section(ctx, dev, args, stream):
    """Configuration 2 (Stokes-I w-projection: 20.16M visibilities, 2048^2,
    32 w planes, supports 8-64, OS 8) and configuration 4 (the same inputs
    with BF16 / FP16 kernel tables, FP32 products and accumulation): per
    storage, grid + degrid Mvis/s with the fastest gridding schedule of a
    few candidates timed on the full data, the roofline of each step, and
    the dirty image of each 16-bit form against the FP32 one (peak-relative
    max and RMS error, dynamic range)."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    ob = sy.observation(2)
    kw = sy.config_spec(2, ob)
    N = kw["N"]
    vd, keep = aw.device_observation(ob, dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    vis = torch.randn((ob.nvis, 1), dtype=torch.complex64, device=dev, generator=gen)
    model = torch.randn((1, N, N), dtype=torch.complex64, device=dev, generator=gen)
    out = torch.empty_like(vis)
    grid = torch.zeros((1, N, N), dtype=torch.complex64, device=dev)
    peak, _ = fp32_peak_tflops(dev.index or 0)
    cands = {"tiles": aw.aw_tune(32, 256, 4, 1024, aw.AW_GRID_TILES, 0),
             "offsets": aw.aw_tune(32, 256, 4, 256, aw.AW_GRID_OFFSETS, 0),
             "hybrid/16": aw.aw_tune(32, 256, 2, 256, aw.AW_GRID_HYBRID, 16),
             "hybrid/24": aw.aw_tune(32, 256, 2, 256, aw.AW_GRID_HYBRID, 24),
             # the region kernel for supports 16-48 (8 and wider on OFFSETS beside it)
             "region": aw.aw_tune(32, 256, 2, 1024, aw.AW_GRID_REGION, 0),
             "region/14": aw.aw_tune(32, 256, 2, 1024, aw.AW_GRID_REGION, 14),
             "region/18": aw.aw_tune(32, 256, 2, 1024, aw.AW_GRID_REGION, 18),
             "region/22": aw.aw_tune(32, 256, 2, 1024, aw.AW_GRID_REGION, 22)}

    def ms_of(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res, images = {}, {}
    for name, stg in (("fp32", aw.AW_STORAGE_FP32), ("bf16", aw.AW_STORAGE_BF16), ("fp16", aw.AW_STORAGE_FP16)):
        kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID, storage=stg)
        kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID, storage=stg)
        grid_ms, plans = {}, {}
        for cname, t in cands.items():
            plans[cname] = aw.aw_plan_create(ctx, vd, kg, tune=t)
            p_ = plans[cname]

            def g_():
                grid.zero_()
                aw.aw_grid_batched(ctx, p_, kg, vis, None, grid)
            grid_ms[cname] = ms_of(g_)
        best = min(grid_ms, key=grid_ms.get)
        plan = plans[best]
        info = aw.aw_plan_query(plan)
        d_ms = ms_of(lambda: aw.aw_degrid(ctx, plan, kd, model, out))
        st = None
        grid.zero_()
        st = aw.aw_grid_batched(ctx, plan, kg, vis, None, grid, want_stats=True)
        img = torch.empty((1, N, N), dtype=torch.float32, device=dev)
        aw.aw_fft_to_image(ctx, kg, grid.clone(), st.weight_sum, img)
        images[name] = img
        flops = 8.0 * info.mean_taps * info.nvalid     # one complex MAC (8 flop) per tap
        mean_taps = float(info.mean_taps)
        g_ms = grid_ms[best]
        res[name] = {"mvis_s": ob.nvis / ((g_ms + d_ms) / 1e3) / 1e6, "grid_ms": g_ms, "degrid_ms": d_ms,
                     "grid_schedule": best, "grid_ms_by_schedule": grid_ms,
                     "roofline": {"grid": {"bound": "alu", "achieved": flops / (g_ms / 1e3) / 1e12, "peak": peak,
                                           "unit": "TFLOP/s", "frac": flops / (g_ms / 1e3) / 1e12 / peak},
                                  "degrid": {"bound": "alu", "achieved": flops / (d_ms / 1e3) / 1e12, "peak": peak,
                                             "unit": "TFLOP/s", "frac": flops / (d_ms / 1e3) / 1e12 / peak}},
                     "table_bytes": int(aw.aw_kernel_set_info(kg).bytes)}
        del plans, plan, kg, kd
        torch.cuda.empty_cache()
    # configuration 4's image error: each 16-bit form against the FP32 path
    # (the FP32 path itself is held to 1e-5 of the FP64 oracle by the tests),
    # over the inner half of the Stokes I image
    q = slice(N // 4, 3 * N // 4)
    ref = images["fp32"][0, q, q]
    pk = float(ref.abs().max())
    for name in ("bf16", "fp16"):
        d = images[name][0, q, q] - ref
        res[name]["dirty_image_vs_fp32"] = {"max_rel_peak": float(d.abs().max()) / pk,
                                            "rms_rel_peak": float(d.pow(2).mean().sqrt()) / pk}
    info_all = {"workload": "configuration 2: Stokes-I w-projection, %d visibilities (2000 samples x 16 channels "
                            "1.2-1.5 GHz), 2048^2, 32 w planes, supports 8-64, OS 8; configuration 4: the same "
                            "inputs with BF16 / FP16 kernel tables" % ob.nvis,
                "nvis": int(ob.nvis), "mean_taps": mean_taps}
    return {**info_all, **res}


# ----------------------------------------------------------------------------- learned surrogate
def clean_section(ctx, dev, args, ob, kw, plan, kg, kd, stream):
    """Cotton-Schwab cleaning (aw_clean) on the bench workload.  The observed
    visibilities are the library's own prediction of the generator's point
    sources (Stokes I, Q, U, V = 1, 0.05, -0.03, 0.005 of the flux), so the
    loop must converge to them; timed with CUDA events.  The Hogbom minor
    cycle is also timed alone, beside the oracle's FP32 minor cycle on the
    same image."""
    import torch
    from oracle import clean as ocl
    from paper_2206_15117_gb300 import aw
    N = kw["N"]
    dl = kw["dl"]
    src = np.asarray(ob.sources)
    qx = np.clip(np.rint(src[:, 0] / dl).astype(int) + N // 2, N // 4, 3 * N // 4 - 1)
    qy = np.clip(np.rint(src[:, 1] / dl).astype(int) + N // 2, N // 4, 3 * N // 4 - 1)
    truth = np.zeros((4, N, N), np.float32)
    for k in range(len(src)):
        truth[:, qy[k], qx[k]] += np.float32(src[k, 2]) * np.array([1.0, 0.05, -0.03, 0.005], np.float32)
    t_dev = torch.as_tensor(truth, device=dev)
    g = torch.empty((4, N, N), dtype=torch.complex64, device=dev)
    aw.aw_image_to_grid(ctx, kd, t_dev, g)
    vis_obs = torch.empty((ob.nvis, 4), dtype=torch.complex64, device=dev)
    aw.aw_degrid(ctx, plan, kd, g, vis_obs)
    del g
    model = torch.empty((4, N, N), dtype=torch.float32, device=dev)
    resid = torch.empty_like(model)
    psf = torch.empty((N, N), dtype=torch.float32, device=dev)
    cfg = dict(n_major=args.clean_major, max_minor=2000, gain=0.1, threshold=0.002, cycle_factor=1.5,
               patch_half=256)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    rep = aw.aw_clean(ctx, plan, kg, kd, vis_obs, None, model, resid, psf, **cfg)
    b.record(stream)
    torch.cuda.synchronize()
    clean_ms = a.elapsed_time(b)
    m = model[0].cpu().numpy()
    flux_true = float(truth[0].sum())
    flux_at_src = float(sum(m[qy[k], qx[k]] for k in set(range(len(src)))))
    # the minor cycle alone, on the dirty image of the observation
    gd = torch.zeros((4, N, N), dtype=torch.complex64, device=dev)
    aw.aw_grid_batched(ctx, plan, kg, vis_obs, None, gd)
    dirty = torch.empty((4, N, N), dtype=torch.float32, device=dev)
    aw.aw_fft_to_image(ctx, kg, gd, float(rep.weight_sum), dirty)
    del gd
    dirty_host = dirty.cpu().numpy()
    psf_host = psf.cpu().numpy()
    win = ocl.default_window(N)
    m2 = torch.zeros_like(model)
    n_it = 1000
    torch.cuda.synchronize()
    a.record(stream)
    n_done = aw.aw_hogbom(ctx, dirty, psf, 0.1, 0.0, n_it, 256, win, m2)
    b.record(stream)
    torch.cuda.synchronize()
    hog_ms = a.elapsed_time(b)
    n_cpu = 20
    t0 = time.perf_counter()
    _, _, n_cpu_done = ocl.hogbom(dirty_host, psf_host, 0.1, 0.0, n_cpu, 256, win)
    cpu_s = time.perf_counter() - t0
    del vis_obs, model, resid, psf, dirty, m2
    torch.cuda.empty_cache()
    return {"workload": "the bench workload (%d visibilities, 4096^2 x 4) predicted from the generator's "
                        "%d point sources; gain 0.1, cycle factor 1.5, PSF patch 513^2, threshold 2 mJy"
                        % (ob.nvis, len(src)),
            "ms_total": clean_ms, "n_major": rep.n_major, "n_minor": rep.n_minor,
            "ms_per_major_cycle": clean_ms / max(rep.n_major + 2, 1),
            "peak_first": rep.peak_first, "peak_last": rep.peak_last, "psf_sidelobe": rep.sidelobe,
            "stokes_i_flux_true": flux_true, "stokes_i_flux_on_source_pixels": flux_at_src,
            "hogbom_iterations_per_s": n_done / (hog_ms / 1e3), "hogbom_iterations": n_done,
            "oracle_hogbom_iterations_per_s": n_cpu_done / cpu_s,
            "note": "ms_per_major_cycle counts the PSF and final residual passes as cycles"}


def mosaic_section(ctx, dev, args, stream):
    """Image-domain mosaic round trip (Sec. 2.2) at the mosaic geometry of the
    learned-kernel workload: 7 hexagonal fields 1 deg apart at dec -45 deg,
    2048^2 x 4 Stokes planes over 3 deg each, into a 4096^2 common frame at the
    same pixel size; Airy power beams of a 12 m dish at 1.35 GHz.  Timed: the 7
    reprojections to the common frame (Keys cubic) and the Eq. 1 combination;
    then the 7 reprojections of the model back to the fields."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    Nf, Nm = 2048, 4096
    dl = math.radians(3.0) / Nf
    dec0 = math.radians(-45.0)
    ra0 = 1.0
    fields = []
    for (ex_deg, no_deg) in sy.mosaic_offsets():
        fields.append(aw.sky_frame(ra0 + math.radians(ex_deg) / math.cos(dec0), dec0 + math.radians(no_deg), dl, Nf))
    mframe = aw.sky_frame(ra0, dec0, dl, Nm)
    gen = torch.Generator(device=dev)
    gen.manual_seed(77)
    imgs = torch.randn((len(fields), 4, Nf, Nf), dtype=torch.float32, device=dev, generator=gen)
    # Airy power beams of each pointing on the common frame (flat-sky offsets)
    q = (torch.arange(Nm, device=dev, dtype=torch.float64) - Nm // 2) * dl
    lam = 299792458.0 / 1.35e9
    beams = torch.empty((len(fields), Nm, Nm), dtype=torch.float32, device=dev)
    from scipy.special import j1
    for f, (ex_deg, no_deg) in enumerate(sy.mosaic_offsets()):
        r = torch.hypot(q[None, :] - math.radians(ex_deg), q[:, None] - math.radians(no_deg))
        x = (math.pi * 12.0 / lam * r).cpu().numpy()
        e = np.where(x == 0, 1.0, 2.0 * j1(np.where(x == 0, 1.0, x)) / np.where(x == 0, 1.0, x))
        beams[f] = torch.as_tensor((e * e).astype(np.float32), device=dev)
    gam = torch.empty((Nm, Nm), dtype=torch.float32, device=dev)
    aw.mosaic_gamma(ctx, beams, 0.2, gam)
    onm = torch.empty((len(fields), 4, Nm, Nm), dtype=torch.float32, device=dev)
    mosaic = torch.empty((4, Nm, Nm), dtype=torch.float32, device=dev)
    back = torch.empty_like(imgs)

    def forward():
        for f, fr in enumerate(fields):
            aw.aw_reproject(ctx, imgs[f], fr, onm[f], mframe, aw.AW_INTERP_CUBIC)
        aw.aw_mosaic_combine(ctx, onm, beams, gam, mosaic)

    def backward():
        for f, fr in enumerate(fields):
            aw.aw_reproject(ctx, mosaic, mframe, back[f], fr, aw.AW_INTERP_CUBIC)

    res = {}
    for name, fn in (("forward", forward), ("backward", backward)):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / reps
    out_px_fwd = len(fields) * Nm * Nm
    out_px_bwd = len(fields) * Nf * Nf
    del imgs, beams, gam, onm, mosaic, back
    torch.cuda.empty_cache()
    return {"workload": "7 fields of 2048^2 x 4 (3 deg, hexagonal 1 deg apart, dec -45) <-> 4096^2 x 4 common frame, "
                        "Keys cubic",
            "ms_fields_to_mosaic_and_combine": res["forward"], "ms_mosaic_to_fields": res["backward"],
            "gpix_per_s_fields_to_mosaic": out_px_fwd / (res["forward"] / 1e3) / 1e9,
            "gpix_per_s_mosaic_to_fields": out_px_bwd / (res["backward"] / 1e3) / 1e9,
            "note": "a pixel = all 4 Stokes planes; FP64 position (3x3 rotation) and floor, FP32 weights and 4x4 interpolation"}


def baselines_section(ctx, dev, ob, kw, tune, vis, model, grid, vis_out, stream, averaged):
    """Per-baseline Mueller kernels on the bench workload: the 36 antennas in
    two types (two dish generations) with their own leakage terms, so 4
    baseline classes with their own kernels, M = J_ti kron conj(J_tj), instead
    of the baseline-averaged set.  Same visibilities, schedule and supports;
    4x the kernel tables.  Timed: aw_grid_batched and aw_degrid as in the
    main step."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    rng = np.random.default_rng(sy.BASE_SEED + 400)
    ant_type = np.zeros(36, np.uint8)
    ant_type[rng.permutation(36)[:18]] = 1
    type_leak = [(0.01 * np.exp(0.4j), 0.01 * np.exp(-1.3j)), (0.015 * np.exp(-0.7j), 0.012 * np.exp(2.1j))]
    rt = sy.row_antenna_types(36, ob.uvw.shape[0], ant_type)
    t0 = time.perf_counter()
    kg = aw.aw_make_kernels(ctx, **kw, type_leak=type_leak, role=aw.AW_ROLE_GRID)
    kd = aw.aw_make_kernels(ctx, **kw, type_leak=type_leak, role=aw.AW_ROLE_DEGRID)
    t_synth = time.perf_counter() - t0
    vd, keep = aw.device_observation(ob, dev, row_types=rt)
    t0 = time.perf_counter()
    plan = aw.aw_plan_create(ctx, vd, kg, tune=tune)
    t_plan = time.perf_counter() - t0
    info = aw.aw_kernel_set_info(kg)

    def step(ev=None):
        grid.zero_()
        if ev: ev[0].record(stream)
        aw.aw_grid_batched(ctx, plan, kg, vis, None, grid)
        if ev: ev[1].record(stream)
        aw.aw_degrid(ctx, plan, kd, model, vis_out)
        if ev: ev[2].record(stream)

    step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(3)]
    for e in evs:
        step(e)
    torch.cuda.synchronize()
    gm = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    dm = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    nvis = int(ob.nvis)
    out = {"workload": "bench workload with 2 antenna types (18 + 18 antennas): 4 baseline classes x 1024 bins, "
                       "FP32 tables",
           "classes": 4, "nbins": int(info.nbins), "table_bytes_per_set": int(info.bytes),
           "grid_ms": gm, "degrid_ms": dm, "mvis_s": nvis / ((gm + dm) / 1e3) / 1e6,
           "vs_baseline_averaged": (averaged["grid_ms"] + averaged["degrid_ms"]) / (gm + dm),
           "once_per_dataset_s": {"kernel_synthesis_grid_and_degrid": t_synth, "plan_sort": t_plan}}
    del kg, kd, plan, vd, keep
    torch.cuda.empty_cache()
    return out


def uvmosaic_section(ctx, dev, args, stream):
    """Image-domain against UV-domain mosaicing of the 7 hexagonal fields of the
    mosaic workload (Sec. 2.2), on the same visibilities (a seeded fraction of
    each field's 10M).  Image domain: each field gridded at its own phase centre
    on 2048^2 x 4 (3 deg; GRID kernels, 4 w planes, supports 8-32), imaged,
    reprojected to a 4096^2 common frame (Keys cubic) and combined with Eq. 1.
    UV domain: each field phase-rotated to the mosaic centre and gridded onto
    one 4096^2 x 4 grid (6 deg) with beam-weighted kernels centred on its
    pointing; the larger field doubles the uv extent of the beam and w kernels,
    so the supports are doubled (16-64); one FFT, then gamma.  Kernel
    synthesis, plans and beams are prepared before the timed regions."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    g = sy.grid_geometry(5)
    Nf, dl = g["N"], g["dl"]
    Nm = 2 * Nf
    dec0 = math.radians(sy.DEC_DEG)
    ra0 = 1.0
    centre = (ra0, dec0)
    fr_m = aw.sky_frame(ra0, dec0, dl, Nm)
    offs = sy.mosaic_offsets()
    fields = []
    gen = torch.Generator(device=dev)
    gen.manual_seed(91)
    nvis_total = 0
    for f, (ex_deg, no_deg) in enumerate(offs):
        ob = sy.observation(5, field=f, vis_fraction=args.uvmosaic_fraction)
        pc = (ra0 + math.radians(ex_deg) / math.cos(dec0), dec0 + math.radians(no_deg))
        # pointing of field f in the common frame
        B0 = np.array([[-math.sin(ra0), math.cos(ra0), 0.0],
                       [-math.sin(dec0) * math.cos(ra0), -math.sin(dec0) * math.sin(ra0), math.cos(dec0)]])
        sv = np.array([math.cos(pc[1]) * math.cos(pc[0]), math.cos(pc[1]) * math.sin(pc[0]), math.sin(pc[1])])
        lp, mp = B0 @ sv
        base = dict(OS=8, W=7.0, npol=4, nw=4, w_max=ob.w_max, pa=list(ob.pa_centres), fbin_freqs=list(ob.fbin_freqs),
                    dish_d=12.0, d_xy=0.01 * np.exp(0.4j), d_yx=0.01 * np.exp(-1.3j), eps=0.2)
        kimg = aw.aw_make_kernels(ctx, N=Nf, dl=dl, supports=[8, 16, 24, 32], **base)
        kuv = aw.aw_make_kernels(ctx, N=Nm, dl=dl, supports=[16, 32, 48, 64], role=aw.AW_ROLE_BEAM,
                                 point_l=float(lp), point_m=float(mp), **base)
        vd, keep = aw.device_observation(ob, dev)
        plan_img = aw.aw_plan_create(ctx, vd, kimg)
        vis = torch.randn((ob.nvis, 4), dtype=torch.complex64, device=dev, generator=gen)
        vrot = torch.empty_like(vis)
        uvw_rot = torch.empty((ob.uvw.shape[0], 3), dtype=torch.float64, device=dev)
        aw.aw_phase_rotate(ctx, vd, uvw_rot, vis, vrot, pc, centre)
        vd_uv, keep_uv = aw.device_observation(ob, dev)
        vd_uv.uvw = uvw_rot.data_ptr()
        plan_uv = aw.aw_plan_create(ctx, vd_uv, kuv)
        fields.append(dict(frame=aw.sky_frame(pc[0], pc[1], dl, Nf), kimg=kimg, kuv=kuv, plan_img=plan_img,
                           plan_uv=plan_uv, vd=vd, keep=(keep, keep_uv, uvw_rot), vis=vis, vrot=vrot,
                           pc=pc, nvis=ob.nvis))
        nvis_total += ob.nvis
    # Airy power beams of the pointings on the common frame (flat-sky offsets), gamma
    q = (torch.arange(Nm, device=dev, dtype=torch.float64) - Nm // 2) * dl
    lam = 299792458.0 / 1.35e9
    from scipy.special import j1
    beams = torch.empty((len(offs), Nm, Nm), dtype=torch.float32, device=dev)
    for f, (ex_deg, no_deg) in enumerate(offs):
        r = torch.hypot(q[None, :] - math.radians(ex_deg), q[:, None] - math.radians(no_deg))
        x = (math.pi * 12.0 / lam * r).cpu().numpy()
        e = np.where(x == 0, 1.0, 2.0 * j1(np.where(x == 0, 1.0, x)) / np.where(x == 0, 1.0, x))
        beams[f] = torch.as_tensor((e * e).astype(np.float32), device=dev)
    gam = torch.empty((Nm, Nm), dtype=torch.float32, device=dev)
    aw.mosaic_gamma(ctx, beams, 0.2, gam)
    grid_f = torch.zeros((4, Nf, Nf), dtype=torch.complex64, device=dev)
    img_f = torch.empty((4, Nf, Nf), dtype=torch.float32, device=dev)
    onm = torch.empty((len(offs), 4, Nm, Nm), dtype=torch.float32, device=dev)
    mosaic = torch.empty((4, Nm, Nm), dtype=torch.float32, device=dev)
    grid_m = torch.zeros((4, Nm, Nm), dtype=torch.complex64, device=dev)
    img_m = torch.empty((4, Nm, Nm), dtype=torch.float32, device=dev)
    ones = torch.ones((1, Nm, Nm), dtype=torch.float32, device=dev)

    def image_domain():
        for f, fd in enumerate(fields):
            grid_f.zero_()
            aw.aw_grid_batched(ctx, fd["plan_img"], fd["kimg"], fd["vis"], None, grid_f)
            aw.aw_fft_to_image(ctx, fd["kimg"], grid_f, float(fd["nvis"]), img_f)
            aw.aw_reproject(ctx, img_f, fd["frame"], onm[f], fr_m, aw.AW_INTERP_CUBIC)
        aw.aw_mosaic_combine(ctx, onm, beams, gam, mosaic)

    def uv_domain():
        grid_m.zero_()
        for fd in fields:
            aw.aw_phase_rotate(ctx, fd["vd"], None, fd["vis"], fd["vrot"], fd["pc"], centre)
            aw.aw_grid_batched(ctx, fd["plan_uv"], fd["kuv"], fd["vrot"], None, grid_m)
        aw.aw_fft_to_image(ctx, fields[0]["kuv"], grid_m, float(nvis_total), img_m)
        aw.aw_mosaic_combine(ctx, img_m[None], ones, gam, mosaic)

    res = {}
    for name, fn in (("image_domain", image_domain), ("uv_domain", uv_domain)):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        res[name] = a.elapsed_time(b) / 3
    out = {"workload": "7 hexagonal fields, %d visibilities in all; image domain 2048^2 x 4 per field + "
                       "reprojection to 4096^2; UV domain one 4096^2 x 4 grid" % nvis_total,
           "ms_image_domain": res["image_domain"], "ms_uv_domain": res["uv_domain"],
           "mvis_s_image_domain": nvis_total / (res["image_domain"] / 1e3) / 1e6,
           "mvis_s_uv_domain": nvis_total / (res["uv_domain"] / 1e3) / 1e6,
           "table_bytes_image_domain": int(sum(aw.aw_kernel_set_info(fd["kimg"]).bytes for fd in fields)),
           "table_bytes_uv_domain": int(sum(aw.aw_kernel_set_info(fd["kuv"]).bytes for fd in fields))}
    del fields, beams, gam, onm, mosaic, grid_m, img_m, grid_f, img_f, ones
    torch.cuda.empty_cache()
    return out


def learned_section(ctx, dev, args):
    """The learned AW-kernel surrogate on the mosaic workload: 4 x 128 SIREN
    trained on the exact full-pol kernels of the configuration-2 bins (32 w
    planes, supports 8-64, OS 8) x 8 PA x 4 frequency bins, then gridding one
    mosaic field (2048^2, its own phase centre) with the network evaluated
    inline and with the exact tables, on the same visibilities; plus the Eq. 1
    weighting of the 7 hexagonal fields."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    stream = torch.cuda.current_stream()
    ob = sy.observation(5, field=0)
    g = sy.grid_geometry(5)
    kw = sy.config_spec(5, ob)
    t0 = time.perf_counter()
    exact = aw.aw_make_kernels(ctx, **kw)
    t_synth = time.perf_counter() - t0
    # 4x finer w sampling: the training set of the network and the reference
    # the two gridding paths are compared against
    kw_fine = {**kw, "nw": 128, "supports": sy.w_supports(128)}
    fine = aw.aw_make_kernels(ctx, **kw_fine)
    S0 = kw["supports"][0]
    k0 = torch.empty(kw["OS"] ** 2 * S0 * S0 * 16, dtype=torch.complex64, device=dev)
    aw.aw_kernel_set_export(exact, 0, k0)
    kmax = float(k0.abs().max())
    pa = np.asarray(kw["pa"])
    chi_c = float(pa.mean())
    chi_h = float(np.abs(pa - chi_c).max()) + 1e-3
    # offsets normalised by the support of the 32-plane layout the network is used with
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, D=1.0,
                                 norm_supports=kw["supports"], w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                                 chi_c=chi_c, chi_h=chi_h, out_scale=kmax, seed=17)
    rep = aw.aw_surrogate_train(ctx, sur, fine, steps=args.learned_steps, batch=65536, lr=3e-4, lr_final=6e-6,
                                seed=5)
    reject = 0.05
    t0 = time.perf_counter()
    tabs, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=reject)
    t_tables = time.perf_counter() - t0
    del tabs
    nw = kw["nw"]
    per = len(kw["pa"]) * len(kw["fbin_freqs"])
    plane_err = [float(err[p * per:(p + 1) * per].max()) for p in range(nw)]
    # the same visibilities through both paths
    rng = np.random.default_rng(11)
    keep = np.sort(rng.choice(ob.nvis, size=max(1, int(ob.nvis * args.learned_fraction)), replace=False))
    obs = sy.Observation(**{**ob.__dict__, "row_of_vis": ob.row_of_vis[keep], "chan_of_vis": ob.chan_of_vis[keep]})
    vd, hold = aw.device_observation(obs, dev)
    plan = aw.aw_plan_create(ctx, vd, exact, tune=aw.aw_tune(64, 128, 4, 0))
    info = aw.aw_plan_query(plan)
    gen = torch.Generator(device=dev)
    gen.manual_seed(55)
    vis = torch.randn((obs.nvis, 4), dtype=torch.complex64, device=dev, generator=gen)
    N = kw["N"]
    g_ex = torch.zeros((4, N, N), dtype=torch.complex64, device=dev)
    g_le = torch.zeros_like(g_ex)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def run_exact():
        g_ex.zero_()
        aw.aw_grid_batched(ctx, plan, exact, vis, None, g_ex)

    def run_learned():
        g_le.zero_()
        aw.aw_grid_learned(ctx, plan, sur, exact, vis, None, g_le)

    img_ex = torch.empty((4, N, N), dtype=torch.float32, device=dev)
    img_le = torch.empty_like(img_ex)
    q = slice(N // 4, 3 * N // 4)

    # reference: the exact kernels at 4x finer w sampling (128 planes)
    plan_f = aw.aw_plan_create(ctx, vd, fine, tune=aw.aw_tune(64, 128, 4, 0))
    info_f = aw.aw_plan_query(plan_f)
    g_ref = torch.zeros_like(g_ex)
    aw.aw_grid_batched(ctx, plan_f, fine, vis, None, g_ref)
    img_ref = torch.empty_like(img_ex)
    aw.aw_fft_to_image(ctx, fine, g_ref, float(info_f.nvalid), img_ref)
    ref = img_ref[:, q, q]
    ref_norm = torch.linalg.vector_norm(ref)

    def err_vs_ref(g, kset):
        img = torch.empty_like(img_ex)
        aw.aw_fft_to_image(ctx, kset, g.clone(), float(info.nvalid), img)
        d = (img - img_ref)[:, q, q]
        return (float(torch.linalg.vector_norm(d) / ref_norm),
                float(ref[0].abs().max() / (d[0].pow(2).mean().sqrt() + 1e-30)))

    ms_ex = timed(run_exact)
    ex_err, ex_dr = err_vs_ref(g_ex, exact)
    # with the per-w-plane rejection of the tables call above
    ms_le = timed(run_learned, reps=1)
    img_err, dr = err_vs_ref(g_le, exact)
    # the network inline on every plane (no rejection): its own speed and error
    tabs2, _, _ = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=1e9)
    del tabs2
    ms_mlp = timed(run_learned, reps=1)
    # the same inline evaluation on the older tensor-core engine (mma.sync), for comparison
    aw.aw_surrogate_set_engine(sur, aw.AW_ENGINE_MMA_SYNC)
    ms_mlp_sync = timed(run_learned, reps=1)
    aw.aw_surrogate_set_engine(sur, aw.AW_ENGINE_TCGEN05)
    run_learned()
    mlp_err, mlp_dr = err_vs_ref(g_le, exact)
    points = float(info.mean_taps) * info.nvalid
    mlp_flops = points * 2.0 * (5 * 128 + 3 * 128 * 128 + 128 * 32)
    # generalisation between training samples: kernel error on an exact set
    # sampled at OS 7 (offsets off the OS 8 training lattice) at the 32 plane
    # centres (between the 128 training planes)
    held = aw.aw_make_kernels(ctx, **{**kw, "OS": 7})
    tabs3, err3, _ = aw.aw_surrogate_tables(ctx, sur, held, reject_rel=1e9)
    del tabs3, held
    plane_err_held = [float(err3[p * per:(p + 1) * per].max()) for p in range(nw)]
    # Eq. 1 over the 7 hexagonal fields on a common 2048^2 frame (Airy power beams)
    Nm = 2048
    dlm = math.radians(4.0) / Nm
    yy, xx = np.mgrid[0:Nm, 0:Nm]
    beams = []
    lam = 299792458.0 / 1.35e9
    from scipy.special import j1
    for (ex_deg, no_deg) in sy.mosaic_offsets():
        r = np.hypot((xx - Nm // 2) * dlm - math.radians(ex_deg), (yy - Nm // 2) * dlm - math.radians(no_deg))
        x = math.pi * 12.0 * r / lam
        E = np.where(x == 0, 1.0, 2.0 * j1(np.where(x == 0, 1.0, x)) / np.where(x == 0, 1.0, x))
        beams.append((E * E).astype(np.float32))
    B = torch.as_tensor(np.stack(beams), device=dev)
    gam = torch.empty((Nm, Nm), dtype=torch.float32, device=dev)
    ms_gamma = timed(lambda: aw.mosaic_gamma(ctx, B, 0.2, gam), reps=10)
    net_bytes = aw.aw_surrogate_nparams(sur) * 2
    # configuration 5 in full: every visibility of the 7 hexagonal fields
    # (10M each), each field gridded onto its own 2048^2 x 4 grid with its own
    # exact tables, with the network inline (per-plane rejection against that
    # field's tables, and every plane learned), and with the exact tables
    full = None
    if not args.no_learned_full:
        del g_ref, plan_f
        torch.cuda.empty_cache()
        tot = {"nvis": 0, "exact_ms": 0.0, "learned_rejection_ms": 0.0, "learned_all_ms": 0.0,
               "rejected_bins": 0, "nbins": 0}
        per_field = []
        for f in range(len(sy.mosaic_offsets())):
            obf = sy.observation(5, field=f)
            kwf = sy.config_spec(5, obf)
            exf = aw.aw_make_kernels(ctx, **kwf)
            vdf, holdf = aw.device_observation(obf, dev)
            pf = aw.aw_plan_create(ctx, vdf, exf, tune=aw.aw_tune(64, 128, 2, 1024, aw.AW_GRID_REGION, 0))
            genf = torch.Generator(device=dev)
            genf.manual_seed(100 + f)
            vf = torch.randn((obf.nvis, 4), dtype=torch.complex64, device=dev, generator=genf)
            gf = torch.zeros((4, N, N), dtype=torch.complex64, device=dev)

            def ex_():
                gf.zero_()
                aw.aw_grid_batched(ctx, pf, exf, vf, None, gf)

            def le_():
                gf.zero_()
                aw.aw_grid_learned(ctx, pf, sur, exf, vf, None, gf)
            t_ex = timed(ex_, reps=3)
            tb, errf, nrejf = aw.aw_surrogate_tables(ctx, sur, exf, reject_rel=reject)
            del tb
            t_rej = timed(le_, reps=1)
            tb, _, _ = aw.aw_surrogate_tables(ctx, sur, exf, reject_rel=1e9)
            del tb
            t_all = timed(le_, reps=1)
            per_field.append({"field": f, "nvis": int(obf.nvis), "exact_ms": t_ex, "learned_rejection_ms": t_rej,
                              "learned_all_ms": t_all, "rejected_bins": int(nrejf)})
            tot["nvis"] += int(obf.nvis)
            tot["exact_ms"] += t_ex
            tot["learned_rejection_ms"] += t_rej
            tot["learned_all_ms"] += t_all
            tot["rejected_bins"] += int(nrejf)
            tot["nbins"] += int(len(errf))
            del exf, vdf, holdf, pf, vf, gf
            torch.cuda.empty_cache()
        full = {"workload": "configuration 5: 7 hexagonal fields 1 deg apart, every visibility (%d), each on "
                            "its own 2048^2 x 4 grid with its own exact tables (1024 bins, supports 8-64, OS 8)"
                            % tot["nvis"],
                "mvis_s_exact_tables": tot["nvis"] / (tot["exact_ms"] / 1e3) / 1e6,
                "mvis_s_learned_with_rejection": tot["nvis"] / (tot["learned_rejection_ms"] / 1e3) / 1e6,
                "mvis_s_learned_inline_all_planes": tot["nvis"] / (tot["learned_all_ms"] / 1e3) / 1e6,
                "rejected_bins": tot["rejected_bins"], "nbins": tot["nbins"], "per_field": per_field}
    degrid = None
    if not args.no_learned_degrid:
        del g_ex, g_le, fine
        if full is None:
            del g_ref, plan_f
        torch.cuda.empty_cache()
        degrid = learned_degrid(ctx, dev, args, kw, kw_fine, vd, obs, stream, timed, kmax, chi_c, chi_h)
    return {"workload": "mosaic field 0 of 7 (hexagonal, 1 deg), 2048^2 x 4, 1024 bins (32 w x 8 PA x 4 freq), "
                        "supports 8-64, OS 8; %d of %d visibilities" % (obs.nvis, ob.nvis),
            "mvis_s_learned_with_rejection": obs.nvis / (ms_le / 1e3) / 1e6,
            "mvis_s_learned_inline_all_planes": obs.nvis / (ms_mlp / 1e3) / 1e6,
            "mvis_s_exact_tables": obs.nvis / (ms_ex / 1e3) / 1e6,
            "grid_ms_learned_with_rejection": ms_le, "grid_ms_learned_inline_all_planes": ms_mlp,
            "grid_ms_exact": ms_ex,
            "inline_mlp_points": points, "inline_engine": "tcgen05 (FP16 operands, FP32 accumulators in TMEM)",
            "inline_mlp_tflops": mlp_flops / (ms_mlp / 1e3) / 1e12,
            "inline_mlp_roofline": {"bound": "tensor", "achieved": mlp_flops / (ms_mlp / 1e3) / 1e12,
                                    "peak": bf16_burst(), "unit": "TFLOP/s",
                                    "frac": (mlp_flops / (ms_mlp / 1e3) / 1e12) / bf16_burst() if bf16_burst() else None,
                                    "peak_source": "measured dense bf16 burst (MEASURED_PEAKS.json); dense FP16 "
                                                   "has the same nominal tensor rate",
                                    "note": "the inline step also runs layer 1 and the sines on the CUDA cores and "
                                            "the gridding atomics"},
            "grid_ms_learned_inline_all_planes_mma_sync": ms_mlp_sync,
            "inline_mlp_tflops_mma_sync": mlp_flops / (ms_mlp_sync / 1e3) / 1e12,
            "reference": "exact kernels at 128 w planes (4x finer); image errors over the inner half, Stokes I-V",
            "dirty_image_rel_err_exact_32_planes_vs_ref": ex_err, "dynamic_range_exact_32_planes": ex_dr,
            "dirty_image_rel_err_learned_with_rejection_vs_ref": img_err, "dynamic_range_learned_with_rejection": dr,
            "dirty_image_rel_err_learned_all_planes_vs_ref": mlp_err, "dynamic_range_learned_all_planes": mlp_dr,
            "train": {"steps": rep.steps, "batch": 65536, "seconds": rep.seconds, "loss_first": rep.loss_first,
                      "loss_last": rep.loss_last, "set": "exact kernels at 128 w planes x 8 PA x 4 freq",
                      "engine": "tcgen05 kind::f16 (FP16 operands, FP32 accumulators and master weights)"},
            "kernel_rel_l2_per_w_plane": [round(e, 4) for e in plane_err],
            "kernel_rel_l2_per_w_plane_held_out_os7": [round(e, 4) for e in plane_err_held],
            "reject_threshold": reject, "rejected_bins": int(nrej), "nbins": int(len(err)),
            "network_bytes_fp16": int(net_bytes), "exact_table_bytes": int(aw.aw_kernel_set_info(exact).bytes),
            "exact_synthesis_s": t_synth, "surrogate_tables_s": t_tables,
            "mosaic_gamma_ms_7x2048^2": ms_gamma, "degrid": degrid, "mosaic_full": full}


def learned_degrid(ctx, dev, args, kw, kw_fine, vd, obs, stream, timed, kmax, chi_c, chi_h):
    """Degridding with the surrogate inline on the same field: a second network
    trained on the exact degridding kernels at 128 w planes, then the model
    grid of a point-source sky predicted inline (per-plane rejection, and
    every plane learned) and with the exact 32-plane tables; errors of the
    predicted visibilities against the exact 128-plane prediction."""
    import torch
    from paper_2206_15117_gb300 import aw
    exact = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    fine = aw.aw_make_kernels(ctx, **kw_fine, role=aw.AW_ROLE_DEGRID)
    S0 = kw["supports"][0]
    k0 = torch.empty(kw["OS"] ** 2 * S0 * S0 * 16, dtype=torch.complex64, device=dev)
    aw.aw_kernel_set_export(exact, 0, k0)
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, D=1.0,
                                 norm_supports=kw["supports"], w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                                 chi_c=chi_c, chi_h=chi_h, out_scale=float(k0.abs().max()), seed=18)
    rep = aw.aw_surrogate_train(ctx, sur, fine, steps=args.learned_steps, batch=65536, lr=3e-4, lr_final=6e-6,
                                seed=6)
    tabs, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=0.05)
    del tabs
    plan = aw.aw_plan_create(ctx, vd, exact, tune=aw.aw_tune(64, 128, 4, 0))
    plan_f = aw.aw_plan_create(ctx, vd, fine, tune=aw.aw_tune(64, 128, 4, 0))
    # a point-source model: 40 sources of 0.1-1 Jy in Stokes I with 5 % Q, U
    N = kw["N"]
    rng = np.random.default_rng(21)
    img = np.zeros((4, N, N), np.float32)
    qx, qy = rng.integers(N // 4, 3 * N // 4, 40), rng.integers(N // 4, 3 * N // 4, 40)
    flux = rng.uniform(0.1, 1.0, 40)
    img[0, qy, qx] = flux
    img[1, qy, qx] = 0.05 * flux
    img[2, qy, qx] = -0.05 * flux
    model = torch.empty((4, N, N), dtype=torch.complex64, device=dev)
    aw.aw_image_to_grid(ctx, exact, torch.as_tensor(img, device=dev), model)
    out_ref = torch.empty((obs.nvis, 4), dtype=torch.complex64, device=dev)
    aw.aw_degrid(ctx, plan_f, fine, model, out_ref)
    out = torch.empty_like(out_ref)
    ref_norm = torch.linalg.vector_norm(out_ref)

    def rel():
        return float(torch.linalg.vector_norm(out - out_ref) / ref_norm)

    ms_ex = timed(lambda: aw.aw_degrid(ctx, plan, exact, model, out))
    e_ex = rel()
    ms_rej = timed(lambda: aw.aw_degrid_learned(ctx, plan, sur, exact, model, out), reps=1)
    e_rej = rel()
    tabs2, _, _ = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=1e9)
    del tabs2
    ms_all = timed(lambda: aw.aw_degrid_learned(ctx, plan, sur, exact, model, out), reps=1)
    e_all = rel()
    n = obs.nvis
    del exact, fine, plan, plan_f, model, out, out_ref
    torch.cuda.empty_cache()
    return {"mvis_s_exact_tables": n / (ms_ex / 1e3) / 1e6, "mvis_s_learned_with_rejection": n / (ms_rej / 1e3) / 1e6,
            "mvis_s_learned_inline_all_planes": n / (ms_all / 1e3) / 1e6,
            "degrid_ms_exact": ms_ex, "degrid_ms_learned_with_rejection": ms_rej,
            "degrid_ms_learned_inline_all_planes": ms_all,
            "reference": "exact degridding kernels at 128 w planes; relative L2 error of the predicted visibilities "
                         "of a 40-source model",
            "vis_rel_err_exact_32_planes": e_ex, "vis_rel_err_learned_with_rejection": e_rej,
            "vis_rel_err_learned_all_planes": e_all, "rejected_bins": int(nrej), "nbins": int(len(err)),
            "train": {"steps": rep.steps, "seconds": rep.seconds, "loss_first": rep.loss_first,
                      "loss_last": rep.loss_last, "set": "exact degridding kernels at 128 w planes x 8 PA x 4 freq"}}


# ----------------------------------------------------------------------------- GPU arm
def wproj_case(reps: int):
    """Configuration 2 for profiling: 20.16M Stokes-I visibilities, 2048^2, 32 w planes (supports 8-64),
    OS 8, FP32 tables; the region schedule with planes 0-17 on the region kernel (the bench's choice for
    this configuration); one untimed grid + degrid, then `reps` timed ones."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import build as awbuild
    from paper_2206_15117_gb300 import synthetic as sy
    awbuild.build()
    ctx = aw.aw_create(0)
    dev = torch.device("cuda", 0)
    ob = sy.observation(2)
    kw = sy.config_spec(2, ob)
    N = kw["N"]
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    vd, keep = aw.device_observation(ob, dev)
    plan = aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(32, 256, 2, 1024, aw.AW_GRID_REGION, 18))
    gen = torch.Generator(device=dev)
    gen.manual_seed(2)
    vis = torch.randn((ob.nvis, 1), dtype=torch.complex64, device=dev, generator=gen)
    model = torch.randn((1, N, N), dtype=torch.complex64, device=dev, generator=gen)
    out = torch.empty_like(vis)
    grid = torch.zeros((1, N, N), dtype=torch.complex64, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    gms, dms = [], []
    for r in range(reps + 1):
        grid.zero_()
        ev[0].record()
        aw.aw_grid_batched(ctx, plan, kg, vis, None, grid)
        ev[1].record()
        aw.aw_degrid(ctx, plan, kd, model, out)
        ev[2].record()
        torch.cuda.synchronize()
        if r:
            gms.append(ev[0].elapsed_time(ev[1]))
            dms.append(ev[1].elapsed_time(ev[2]))
    info = aw.aw_plan_query(plan)
    print(json.dumps({"case": "wproj", "nvis": int(ob.nvis), "mean_taps": float(info.mean_taps), "reps": reps,
                      "grid_ms": statistics.median(gms) if gms else None,
                      "degrid_ms": statistics.median(dms) if dms else None}))
    return 0


def learned_train_case(steps: int):
    """A small case for profiling surrogate training on the tensor cores: an exact full-pol set of
    512^2 x 4, 4 w planes (supports 8, 8, 12, 16), OS 8, one PA and frequency bin; a 5 -> 128 x 4 -> 32
    network trained for `steps` steps on batches of 65,536 points (the configuration-5 batch), so that
    each layer's activations (16.8 MB in FP16) exceed neither the device nor an ncu capture's budget."""
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import build as awbuild
    awbuild.build()
    ctx = aw.aw_create(0)
    N = 512
    kw = dict(N=N, dl=math.radians(2.0) / N, OS=8, W=7.0, npol=4, nw=4, w_max=2000.0, supports=[8, 8, 12, 16])
    exact = aw.aw_make_kernels(ctx, **kw)
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, D=1.0,
                                 norm_supports=kw["supports"], w_max=kw["w_max"], f_c=1.4e9, f_h=0.2e9, chi_c=0.0,
                                 chi_h=1.5, out_scale=1.0, seed=11)
    rep = aw.aw_surrogate_train(ctx, sur, exact, steps=steps, batch=65536, lr=1e-3, lr_final=1e-5, seed=3)
    print(json.dumps({"case": "learned_train", "engine": "tcgen05", "steps": rep.steps, "batch": 65536,
                      "seconds": rep.seconds, "ms_per_step": rep.seconds * 1e3 / max(1, rep.steps),
                      "loss_first": rep.loss_first, "loss_last": rep.loss_last}))
    return 0


def learned_inline_case(engine: int):
    """A small case for profiling the inline surrogate: the full-pol test geometry (256^2 x 4,
    3 w planes x 2 PA x 2 frequency bins, supports 16-24, OS 8), 57,600 visibilities, a randomly
    initialised 5 -> 128 x 4 -> 32 network; three untimed and one timed aw_grid_learned call."""
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import build as awbuild
    from paper_2206_15117_gb300 import synthetic as sy
    awbuild.build()
    ctx = aw.aw_create(0)
    ob = sy.small_observation(n_ant=16, radius_m=180.0, n_t=120, freq=(1.2e9, 1.3e9, 1.4e9, 1.5e9), npa=2, nfb=2,
                              seed=sy.BASE_SEED + 300)
    N = 256
    kw = dict(N=N, dl=math.radians(3.0) / N, OS=8, W=7.0, npol=4, nw=3, w_max=ob.w_max, supports=[16, 20, 24],
              pa=list(ob.pa_centres), fbin_freqs=list(ob.fbin_freqs), dish_d=12.0, d_xy=sy.LEAK_XY, d_yx=sy.LEAK_YX,
              eps=0.2)
    exact = aw.aw_make_kernels(ctx, **kw)
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, seed=5, D=1.0,
                                 norm_supports=kw["supports"], w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                                 chi_c=0.0, chi_h=1.5, out_scale=0.02)
    aw.aw_surrogate_set_engine(sur, engine)
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, exact)
    info = aw.aw_plan_query(plan)
    vis = torch.as_tensor(sy.random_vis(ob.nvis, 4, seed=31), device="cuda")
    grid = torch.zeros((4, N, N), dtype=torch.complex64, device="cuda")
    for _ in range(3):
        aw.aw_grid_learned(ctx, plan, sur, exact, vis, None, grid)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    aw.aw_grid_learned(ctx, plan, sur, exact, vis, None, grid)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    rows = info.mean_taps * info.nvalid
    print(json.dumps({"case": "learned_inline", "engine": engine, "nvis": ob.nvis, "rows": rows, "ms": ms,
                      "network_tflops": rows * 2 * (5 * 128 + 3 * 128 * 128 + 128 * 32) / (ms / 1e3) / 1e12}))
    return 0


def run_ours(args, rank, world, dist):
    import torch
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import build as awbuild

    awbuild.build()
    dev_index = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev_index)
    dev = torch.device("cuda", dev_index)
    stream = torch.cuda.current_stream()
    ctx = aw.aw_create(dev_index)
    ob, kw = workload(args.time_samples, args.subset)
    if world > 1:   # weak scaling: every rank its own seeded replica
        from paper_2206_15117_gb300 import synthetic as sy
        ob = sy.observation(3, time_samples=args.time_samples, seed=sy.BASE_SEED + 3 + 1000 * rank)
    nvis = ob.nvis
    t0 = time.perf_counter()
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    t_synth = time.perf_counter() - t0
    kinfo = aw.aw_kernel_set_info(kg)
    vd, keep = aw.device_observation(ob, dev)
    # autotune on every visibility of 2 of the 32 (PA, frequency) bin pairs:
    # about a tenth of the data with the same density per (bin, tile) and the
    # same support mix; then the full plan
    from paper_2206_15117_gb300 import synthetic as sy
    sub = np.flatnonzero((ob.pa_bin[ob.row_of_vis] == 0) & (ob.fbin[ob.chan_of_vis] < 2))
    ob_sub = sy.Observation(**{**ob.__dict__, "row_of_vis": ob.row_of_vis[sub], "chan_of_vis": ob.chan_of_vis[sub]})
    vd_sub, keep_sub = aw.device_observation(ob_sub, dev)
    t0 = time.perf_counter()
    if args.tune:
        tv = [int(x) for x in args.tune.split(",")]
        tune = aw.aw_tune(*(tv + [0] * (6 - len(tv))))
    else:
        tune = aw.aw_autotune(ctx, vd_sub, kg)
    t_tune = time.perf_counter() - t0
    del vd_sub, keep_sub
    t0 = time.perf_counter()
    plan = aw.aw_plan_create(ctx, vd, kg, tune=tune)
    t_plan = time.perf_counter() - t0
    N = kw["N"]
    confirm = None
    alt_plans = []  # the other schedules' plans, kept for the 16-bit variants
    if not args.tune:
        # the subsample ranks the candidates; the finalists are then timed once more on the
        # full data (the schedules' DRAM behaviour, and how the two parts of the hybrid share
        # the SMs, differ with the number of bins in flight): the tuned choice, the two plain
        # schedules and the hybrid split where the low w planes hold nearest to 25, 30, 35 and
        # 40 % of the visibility-taps, at 2 tile CTAs per SM
        t0 = time.perf_counter()
        cands = [(tune, plan)]
        tiles_ctas = tune.ctas_per_sm if tune.grid_mode == aw.AW_GRID_TILES else 5
        finalists = [aw.aw_tune(tune.tile, tune.chunk, tiles_ctas, 1024, aw.AW_GRID_TILES),
                     aw.aw_tune(tune.tile, tune.chunk, tiles_ctas, 1024, aw.AW_GRID_OFFSETS)]
        for share in (0.25, 0.30, 0.35, 0.40):
            finalists.append(aw.aw_tune(tune.tile, tune.chunk, 2, 1024, aw.AW_GRID_HYBRID,
                                        hybrid_split(aw, plan, kw, share)))
        # the region schedule with the planes of supports up to 32, 40 and 48 cells on the region kernel
        for lim in (32, 40, 48):
            q = sum(1 for s_ in kw["supports"] if s_ <= lim)
            if 0 < q:
                finalists.append(aw.aw_tune(tune.tile, tune.chunk, 2, 1024, aw.AW_GRID_REGION, q))
        key = lambda t_: (t_.grid_mode, t_.ctas_per_sm if t_.grid_mode != aw.AW_GRID_OFFSETS else 0,
                          t_.split_planes if t_.grid_mode in (aw.AW_GRID_HYBRID, aw.AW_GRID_REGION) else 0,
                          t_.dg_tile or 1024)
        seen = {key(tune)}
        for t_ in finalists:
            if key(t_) not in seen:
                seen.add(key(t_))
                cands.append((t_, aw.aw_plan_create(ctx, vd, kg, tune=t_)))
        zv = torch.zeros((nvis, 4), dtype=torch.complex64, device=dev)
        gtmp = torch.zeros((4, N, N), dtype=torch.complex64, device=dev)
        times = []
        for _, p_ in cands:
            ms = []
            for _ in range(3):
                a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a_.record(stream)
                aw.aw_grid_batched(ctx, p_, kg, zv, None, gtmp)
                b_.record(stream)
                torch.cuda.synchronize()
                ms.append(a_.elapsed_time(b_))
            times.append(min(ms[1:]))
        label = lambda t_: SCHEDULES[t_.grid_mode] + ("/%d/%d" % (t_.split_planes, t_.ctas_per_sm)
                                                       if t_.grid_mode == aw.AW_GRID_HYBRID else
                                                       "/%d" % t_.split_planes if t_.grid_mode == aw.AW_GRID_REGION
                                                       else "")
        confirm = {"full_data_grid_ms": {label(t_): ms_ for (t_, _), ms_ in zip(cands, times)},
                   "seconds": None}
        best = int(np.argmin(times))
        tune, plan = cands[best]
        # the 16-bit variants choose between the best plan of each schedule
        alt_plans = []
        if not args.no_variants:
            for mode in (aw.AW_GRID_TILES, aw.AW_GRID_OFFSETS, aw.AW_GRID_HYBRID, aw.AW_GRID_REGION):
                idx = [i for i, (t_, _) in enumerate(cands) if t_.grid_mode == mode and i != best]
                if idx and mode != tune.grid_mode:
                    alt_plans.append(cands[min(idx, key=lambda i: times[i])])
        del cands, zv, gtmp
        torch.cuda.empty_cache()
        confirm["seconds"] = time.perf_counter() - t0
    info = aw.aw_plan_query(plan)
    gen = torch.Generator(device=dev)
    gen.manual_seed(2206_15117 + rank)
    vis = torch.randn((nvis, 4), dtype=torch.complex64, device=dev, generator=gen)
    vis_out = torch.empty_like(vis)
    model = torch.randn((4, N, N), dtype=torch.complex64, device=dev, generator=gen)
    grid = torch.zeros((4, N, N), dtype=torch.complex64, device=dev)
    image = torch.empty((4, N, N), dtype=torch.float32, device=dev)
    # grid (one kernel, or the two concurrent parts of the hybrid schedule), checker +
    # grid-correction (FFT step), degrid
    launches_per_step = 3 + info.grid_kernels
    # pinned host buffers of the end-to-end measurement, allocated up front: allocated after the
    # BF16/FP16 variant sets had been built and freed, the same transfers measured about 9x slower
    host_bufs = None
    if not args.no_e2e:
        host_bufs = (torch.empty((nvis, 4), dtype=torch.complex64, pin_memory=True),
                     torch.empty((nvis, 4), dtype=torch.complex64, pin_memory=True))

    def step(ev=None, kset_g=kg, kset_d=kd, gplan=None):
        grid.zero_()
        if ev: ev[0].record(stream)
        st = aw.aw_grid_batched(ctx, gplan or plan, kset_g, vis, None, grid)
        if ev: ev[1].record(stream)
        aw.aw_fft_to_image(ctx, kset_g, grid, float(info.nvalid), image)
        if ev: ev[2].record(stream)
        aw.aw_degrid(ctx, plan, kset_d, model, vis_out)
        if ev: ev[3].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    clk = ClockSampler(dev_index)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    torch.cuda.nvtx.range_push("timed")
    e_start.record(stream)
    for k in range(args.steps):
        step(evs[k])
    e_end.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clocks = clk.stop()
    if dist:
        dist.barrier()
    total_ms = e_start.elapsed_time(e_end)
    t_grid = [e[0].elapsed_time(e[1]) for e in evs]
    t_fft = [e[1].elapsed_time(e[2]) for e in evs]
    t_deg = [e[2].elapsed_time(e[3]) for e in evs]
    total_ms, job_vis = aggregate(total_ms, nvis, dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_vis / (ms_per_step / 1e3) / 1e6

    # roofline of the dominant kernel: FP32 ALU (complex MACs of the Mueller product)
    flops = 128.0 * info.mean_taps * info.nvalid          # 16 complex MACs x 8 flop per tap
    g_ms, d_ms = statistics.mean(t_grid), statistics.mean(t_deg)
    dom_ms = max(g_ms, d_ms)
    gname = {aw.AW_GRID_TILES: "grid_persistent_kernel", aw.AW_GRID_OFFSETS: "grid_offset_kernel",
             aw.AW_GRID_HYBRID: "grid_persistent_kernel + grid_offset_kernel",
             aw.AW_GRID_REGION: "grid_region_kernel + grid_offset_kernel"}[tune.grid_mode]
    dom = ("aw_grid (%s)" % gname) if g_ms >= d_ms else "aw_degrid (degrid_items_kernel)"
    peak_tflops, peak_src = fp32_peak_tflops(dev_index)
    achieved = flops / (dom_ms / 1e3) / 1e12
    roof = roofline_entry(dom, achieved, peak_tflops, peak_src, flops, g_ms, d_ms,
                          region=tune.grid_mode == aw.AW_GRID_REGION, nvalid=info.nvalid, subset=args.subset)
    alt = bf16_scaled_peak()
    if alt:
        roof["peak_alt"] = {"value": alt, "frac": achieved / alt,
                            "source": "measured bf16 dense burst (MEASURED_PEAKS.json) x 1/32, the nominal ratio "
                                      "of the FP32 CUDA-core rate to the dense 16-bit tensor rate"}

    # variants: BF16 / FP16 kernel tables (FP32 arithmetic).  Without --tune each precision grids
    # with the faster of the two schedules on its own tables, as aw_autotune on that kernel set would
    # choose (halving the table bytes moves the tile schedule's L2 stream, not the atomics)
    schedules = SCHEDULES

    def var_roof(gm_, dm_):
        # every table precision computes in FP32: the same FP32 peak for all three
        return {k_: {"bound": "alu", "achieved": flops / (t_ / 1e3) / 1e12, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": flops / (t_ / 1e3) / 1e12 / peak_tflops}
                for k_, t_ in (("grid", gm_), ("degrid", dm_))}

    variants = {"fp32": {"grid_ms": g_ms, "degrid_ms": d_ms, "mvis_s": nvis / ((g_ms + d_ms) / 1e3) / 1e6,
                         "grid_schedule": schedules[tune.grid_mode], "roofline": var_roof(g_ms, d_ms)}}
    if not args.no_variants:
        for name, stg in (("bf16", aw.AW_STORAGE_BF16), ("fp16", aw.AW_STORAGE_FP16)):
            kg2 = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID, storage=stg)
            kd2 = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID, storage=stg)
            res = {}
            for tn, pl in [(tune, plan)] + alt_plans:
                step(None, kg2, kd2, pl)
                ev2 = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(3)]
                for k in range(3):
                    step(ev2[k], kg2, kd2, pl)
                torch.cuda.synchronize()
                res[schedules[tn.grid_mode]] = (statistics.mean(e[0].elapsed_time(e[1]) for e in ev2),
                                                statistics.mean(e[2].elapsed_time(e[3]) for e in ev2))
            best = min(res, key=lambda k_: res[k_][0])
            gm, dm = res[best]
            variants[name] = {"grid_ms": gm, "degrid_ms": dm, "mvis_s": nvis / ((gm + dm) / 1e3) / 1e6,
                              "grid_schedule": best, "grid_ms_by_schedule": {k_: v_[0] for k_, v_ in res.items()},
                              "table_bytes": int(aw.aw_kernel_set_info(kg2).bytes), "roofline": var_roof(gm, dm)}
            del kg2, kd2
            torch.cuda.empty_cache()
    alt_plans = []

    # the weighted path: the timed steps pass no weight array (natural weights:
    # nothing read); here one gridding call with per-visibility, per-correlation
    # FP32 weights ([nvis][4], 16 B per visibility read by the gridder)
    wgen = torch.Generator(device=dev)
    wgen.manual_seed(7)
    wts = torch.rand((nvis, 4), dtype=torch.float32, device=dev, generator=wgen) + 0.5
    wms = []
    for r_ in range(4):
        grid.zero_()
        a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a_.record(stream)
        aw.aw_grid_batched(ctx, plan, kg, vis, wts, grid)
        b_.record(stream)
        torch.cuda.synchronize()
        if r_:
            wms.append(a_.elapsed_time(b_))
    weighted = {"grid_ms": statistics.median(wms), "grid_ms_natural": g_ms,
                "weight_bytes": int(wts.numel() * 4),
                "note": "the same gridding call with a [nvis][4] FP32 weight array; the timed steps use natural "
                        "weights (no weight array passed, none read)"}
    del wts
    torch.cuda.empty_cache()

    # end to end through the C ABI with host buffers (pinned), copies timed
    e2e = None
    if not args.no_e2e:
        vis_host, out_host = host_bufs
        vis_host.copy_(vis)
        vis_dev = torch.empty_like(vis)
        ne = max(3, min(args.steps, 6))

        def e2e_step(ev=None):
            if ev: ev[0].record(stream)
            vis_dev.copy_(vis_host, non_blocking=True)
            if ev: ev[1].record(stream)
            grid.zero_()
            aw.aw_grid_batched(ctx, plan, kg, vis_dev, None, grid)
            aw.aw_fft_to_image(ctx, kg, grid, float(info.nvalid), image)
            aw.aw_degrid(ctx, plan, kd, model, vis_out)
            if ev: ev[2].record(stream)
            out_host.copy_(vis_out, non_blocking=True)
            if ev: ev[3].record(stream)

        e2e_step()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(ne)]
        a.record(stream)
        for k in range(ne):
            e2e_step(pev[k])
        b.record(stream)
        torch.cuda.synchronize()
        e_ms_serial = a.elapsed_time(b) / ne
        e_parts = {"h2d_ms": statistics.mean(e[0].elapsed_time(e[1]) for e in pev),
                   "compute_ms": statistics.mean(e[1].elapsed_time(e[2]) for e in pev),
                   "d2h_ms": statistics.mean(e[2].elapsed_time(e[3]) for e in pev),
                   "serial_ms_per_step": e_ms_serial}
        # the same steps pipelined over two device buffers of visibilities and of
        # predictions: step k+1's visibilities are copied in on their own stream during step k
        # (into the buffer step k-1 gridded from), and step k's predictions are copied out on
        # a third stream during step k+1 (step k+2 reuses that buffer after the copy)
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        vis_b = [vis_dev, torch.empty_like(vis)]
        out_b = [vis_out, torch.empty_like(vis_out)]
        ev_in, ev_grid, ev_done, ev_out = ([torch.cuda.Event(), torch.cuda.Event()] for _ in range(4))

        def pipelined(n):
            s_in.wait_stream(stream)
            with torch.cuda.stream(s_in):
                vis_b[0].copy_(vis_host, non_blocking=True)
            ev_in[0].record(s_in)
            for k in range(n):
                b = k % 2
                if k + 1 < n:
                    if k >= 1:
                        s_in.wait_event(ev_grid[1 - b])   # step k-1 has gridded from that buffer
                    with torch.cuda.stream(s_in):
                        vis_b[1 - b].copy_(vis_host, non_blocking=True)
                    ev_in[1 - b].record(s_in)
                stream.wait_event(ev_in[b])
                grid.zero_()
                aw.aw_grid_batched(ctx, plan, kg, vis_b[b], None, grid)
                ev_grid[b].record(stream)
                aw.aw_fft_to_image(ctx, kg, grid, float(info.nvalid), image)
                if k >= 2:
                    stream.wait_event(ev_out[b])      # step k-2's predictions have left that buffer
                aw.aw_degrid(ctx, plan, kd, model, out_b[b])
                ev_done[b].record(stream)
                s_out.wait_event(ev_done[b])
                with torch.cuda.stream(s_out):
                    out_host.copy_(out_b[b], non_blocking=True)
                ev_out[b].record(s_out)
            stream.wait_stream(s_out)

        pipelined(2)     # also captures the gridding graph of each buffer
        torch.cuda.synchronize()
        a.record(stream)
        pipelined(ne)
        b.record(stream)
        torch.cuda.synchronize()
        e_ms = a.elapsed_time(b) / ne
        nbytes = vis_host.numel() * 8
        e2e = {"value": world * nvis / (e_ms / 1e3) / 1e6, "unit": UNIT, "h2d_bytes_per_step": int(nbytes),
               "d2h_bytes_per_step": int(nbytes), "ms_per_step": e_ms, "parts": e_parts,
               "how": "every step: pinned host visibilities copied in, grid + FFT + degrid, predicted visibilities "
                      "copied out; two device buffers each way, copies on their own streams overlapped with the "
                      "neighbouring steps' compute (parts: the same steps run serially)"}
        del pipelined, vis_b, out_b
        torch.cuda.empty_cache()

    clean = None
    if not args.no_clean and not args.subset:
        clean = clean_section(ctx, dev, args, ob, kw, plan, kg, kd, stream)
    mosaic = None
    if not args.no_mosaic and not args.subset:
        mosaic = mosaic_section(ctx, dev, args, stream)
        mosaic["uv_vs_image_domain"] = uvmosaic_section(ctx, dev, args, stream)
    baselines = None
    if not args.no_baselines and not args.subset:
        baselines = baselines_section(ctx, dev, ob, kw, tune, vis, model, grid, vis_out, stream, variants["fp32"])
    learned = None
    if not args.no_learned or not args.no_wproj:
        # free the FP32 workload before the other configurations
        del vis, vis_out, model, kd
        torch.cuda.empty_cache()
    wproj = None
    if not args.no_wproj and not args.subset:
        wproj = wproj_section(ctx, dev, args, stream)
        torch.cuda.empty_cache()
    if not args.no_learned:
        learned = learned_section(ctx, dev, args)
    cpu = None
    if rank == 0 and not args.no_cpu:
        smp = oracle_sample(ob, kw)
        t1 = oracle_step(smp)
        nthr = host_cores()
        oracle_step_parallel(smp, nthr)   # warm-up (shards, threads)
        tp = statistics.median([oracle_step_parallel(smp, nthr) for _ in range(3)])
        cpu = {"value": oracle_mvis(smp, tp), "unit": UNIT, "cores": nthr, "kind": "oracle",
               "sample": sample_text(smp, nthr), "seconds": tp,
               "value_sample_unscaled": oracle_mvis_unscaled(smp, tp),
               "one_thread": {"value": oracle_mvis(smp, t1), "seconds": t1,
                              "value_sample_unscaled": oracle_mvis_unscaled(smp, t1)}}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(ob, kw, info),
                "parallelism": "replicas" if world > 1 else "single",
                "breakdown_ms": {"grid": g_ms, "fft_to_image": statistics.mean(t_fft), "degrid": d_ms},
                "weighted_grid": weighted,
                "once_per_dataset_s": {"kernel_synthesis_grid_and_degrid": t_synth, "autotune": t_tune,
                                       "plan_sort": t_plan, "table_bytes_per_set": int(kinfo.bytes)},
                "cold": {"value": nvis * world / (t_synth + t_tune + t_plan + ms_per_step / 1e3) / 1e6, "unit": UNIT,
                         "includes": "kernel synthesis of both sets, autotune, plan sort and one step"},
                "roofline": roof, "variants": variants, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": {"sm_mhz": clocks["sm_mhz"], "sm_max_mhz": clocks["sm_max_mhz"],
                           "reasons": clocks["reasons"]},
                "gpu_launches": launches_per_step * args.steps,
                "tune": {"tile": tune.tile, "chunk": tune.chunk, "ctas_per_sm": tune.ctas_per_sm,
                         "dg_tile": tune.dg_tile or 1024, "degrid_items": info.nitems_degrid,
                         "grid_schedule": SCHEDULES[tune.grid_mode], "split_planes": tune.split_planes,
                         "confirmed": confirm},
                "clean": clean, "mosaic": mosaic, "per_baseline_kernels": baselines, "learned": learned,
                "wproj_stokes_i": wproj}
        print(json.dumps(line), flush=True)
    return 0


def aggregate(total_ms: float, nvis: int, dist=None, device=None):
    """Whole-job timing over replicas: the slowest rank's timed region (max)
    and the visibilities of all ranks (sum)."""
    if dist is None:
        return float(total_ms), int(nvis)
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    n = torch.tensor([float(nvis)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


SCHEDULES = ["tiles", "offsets", "hybrid", "region"]


def hybrid_split(aw, plan, kw, share: float) -> int:
    """Number of low w planes whose share of the plan's visibility-taps (sum
    of S^2) is nearest to `share`, from the plan's own bins; 1..nw-1."""
    import torch
    info = aw.aw_plan_query(plan)
    b = torch.empty(int(info.nvis), dtype=torch.int32, device="cuda")
    v = torch.empty(int(info.nvis), dtype=torch.uint8, device="cuda")
    aw.aw_plan_coords(plan, bin=b, valid=v)
    per_plane = len(kw["pa"]) * len(kw["fbin_freqs"])
    bins = b[v == 1].to(torch.int64)
    planes = (bins // per_plane) % kw["nw"]
    sup = torch.as_tensor(kw["supports"], dtype=torch.float64, device=bins.device)
    taps = torch.bincount(planes, weights=sup[planes] ** 2, minlength=kw["nw"]).cpu().numpy()
    below = np.concatenate([[0.0], np.cumsum(taps) / max(taps.sum(), 1.0)])   # below[q]: share of planes < q
    q = int(np.argmin(np.abs(below - share)))
    return max(1, min(q, kw["nw"] - 1))


# DRAM bytes per visibility of the dominant kernels from the one-bin-pair ncu capture summarised in
# profiles/dram_traffic_fullpol_aw_1pair.md (1,139,896 visibilities: region gridding 146.5 MB,
# degridding 96.5 MB); scaled to a workload by its visibility count (the per-visibility bytes scale;
# the tables touched per visibility grow with the bins, so the figure is a lower bound).
TRAFFIC_PER_VIS = {"region": 146.5e6 / 1139896, "degrid_items_kernel": 96.5e6 / 1139896}


def roofline_entry(kernel, achieved, peak, peak_src, flops, g_ms, d_ms, region, nvalid, subset):
    """The `roofline` object of the dominant step (gridding if g_ms >= d_ms).  `traffic` is the
    scaled one-bin-pair capture when it describes the kernel that runs: the degridder; the region
    capture predates the region kernel's three-pass units (supports 20 and 24), so for the region
    schedule `traffic` is null and the previous figure stands beside it, labelled.  Null at the
    subset scale and for the other schedules."""
    traffic, traffic_prev = None, None
    if not subset:
        if g_ms >= d_ms and region:
            traffic_prev = TRAFFIC_PER_VIS["region"] * nvalid
        elif g_ms < d_ms:
            traffic = TRAFFIC_PER_VIS["degrid_items_kernel"] * nvalid
    roof = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "traffic_source": ("profiles/dram_traffic_fullpol_aw_1pair.md, scaled by the visibility count "
                               "(lower bound)") if traffic else None,
            "peak_source": peak_src, "flops_per_launch": flops}
    if traffic_prev:
        roof["traffic_previous_region_kernel"] = {
            "bytes": traffic_prev,
            "source": "profiles/dram_traffic_fullpol_aw_1pair.md (the region kernel with paired passes, before "
                      "the three-pass units), scaled by the visibility count (lower bound)"}
    return roof


def fp32_peak_tflops(device_index: int = 0):
    """FP32 CUDA-core peak from the device's SM count, 128 FP32 lanes per SM,
    2 flop per FMA and the maximum SM clock (MEASURED_PEAKS.json's, else the
    nominal 2070 MHz).  Returns (TFLOP/s, how it was derived)."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    try:
        j = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        mhz, src = float(j["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    except Exception:
        mhz, src = 2070.0, "nominal maximum SM clock"
    return (sms * 128 * 2 * mhz * 1e6 / 1e12,
            "FP32 CUDA-core peak derived: %d SMs (device) x 128 FP32 lanes x 2 flop x %.0f MHz (%s)" % (sms, mhz, src))


def bf16_burst():
    """The measured dense bf16 tensor burst (TFLOP/s), or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"])
    except Exception:
        return None


def bf16_scaled_peak():
    """The measured dense bf16 tensor burst scaled by 1/32 (nominal FP32
    CUDA-core : dense 16-bit tensor ratio), or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]) / 32.0
    except Exception:
        return None


def main():
    args = parse()
    if args.learned_inline_case is not None:
        return learned_inline_case(args.learned_inline_case)
    if args.learned_train_case is not None:
        return learned_train_case(args.learned_train_case)
    if args.wproj_case is not None:
        return wproj_case(args.wproj_case)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            tdist.init_process_group("nccl")
        else:
            tdist.init_process_group("gloo")
        dist = tdist
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    else:
        rc = run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
