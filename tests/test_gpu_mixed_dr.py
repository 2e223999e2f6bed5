"""GPU: the mixed-precision form on configuration-2 data (w-projection Stokes I,
2048^2, 32 w planes, OS 8): dirty images from BF16 / FP16 / FP32 kernel tables
against the FP64 oracle's dirty image of the same point-source visibilities
(20 sources, noise 0.01 Jy).  Reports the maximum and RMS error and the
error-limited dynamic range DR = peak / RMS(image - oracle image), and bounds
the dynamic-range loss DR_fp32 / DR_mixed."""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import case_wproj, oracle_coords, oracle_spec, used_bins

pytestmark = pytest.mark.gpu


def test_mixed_precision_dynamic_range():
    from paper_2206_15117_gb300 import aw
    ctx = aw.aw_create(0)
    ob, kw = case_wproj(vis_fraction=0.002)
    # point-source visibilities (Eq. 2 evaluated directly by the oracle) plus noise
    uvwl = oc.uvw_lambda(ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    src = ob.sources
    V = oc.dft_predict(uvwl, src[:, :2], src[:, 2] + 0j)
    V = (V + sy.random_vis(ob.nvis, 1, sigma=0.01, seed=3)[:, 0]).astype(np.complex64)
    co = oracle_coords(ob, kw)
    G, ws, _ = oc.grid(oc.make_kernels(oracle_spec(kw), bins=used_bins(co)), co, V)
    ref = oc.fft_to_image(G, 7.0, ws)[0]
    N = kw["N"]
    q = slice(N // 4, 3 * N // 4)
    peak = np.abs(ref[q, q]).max()
    vd, keep = aw.device_observation(ob)
    report = {}
    for name, st in (("fp32", aw.AW_STORAGE_FP32), ("bf16", aw.AW_STORAGE_BF16), ("fp16", aw.AW_STORAGE_FP16)):
        ks = aw.aw_make_kernels(ctx, **kw, storage=st)
        plan = aw.aw_plan_create(ctx, vd, ks)
        grid = torch.zeros((1, N, N), dtype=torch.complex64, device="cuda")
        s = aw.aw_grid(ctx, plan, ks, torch.as_tensor(V.reshape(-1, 1), device="cuda"), None, grid, want_stats=True)
        img = torch.empty((1, N, N), dtype=torch.float32, device="cuda")
        aw.aw_fft_to_image(ctx, ks, grid, s.weight_sum, img)
        d = (img.cpu().numpy()[0] - ref)[q, q]
        rms = float(np.sqrt(np.mean(d * d)))
        report[name] = {"max_abs_err": float(np.abs(d).max()), "rms_err": rms, "dr": float(peak / rms),
                        "peak_jy": float(peak)}
    for name in ("bf16", "fp16"):
        report[name]["dr_loss_vs_fp32"] = report["fp32"]["dr"] / report[name]["dr"]
    print(json.dumps(report))
    out = os.environ.get("AW_REPORT_DIR")
    if out:
        with open(os.path.join(out, "mixed_precision_dr.json"), "w") as f:
            json.dump(report, f, indent=1)
    assert report["fp32"]["dr"] > 1e5
    assert report["fp16"]["dr"] > 1e3 and report["bf16"]["dr"] > 1e2
    assert report["fp16"]["max_abs_err"] < 5e-4 * peak and report["bf16"]["max_abs_err"] < 4e-3 * peak
