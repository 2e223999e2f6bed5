"""The bounds-checked build of the library (-DAW_BOUNDS_CHECK: the gridding
and degridding kernels check every grid, table, shared-memory, record and
output index and record the first bad one) run over the three gridding schedules,
several tile / chunk / super-tile choices, ragged and flagged inputs, the
subtracting degridder, full-pol and Stokes-I cases: no check may fail, and the
results still match the FP64 oracle.  The library is built and loaded in a
child process (compute-sanitizer is not available on these machines)."""
import json
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent('''
    import json, sys
    import numpy as np
    import torch
    sys.path.insert(0, %r)
    from paper_2206_15117_gb300 import aw
    from paper_2206_15117_gb300 import synthetic as sy
    from oracle import core as oc
    from tests.gpu_cases import case_fullpol, case_stokes_i_cfg1, case_wproj, rel_err, used_bins
    assert aw.load()._name.endswith("libaw_checked.so"), aw.load()._name
    aw.aw_debug_bounds_status(reset=True)
    ctx = aw.aw_create(0)
    report = {}
    cases = [("fullpol", case_fullpol(n_t=12), [(8, 32, 3, 0, 0), (64, 128, 4, 256, 1), (32, 256, 2, 1024, 1),
                                                 (16, 512, 2, 32, 0), (32, 256, 2, 256, 2, 1),
                                                 (32, 256, 2, 256, 3)]),
             ("fullpol_wide", case_fullpol(n_t=200, radius=60.0, supports=(16, 40, 56)), [(32, 256, 2, 256, 3)]),
             ("stokes_i", case_stokes_i_cfg1(time_samples=20), [(16, 128, 2, 0, 0), (32, 256, 2, 256, 1),
                                                              (16, 128, 3, 256, 2, 1)]),
             ("wproj_region", case_wproj(vis_fraction=0.001), [(32, 256, 2, 256, 3), (32, 256, 2, 256, 3, 14)])]
    for name, (ob, kw), tunes in cases:
        npol, N = kw["npol"], kw["N"]
        kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
        kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
        flags = (np.random.default_rng(1).random(ob.nvis) < 0.05).astype(np.uint8)
        vd, keep = aw.device_observation(ob, flags=flags)
        v_np = sy.random_vis(ob.nvis, npol, seed=2)
        m_np = sy.random_grid(npol, N, seed=3)
        vis = torch.as_tensor(v_np, device="cuda")
        model = torch.as_tensor(m_np, device="cuda")
        spec = oc.KernelSpec(**kw)
        co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin, flags)
        bins = used_bins(co)
        G, _, _ = oc.grid(oc.make_kernels(spec, bins=bins), co, v_np)
        V = oc.degrid(oc.make_kernels(oc.KernelSpec(**kw, role=oc.ROLE_DEGRID), bins=bins), co,
                      m_np.astype(np.complex128))
        worst = 0.0
        for t in tunes:
            plan = aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(*t))
            for fn in (aw.aw_grid, aw.aw_grid_batched):
                grid = torch.zeros((npol, N, N), dtype=torch.complex64, device="cuda")
                fn(ctx, plan, kg, vis, None, grid)
                worst = max(worst, max(rel_err(grid.cpu().numpy(), G)))
            out = torch.empty((ob.nvis, npol), dtype=torch.complex64, device="cuda")
            aw.aw_degrid(ctx, plan, kd, model, out)
            worst = max(worst, max(rel_err(out.cpu().numpy(), V)))
            aw.aw_degrid_subtract(ctx, plan, kd, model, vis, out)
            worst = max(worst, max(rel_err(out.cpu().numpy(), np.where((co.valid == 1)[:, None], v_np - V, v_np))))
        report[name] = worst
    report["status"] = aw.aw_debug_bounds_status()
    print("REPORT " + json.dumps(report))
''') % ROOT


def test_bounds_checked_build_reports_no_bad_index():
    from paper_2206_15117_gb300 import build as awbuild
    lib = awbuild.build(bounds_check=True)
    env = dict(os.environ, AW_LIBAW=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=900,
                       cwd=ROOT)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    line = [l for l in r.stdout.splitlines() if l.startswith("REPORT ")][-1]
    rep = json.loads(line[len("REPORT "):])
    assert rep["status"] == 0, rep
    assert rep["fullpol"] < 1e-5 and rep["stokes_i"] < 1e-5 and rep["fullpol_wide"] < 1e-5, rep
    assert rep["wproj_region"] < 1e-5, rep


def test_normal_build_has_no_bounds_checks():
    from paper_2206_15117_gb300 import aw
    if os.environ.get("AW_LIBAW"):
        pytest.skip("another build is loaded")
    with pytest.raises(aw.AWError) as ei:
        aw.aw_debug_bounds_status()
    assert ei.value.code == aw.AW_EUNSUPPORTED
