"""GPU parity of the UV-domain mosaic path (Sec. 2.2) through the C ABI:
beam-weighted kernels (AW_ROLE_BEAM) with a pointing offset, phase rotation of
visibilities, and a two-field UV-domain mosaic image, against the FP64 oracle
on the same seeded inputs."""
import math

import numpy as np
import pytest
import torch

from oracle import core as oc
from oracle import mosaic as om
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, case_fullpol, rel_err, used_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _export(ks, b, S, OS, P):
    from paper_2206_15117_gb300 import aw
    out = torch.empty(OS * OS * S * S * P, dtype=torch.complex64, device="cuda")
    aw.aw_kernel_set_export(ks, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(OS, OS, S, S, P)


@pytest.mark.parametrize("role,offset", [(3, (0.0, 0.0)), (3, (0.012, -0.008)), (1, (0.012, -0.008)),
                                         (0, (-0.01, 0.005))])
def test_synthesis_with_pointing_offset_matches_oracle(ctx, role, offset):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol()
    kw = {**kw, "point_l": offset[0], "point_m": offset[1]}
    ks = aw.aw_make_kernels(ctx, **kw, role=role)
    spec = oc.KernelSpec(**kw, role=role)
    for b in (0, spec.nbins - 1):
        S = spec.supports[b // (spec.npa * spec.nfb)]
        got = _export(ks, b, S, spec.OS, 16)
        ref = oc.synth_bin(spec, b)
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()


def test_phase_rotation_matches_oracle(ctx):
    from paper_2206_15117_gb300 import aw
    ob = sy.small_observation(n_ant=12, radius_m=400.0, n_t=20, freq=(1.2e9, 1.3e9, 1.4e9))
    A, B = (1.0, math.radians(-45.0)), (1.0 + math.radians(0.8), math.radians(-44.6))
    v = (np.random.default_rng(7).normal(size=(ob.nvis, 4)) +
         1j * np.random.default_rng(8).normal(size=(ob.nvis, 4))).astype(np.complex64)
    vd, keep = aw.device_observation(ob)
    uvw_out = torch.empty((ob.uvw.shape[0], 3), dtype=torch.float64, device="cuda")
    vin = torch.as_tensor(v, device="cuda")
    vout = torch.empty_like(vin)
    aw.aw_phase_rotate(ctx, vd, uvw_out, vin, vout, A, B)
    uref, vref = oc.phase_rotate(ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, v.astype(np.complex128), A, B)
    assert np.abs(uvw_out.cpu().numpy() - uref).max() < 1e-9
    assert np.abs(vout.cpu().numpy() - vref).max() < 2e-6 * np.abs(vref).max()
    aw.aw_phase_rotate(ctx, vd, None, vin, vin, A, B)          # in place
    assert np.abs(vin.cpu().numpy() - vref).max() < 2e-6 * np.abs(vref).max()


def test_two_field_uv_mosaic_matches_oracle(ctx):
    # two pointings of one array: field 0 at the mosaic centre, field 1 offset by about a
    # degree; field 1 is phase-rotated to the mosaic centre and both are gridded onto one
    # grid with beam-weighted kernels centred on their pointings
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=20)
    centre = (1.0, math.radians(-45.0))
    p1 = (1.0 + math.radians(0.9) / math.cos(centre[1]), centre[1] + math.radians(0.3))
    fr = om.frame(*centre, kw["dl"], kw["N"])
    l1, m1, _ = om.radec_to_lmn(fr, p1[0], p1[1])
    rng = np.random.default_rng(12)
    N = kw["N"]
    grid = torch.zeros((4, N, N), dtype=torch.complex64, device="cuda")
    G_ref = np.zeros((4, N, N), np.complex128)
    ws_gpu = ws_ref = 0.0
    keep = []
    for f, (pt, off) in enumerate([(centre, (0.0, 0.0)), (p1, (float(l1), float(m1)))]):
        v = (rng.normal(size=(ob.nvis, 4)) + 1j * rng.normal(size=(ob.nvis, 4))).astype(np.complex64)
        kwf = {**kw, "point_l": off[0], "point_m": off[1]}
        kb = aw.aw_make_kernels(ctx, **kwf, role=aw.AW_ROLE_BEAM)
        vd, k = aw.device_observation(ob)
        vin = torch.as_tensor(v, device="cuda")
        uvw_rot = torch.empty((ob.uvw.shape[0], 3), dtype=torch.float64, device="cuda")
        aw.aw_phase_rotate(ctx, vd, uvw_rot, vin, vin, pt, centre)
        vd.uvw = uvw_rot.data_ptr()
        plan = aw.aw_plan_create(ctx, vd, kb)
        st = aw.aw_grid(ctx, plan, kb, vin, None, grid, want_stats=True)
        ws_gpu += st.weight_sum
        keep += [k, uvw_rot, plan, kb]
        # the oracle on the same data
        uvw_r, vr = oc.phase_rotate(ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, v.astype(np.complex128), pt,
                                    centre)
        spec = oc.KernelSpec(**kwf, role=oc.ROLE_BEAM)
        co = oc.coords(spec, uvw_r, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin)
        G, ws, _ = oc.grid(oc.make_kernels(spec, bins=used_bins(co)), co, vr)
        G_ref += G
        ws_ref += ws
    assert ws_gpu == pytest.approx(ws_ref, rel=1e-12)
    l2, mx = rel_err(grid.cpu().numpy(), G_ref)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    img = torch.empty((4, N, N), dtype=torch.float32, device="cuda")
    aw.aw_fft_to_image(ctx, keep[3], grid, ws_gpu, img)
    ref_img = oc.fft_to_image(G_ref, kw["W"], ws_ref)
    q = slice(N // 4, 3 * N // 4)
    assert np.abs(img.cpu().numpy()[:, q, q] - ref_img[:, q, q]).max() < 1e-5 * np.abs(ref_img[:, q, q]).max()
