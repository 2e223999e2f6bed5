"""GPU parity of per-baseline Mueller kernels (antenna types with their own
leakage terms, one kernel class per ordered type pair; Sec. 2.1 without the
baseline averaging of Sec. 3.2) through the C ABI against the FP64 oracle on
the same seeded inputs: class tables, bins of the plan (bit-exact, flipped
samples take the swapped class), gridding and degridding."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, case_fullpol, rel_err, used_bins

pytestmark = pytest.mark.gpu

TYPE_LEAK = [(0.02 * np.exp(0.4j), 0.015 * np.exp(-1.3j)),
             (-0.03 + 0.01j, 0.02j),
             (0.01 - 0.02j, -0.025 + 0.0j)]
N_ANT = 16
ANT_TYPE = np.array([0, 1, 2, 2, 0, 1, 1, 2, 0, 0, 2, 1, 0, 2, 1, 0])


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _case(n_t=16, nw=2, npa=1, nfb=2):
    ob, kw = case_fullpol(n_t=n_t, nw=nw, npa=npa, nfb=nfb, n_ant=N_ANT, supports=(16, 20, 24)[:nw])
    kw = {**kw, "type_leak": TYPE_LEAK}
    rt = sy.row_antenna_types(N_ANT, ob.uvw.shape[0], ANT_TYPE)
    return ob, kw, rt


def _export(ks, b, S, OS, P):
    from paper_2206_15117_gb300 import aw
    out = torch.empty(OS * OS * S * S * P, dtype=torch.complex64, device="cuda")
    aw.aw_kernel_set_export(ks, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(OS, OS, S, S, P)


@pytest.mark.parametrize("role", [0, 1, 3])
def test_class_tables_match_oracle(ctx, role):
    from paper_2206_15117_gb300 import aw
    _, kw, _ = _case()
    ks = aw.aw_make_kernels(ctx, **kw, role=role)
    spec = oc.KernelSpec(**kw, role=role)
    info = aw.aw_kernel_set_info(ks)
    assert info.nbins == spec.nbins == 9 * spec.nw * spec.npa * spec.nfb
    per = spec.nw * spec.npa * spec.nfb
    for b in (0, 5 * per + 1, spec.nbins - 1):
        S = int(spec.supports[spec.plane_of(b)])
        got = _export(ks, b, S, spec.OS, 16)
        ref = oc.synth_bin(spec, b)
        assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max(), b


def test_plan_bins_with_row_types_bit_exact(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw, rt = _case()
    ks = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob, row_types=rt)
    plan = aw.aw_plan_create(ctx, vd, ks)
    n = ob.nvis
    out = {k: torch.empty(n, dtype=torch.int32, device="cuda") for k in ("x0", "y0", "fx", "fy", "bin")}
    out["flip"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    out["valid"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    aw.aw_plan_coords(plan, **out)
    torch.cuda.synchronize()
    spec = oc.KernelSpec(**kw)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin, row_types=rt)
    for k in ("x0", "y0", "fx", "fy", "bin", "flip", "valid"):
        np.testing.assert_array_equal(out[k].cpu().numpy(), getattr(co, k), err_msg=k)
    # every class is used, flipped samples included
    cls = co.bin // (spec.nw * spec.npa * spec.nfb)
    assert set(np.unique(cls[co.valid == 1])) == set(range(9))
    assert np.any((co.flip == 1) & (cls % 3 != cls // 3))


@pytest.mark.parametrize("grid_mode", [0, 1, 3])
def test_grid_and_degrid_parity(ctx, grid_mode):
    from paper_2206_15117_gb300 import aw
    ob, kw, rt = _case()
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    vd, keep = aw.device_observation(ob, row_types=rt)
    plan = aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(32, 256, 2, 0, grid_mode))
    vis = sy.random_vis(ob.nvis, 4, seed=61)
    w = sy.random_weights(ob.nvis, 4, seed=62)
    model = sy.random_grid(4, kw["N"], seed=63)
    N = kw["N"]
    grid = torch.zeros((4, N, N), dtype=torch.complex64, device="cuda")
    st = aw.aw_grid(ctx, plan, kg, torch.as_tensor(vis, device="cuda"), torch.as_tensor(w, device="cuda"), grid,
                    want_stats=True)
    out = torch.empty((ob.nvis, 4), dtype=torch.complex64, device="cuda")
    aw.aw_degrid(ctx, plan, kd, torch.as_tensor(model, device="cuda"), out)
    spec_g, spec_d = oc.KernelSpec(**kw, role=oc.ROLE_GRID), oc.KernelSpec(**kw, role=oc.ROLE_DEGRID)
    co = oc.coords(spec_g, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin, row_types=rt)
    bins = used_bins(co)
    G, ws, _ = oc.grid(oc.make_kernels(spec_g, bins=bins), co, vis, w)
    l2, mx = rel_err(grid.cpu().numpy(), G)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    assert st.weight_sum == pytest.approx(ws, rel=1e-12)
    V = oc.degrid(oc.make_kernels(spec_d, bins=bins), co, model.astype(np.complex128))
    l2, mx = rel_err(out.cpu().numpy(), V)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)


def test_class_count_mismatch_and_bad_specs_are_rejected(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw, rt = _case(n_t=6)
    k3 = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob, row_types=rt)
    plan = aw.aw_plan_create(ctx, vd, k3)
    # the same geometry but 2 types: 4 classes, not 9
    k2 = aw.aw_make_kernels(ctx, **{**kw, "type_leak": TYPE_LEAK[:2]})
    grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
    vis = torch.as_tensor(sy.random_vis(ob.nvis, 4, seed=1), device="cuda")
    with pytest.raises(RuntimeError):
        aw.aw_grid(ctx, plan, k2, vis, None, grid)
    with pytest.raises(RuntimeError):
        aw.aw_make_kernels(ctx, **{**kw, "type_leak": TYPE_LEAK * 6})          # 18 types
    with pytest.raises(RuntimeError):
        aw.aw_make_kernels(ctx, **{**kw, "npol": 1, "supports": [8] * kw["nw"]})  # no Mueller term
    # the surrogate has no baseline-class input
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, seed=5, D=1.0,
                                 norm_supports=list(kw["supports"]), w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                                 chi_c=0.0, chi_h=1.5, out_scale=0.02)
    with pytest.raises(RuntimeError):
        aw.aw_surrogate_tables(ctx, sur, k3, reject_rel=0.1)
    with pytest.raises(RuntimeError):
        aw.aw_grid_learned(ctx, plan, sur, k3, vis, None, grid)
