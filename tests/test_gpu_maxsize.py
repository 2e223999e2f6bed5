"""GPU parity at the largest grid the ABI accepts (N = 16384): Stokes-I
w-projection gridding against the FP64 oracle over the whole grid, and
degridding against the oracle on sampled visibilities, with baselines that
reach the outer cells of the grid (and a few that fall outside it)."""
import math

import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, rel_err, used_bins

pytestmark = pytest.mark.gpu

N = 16384


@pytest.fixture(scope="module")
def case():
    from paper_2206_15117_gb300 import aw
    ctx = aw.aw_create(0)
    ob = sy.small_observation(n_ant=24, radius_m=3000.0, n_t=12, freq=(1.2e9, 1.45e9), z_spread_m=20.0)
    # the cell size puts the 12 longest samples (in cells) past the edge and the next ones a few
    # cells inside it
    r = np.abs(ob.uvw[ob.row_of_vis, :2]).max(1) * ob.freq[ob.chan_of_vis] / oc.C_LIGHT
    dl = (0.5 - 6.0 / N) / np.quantile(r, 1 - 12 / ob.nvis)
    nw = 8
    kw = dict(N=N, dl=dl, OS=8, W=7.0, npol=1, nw=nw, w_max=ob.w_max, supports=[8, 8, 12, 12, 16, 16, 20, 24])
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, kg)
    co = oc.coords(oc.KernelSpec(**kw), ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    return dict(aw=aw, ctx=ctx, ob=ob, kw=kw, kg=kg, kd=kd, vd=vd, keep=keep, plan=plan, co=co)


def test_coordinates_reach_the_grid_edge(case):
    co, aw = case["co"], case["aw"]
    info = aw.aw_plan_query(case["plan"])
    assert info.nvalid == int(co.valid.sum())
    v = co.valid == 1
    assert max(co.x0[v].max(), co.y0[v].max()) > N - 128
    assert min(co.x0[v].min(), co.y0[v].min()) < 128
    assert 0 < info.n_outside == int((co.valid == 0).sum())


def test_grid_matches_oracle_at_n16384(case):
    aw, ob, kw, co = case["aw"], case["ob"], case["kw"], case["co"]
    vis = sy.random_vis(ob.nvis, 1, seed=91)
    w = sy.random_weights(ob.nvis, 1, seed=92)
    grid = torch.zeros((1, N, N), dtype=torch.complex64, device="cuda")
    st = aw.aw_grid_batched(case["ctx"], case["plan"], case["kg"], torch.as_tensor(vis, device="cuda"),
                            torch.as_tensor(w, device="cuda"), grid, want_stats=True)
    G, ws, _ = oc.grid(oc.make_kernels(oc.KernelSpec(**kw), bins=used_bins(co)), co, vis, w)
    g = grid.cpu().numpy()
    del grid
    torch.cuda.empty_cache()
    l2, mx = rel_err(g, G)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    assert st.weight_sum == pytest.approx(ws, rel=1e-12)


def test_sampled_degrid_matches_oracle_at_n16384(case):
    aw, ob, kw, co = case["aw"], case["ob"], case["kw"], case["co"]
    model = sy.random_grid(1, N, seed=93)
    out = torch.empty((ob.nvis, 1), dtype=torch.complex64, device="cuda")
    aw.aw_degrid(case["ctx"], case["plan"], case["kd"], torch.as_tensor(model, device="cuda"), out)
    v = out.cpu().numpy()
    rng = np.random.default_rng(94)
    # the outermost valid samples and a random set
    valid = np.flatnonzero(co.valid == 1)
    edge = valid[np.argsort(-np.maximum(np.abs(co.x0[valid] - N // 2), np.abs(co.y0[valid] - N // 2)))[:8]]
    idx = np.unique(np.concatenate([edge, rng.choice(ob.nvis, 24, replace=False)]))
    ref = oc.degrid_sampled(oc.KernelSpec(**kw, role=oc.ROLE_DEGRID), model, co, idx)
    l2, mx = rel_err(v[idx], ref)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    assert np.all(v[co.valid == 0] == 0)
