"""GPU parity at the benchmark's full size (64M visibilities, 4096^2 x 4,
1024 full-pol AW bins), in the launch configurations bench.py times (the tile
and the offset-grouped gridding schedules): sampled degridded visibilities
against the FP64 oracle computed one by one, and the adjoint identity of both
gridding schedules over the whole data (a grid cell of this workload sums
thousands of visibilities, so gridded cells are checked through that
identity rather than one by one)."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

N_SAMPLE = 24


@pytest.fixture(scope="module")
def full(request):
    import bench
    from paper_2206_15117_gb300 import aw
    ctx = aw.aw_create(0)
    ob, kw = bench.workload(2000)
    vd, keep = aw.device_observation(ob)
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    plan = aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(64, 128, 4, 0))
    plan_off = aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(64, 128, 5, 1024, aw.AW_GRID_OFFSETS))
    return dict(aw=aw, ctx=ctx, ob=ob, kw=kw, vd=vd, keep=keep, kg=kg, plan=plan, plans=[plan, plan_off])


def test_sampled_degrid_matches_oracle_at_full_size(full):
    aw, ctx, ob, kw, plan = full["aw"], full["ctx"], full["ob"], full["kw"], full["plan"]
    kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    model = sy.random_grid(4, kw["N"], seed=77)
    out = torch.empty((ob.nvis, 4), dtype=torch.complex64, device="cuda")
    aw.aw_degrid(ctx, plan, kd, torch.as_tensor(model, device="cuda"), out)
    rng = np.random.default_rng(9)
    idx = np.sort(rng.choice(ob.nvis, size=N_SAMPLE, replace=False))
    got = out[torch.as_tensor(idx, device="cuda")].cpu().numpy()
    spec = oc.KernelSpec(**kw, role=oc.ROLE_DEGRID)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis[idx], ob.chan_of_vis[idx], ob.freq, ob.pa_bin, ob.fbin)
    ref = oc.degrid_sampled(spec, model, co, np.arange(N_SAMPLE))
    err = np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert np.all(err < 1e-5), err
    assert len(set(co.bin.tolist())) > N_SAMPLE // 2       # spread over many bins


@pytest.mark.parametrize("schedule", [0, 1])
def test_adjoint_identity_of_the_gridders_at_full_size(full, schedule):
    aw, ctx, ob, kw, kg = full["aw"], full["ctx"], full["ob"], full["kw"], full["kg"]
    plan = full["plans"][schedule]
    ka = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_ADJOINT)
    N = kw["N"]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    v = torch.randn((ob.nvis, 4), dtype=torch.complex64, device="cuda", generator=gen)
    x = torch.randn((4, N, N), dtype=torch.complex64, device="cuda", generator=gen)
    g = torch.zeros((4, N, N), dtype=torch.complex64, device="cuda")
    aw.aw_grid_batched(ctx, plan, kg, v, None, g)
    dx = torch.empty_like(v)
    aw.aw_degrid(ctx, plan, ka, x, dx)
    # the w < 0 flip conjugates: the identity holds for the real inner product
    lhs = float(torch.sum((torch.conj(g) * x).real.double()))
    rhs = float(torch.sum((torch.conj(v) * dx).real.double()))
    scale = float(torch.linalg.vector_norm(g.double()) * torch.linalg.vector_norm(x.double()))
    # FP32 sums over 64M x 16 x S^2 terms: relative 1e-4 of the inner product,
    # which itself is ~1e-4 of the norm product for random data
    assert abs(lhs - rhs) < 1e-4 * abs(lhs) + 1e-8 * scale, (lhs, rhs, scale)
