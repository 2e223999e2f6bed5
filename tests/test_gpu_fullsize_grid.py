"""Element-wise gridding parity on the benchmark's own geometry: the full-pol
AW workload (4096^2 x 4 grid over 3 deg, 32 w planes with supports 16..72,
8 parallactic-angle x 4 beam-frequency bins, OS 8), restricted to every
visibility (capped) of eight bins whose w planes cover each support of the
set, gridded by each schedule the benchmark can time — TILES, OFFSETS, the
HYBRID split at 7 planes and REGION, each one-shot and graph-captured — and
compared cell by cell with the FP64 oracle (relative L2 and max-abs within
1e-5).  BF16 and FP16 tables are held to their stated bounds (4e-3 / 5e-4),
and the degridder on the same subset to 1e-5.  The kernel blocks of supports
32..72 (Sec. 3.2's full-pol kernels of the wide w planes) are thereby
compared one by one, not only through the adjoint identity."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, rel_err

pytestmark = pytest.mark.gpu

PLANES = (0, 6, 11, 17, 20, 24, 27, 31)     # supports 16, 24, 32, 40, 48, 56, 64, 72
CAP = 12_000
SPLIT = 7


@pytest.fixture(scope="module")
def sub():
    import bench
    from paper_2206_15117_gb300 import aw
    ob, kw = bench.workload(2000)
    spec = oc.KernelSpec(**kw)
    sup = np.asarray(spec.supports)
    assert sorted(set(sup[list(PLANES)].tolist())) == [16, 24, 32, 40, 48, 56, 64, 72]
    rng = np.random.default_rng(2206)
    pairs = [(a, f) for a in range(spec.npa) for f in range(spec.nfb)]
    order = rng.permutation(len(pairs))
    picks, sel, pair_bins = [], [], {}

    def bins_of_pair(a, f):
        # the valid visibilities of one (PA, frequency) bin pair and their bins
        if (a, f) not in pair_bins:
            cand = np.flatnonzero((ob.pa_bin[ob.row_of_vis] == a) & (ob.fbin[ob.chan_of_vis] == f))
            co = oc.coords(spec, ob.uvw, ob.row_of_vis[cand], ob.chan_of_vis[cand], ob.freq, ob.pa_bin, ob.fbin)
            pair_bins[(a, f)] = (cand[co.valid == 1], co.bin[co.valid == 1])
        return pair_bins[(a, f)]

    for i, p in enumerate(PLANES):
        best = None
        for j in range(len(pairs)):
            a, f = pairs[order[(i + j) % len(pairs)]]
            cand, cbin = bins_of_pair(a, f)
            b = spec.bin_index(p, a, f)
            idx = cand[cbin == b]
            if best is None or idx.size > best[1].size:
                best = (b, idx)
            if idx.size >= 4000:
                break
        b, idx = best
        if idx.size > CAP:
            idx = np.sort(rng.choice(idx, CAP, replace=False))
        picks.append(int(b))
        sel.append(idx)
    keep = np.sort(np.concatenate(sel))
    sob = sy.Observation(**{**ob.__dict__, "row_of_vis": ob.row_of_vis[keep], "chan_of_vis": ob.chan_of_vis[keep]})
    co = oc.coords(spec, sob.uvw, sob.row_of_vis, sob.chan_of_vis, sob.freq, sob.pa_bin, sob.fbin)
    assert np.all(co.valid == 1) and sorted(set(co.bin.tolist())) == sorted(picks)
    vis = sy.random_vis(keep.size, 4, seed=41)
    G, ws, _ = oc.grid(oc.make_kernels(spec, bins=picks), co, vis)
    model = sy.random_grid(4, kw["N"], seed=42)
    V = oc.degrid(oc.make_kernels(oc.KernelSpec(**kw, role=oc.ROLE_DEGRID), bins=picks), co,
                  model.astype(np.complex128))
    ctx = aw.aw_create(0)
    vd, tens = aw.device_observation(sob)
    return dict(aw=aw, ctx=ctx, kw=kw, vd=vd, tens=tens, vis=vis, G=G, ws=ws, model=model, V=V, co=co,
                nvis=int(keep.size), kernels={})


def _kernels(s, storage, role):
    aw = s["aw"]
    key = (storage, role)
    if key not in s["kernels"]:
        s["kernels"][key] = aw.aw_make_kernels(s["ctx"], **s["kw"], role=role, storage=storage)
    return s["kernels"][key]


def _tune(aw, schedule):
    if schedule == "tiles":
        return aw.aw_tune(64, 128, 4, 1024, aw.AW_GRID_TILES, 0)
    if schedule == "offsets":
        return aw.aw_tune(64, 128, 5, 1024, aw.AW_GRID_OFFSETS, 0)
    if schedule == "region":
        return aw.aw_tune(64, 128, 2, 1024, aw.AW_GRID_REGION, 0)
    return aw.aw_tune(64, 128, 2, 1024, aw.AW_GRID_HYBRID, SPLIT)


def _grid(s, storage, schedule, batched):
    aw = s["aw"]
    kg = _kernels(s, storage, aw.AW_ROLE_GRID)
    plan = aw.aw_plan_create(s["ctx"], s["vd"], kg, tune=_tune(aw, schedule))
    N = s["kw"]["N"]
    g = torch.zeros((4, N, N), dtype=torch.complex64, device="cuda")
    v = torch.as_tensor(s["vis"], device="cuda")
    fn = aw.aw_grid_batched if batched else aw.aw_grid
    st = fn(s["ctx"], plan, kg, v, None, g, want_stats=True)
    torch.cuda.synchronize()
    return g.cpu().numpy(), st, plan


@pytest.mark.parametrize("batched", [False, True])
@pytest.mark.parametrize("schedule", ["tiles", "offsets", "hybrid", "region"])
def test_fp32_gridding_matches_oracle_on_the_bench_geometry(sub, schedule, batched):
    g, st, _ = _grid(sub, 0, schedule, batched)
    l2, mx = rel_err(g, sub["G"])
    assert l2 < TOL_FP32 and mx < TOL_FP32, (schedule, batched, l2, mx)
    assert abs(st.weight_sum - sub["ws"]) < 1e-9 * sub["ws"]
    # every support's block contributed: the oracle grid is non-zero far from
    # the small-support footprints too
    assert np.count_nonzero(sub["G"][0]) > 100_000


@pytest.mark.parametrize("schedule", ["tiles", "hybrid", "region"])
@pytest.mark.parametrize("storage,tol", [(1, 4e-3), (2, 5e-4)])
def test_reduced_precision_gridding_on_the_bench_geometry(sub, storage, tol, schedule):
    g, _, _ = _grid(sub, storage, schedule, True)
    l2, mx = rel_err(g, sub["G"])
    assert l2 < tol and mx < 4 * tol, (storage, schedule, l2, mx)
    assert l2 > 1e-6


@pytest.mark.parametrize("storage,tol", [(0, TOL_FP32), (1, 4e-3), (2, 5e-4)])
def test_degridding_matches_oracle_on_the_bench_geometry(sub, storage, tol):
    aw = sub["aw"]
    kd = _kernels(sub, storage, aw.AW_ROLE_DEGRID)
    plan = aw.aw_plan_create(sub["ctx"], sub["vd"], kd, tune=_tune(aw, "tiles"))
    out = torch.empty((sub["nvis"], 4), dtype=torch.complex64, device="cuda")
    aw.aw_degrid(sub["ctx"], plan, kd, torch.as_tensor(sub["model"], device="cuda"), out)
    l2, mx = rel_err(out.cpu().numpy(), sub["V"])
    assert l2 < tol and mx < (4 * tol if storage else tol), (storage, l2, mx)
