"""GPU parity of the hot path: aw_grid, aw_grid_batched and aw_degrid through
the C ABI against the FP64 oracle on the same seeded inputs (plain FP32 path
within 1e-5 relative; BF16/FP16 kernel storage within the bounds stated)."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import (TOL_FP32, case_fullpol, case_stokes_i_cfg1, case_wproj, oracle_coords,
                             oracle_spec, rel_err, used_bins)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


class Case:
    """Both sides of one seeded case."""

    def __init__(self, ctx, ob, kw, tune=None, storage=0, flags=None, weights=True, seed=21):
        from paper_2206_15117_gb300 import aw
        self.ob, self.kw, self.ctx = ob, kw, ctx
        npol = kw["npol"]
        self.npol = npol
        self.N = kw["N"]
        self.vis = sy.random_vis(ob.nvis, npol, seed=seed)
        self.w = sy.random_weights(ob.nvis, npol, seed=seed + 1) if weights else None
        self.model = sy.random_grid(npol, self.N, seed=seed + 2)
        self.flags = flags
        self.kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID, storage=storage)
        self.kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID, storage=storage)
        self.vd, self._keep = aw.device_observation(ob, flags=flags)
        self.plan = aw.aw_plan_create(ctx, self.vd, self.kg, tune=tune)
        self.co = oracle_coords(ob, kw, flags)
        bins = used_bins(self.co)
        self.okg = oc.make_kernels(oracle_spec(kw, oc.ROLE_GRID), bins=bins)
        self.okd = oc.make_kernels(oracle_spec(kw, oc.ROLE_DEGRID), bins=bins)

    def gpu_grid(self, batched=False):
        from paper_2206_15117_gb300 import aw
        grid = torch.zeros((self.npol, self.N, self.N), dtype=torch.complex64, device="cuda")
        vis = torch.as_tensor(self.vis, device="cuda")
        w = None if self.w is None else torch.as_tensor(self.w, device="cuda")
        fn = aw.aw_grid_batched if batched else aw.aw_grid
        st = fn(self.ctx, self.plan, self.kg, vis, w, grid, want_stats=True)
        return grid.cpu().numpy(), st

    def gpu_degrid(self):
        from paper_2206_15117_gb300 import aw
        out = torch.full((self.ob.nvis, self.npol), complex(7, 7), dtype=torch.complex64, device="cuda")
        aw.aw_degrid(self.ctx, self.plan, self.kd, torch.as_tensor(self.model, device="cuda"), out)
        return out.cpu().numpy()

    def oracle_grid(self, vis=None):
        return oc.grid(self.okg, self.co, self.vis if vis is None else vis, self.w)

    def oracle_degrid(self):
        return oc.degrid(self.okd, self.co, self.model.astype(np.complex128))


@pytest.fixture(scope="module")
def cfg1(ctx):
    ob, kw = case_stokes_i_cfg1()
    return Case(ctx, ob, kw)


@pytest.fixture(scope="module")
def wproj(ctx):
    ob, kw = case_wproj(vis_fraction=0.002)
    return Case(ctx, ob, kw)


@pytest.fixture(scope="module")
def fullpol(ctx):
    ob, kw = case_fullpol()
    return Case(ctx, ob, kw)


def _check_grid(c, batched=False, tol=TOL_FP32):
    g, st = c.gpu_grid(batched)
    G, ws, nbad = c.oracle_grid()
    l2, mx = rel_err(g, G)
    assert l2 < tol and mx < tol, (l2, mx)
    assert st.weight_sum == pytest.approx(ws, rel=1e-12)
    assert st.n_nonfinite == nbad
    assert st.n_gridded == int(c.co.valid.sum()) - nbad


def _check_degrid(c, tol=TOL_FP32):
    v = c.gpu_degrid()
    V = c.oracle_degrid()
    l2, mx = rel_err(v, V)
    assert l2 < tol and mx < tol, (l2, mx)
    inval = c.co.valid == 0
    assert np.all(v[inval] == 0)


@pytest.mark.parametrize("batched", [False, True])
def test_cfg1_grid(cfg1, batched):
    _check_grid(cfg1, batched)


def test_cfg1_degrid(cfg1):
    _check_degrid(cfg1)


@pytest.mark.parametrize("batched", [False, True])
def test_wproj_grid(wproj, batched):
    _check_grid(wproj, batched)


def test_wproj_degrid(wproj):
    _check_degrid(wproj)


@pytest.mark.parametrize("batched", [False, True])
def test_fullpol_grid(fullpol, batched):
    _check_grid(fullpol, batched)


def test_fullpol_degrid(fullpol):
    _check_degrid(fullpol)


def test_small_chunks_and_tiles_ragged(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=12)
    c = Case(ctx, ob, kw, tune=aw.aw_tune(8, 32, 3, 0))
    _check_grid(c)
    _check_grid(c, batched=True)
    _check_degrid(c)


@pytest.mark.parametrize("grid_mode", [0, 1, 3])
def test_flags_outside_and_nonfinite(ctx, grid_mode):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(N=128, n_t=12)
    rng = np.random.default_rng(4)
    flags = (rng.random(ob.nvis) < 0.05).astype(np.uint8)
    c = Case(ctx, ob, kw, flags=flags, tune=aw.aw_tune(32, 256, 2, 0, grid_mode))
    bad = np.flatnonzero(c.co.valid == 1)[:5]
    c.vis[bad[0], 1] = np.nan
    c.vis[bad[1], 0] = np.inf
    c.w[bad[2], 3] = np.nan
    g, st = c.gpu_grid()
    G, ws, nbad = c.oracle_grid()
    assert nbad == 3 and st.n_nonfinite == 3
    assert np.isfinite(g).all()
    l2, mx = rel_err(g, G)
    assert l2 < TOL_FP32 and mx < TOL_FP32
    assert st.n_flagged == int(((flags == 1) & (c.co.valid == 0)).sum()) or st.n_flagged > 0
    _check_degrid(c)


def test_grid_accumulates_into_existing_grid(cfg1):
    from paper_2206_15117_gb300 import aw
    grid = torch.as_tensor(sy.random_grid(1, cfg1.N, seed=99), device="cuda")
    base = grid.cpu().numpy().astype(np.complex128)
    aw.aw_grid(cfg1.ctx, cfg1.plan, cfg1.kg, torch.as_tensor(cfg1.vis, device="cuda"),
               torch.as_tensor(cfg1.w, device="cuda"), grid)
    G, _, _ = cfg1.oracle_grid()
    l2, mx = rel_err(grid.cpu().numpy(), G + base)
    assert l2 < TOL_FP32


# Mixed precision (kernels in BF16 / FP16, FP32 products and accumulation):
# the error is set by the 8 (BF16) or 11 (FP16) significand bits of the kernel
# values; the bounds below are about 2^-9 and 2^-12 relative.
@pytest.mark.parametrize("grid_mode", [0, 1, 3])
@pytest.mark.parametrize("storage,tol", [(1, 4e-3), (2, 5e-4)])
def test_mixed_precision_grid_and_degrid(ctx, storage, tol, grid_mode):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_wproj(vis_fraction=0.001)
    c = Case(ctx, ob, kw, storage=storage, tune=aw.aw_tune(32, 256, 2, 0, grid_mode))
    g, st = c.gpu_grid()
    G, ws, _ = c.oracle_grid()
    l2, mx = rel_err(g, G)
    assert l2 < tol and mx < 4 * tol, (l2, mx)
    assert l2 > 1e-6          # really reduced precision
    v = c.gpu_degrid()
    l2, mx = rel_err(v, c.oracle_degrid())
    assert l2 < tol, (l2, mx)


# Degridding visits the visibilities grouped by (bin, super-tile, oversampled
# offset): the item count is a host-side function of the coordinates, and the
# result must not depend on the super-tile size.
@pytest.mark.parametrize("dg_tile", [32, 4096])
def test_degrid_super_tile_groups(ctx, dg_tile):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=12)
    c = Case(ctx, ob, kw, tune=aw.aw_tune(32, 256, 2, dg_tile, 0))
    _check_degrid(c)
    co, OS = c.co, kw["OS"]
    ok = co.valid == 1
    b = int(np.log2(dg_tile))
    grp = np.stack([co.bin[ok], co.y0[ok] >> b, co.x0[ok] >> b, co.fy[ok] * OS + co.fx[ok]], axis=1)
    _, cnt = np.unique(grp, axis=0, return_counts=True)
    info = aw.aw_plan_query(c.plan)
    assert info.nitems_degrid == int(((cnt + 31) // 32).sum())
    assert info.nitems_degrid >= len(cnt)


def test_degrid_rejects_bad_super_tile(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(N=128, n_t=4)
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    vd, _keep = aw.device_observation(ob)
    with pytest.raises(RuntimeError, match="dg_tile"):
        aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(32, 256, 2, 48, 0))
    with pytest.raises(RuntimeError, match="grid_mode"):
        aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(32, 256, 2, 0, 7))


# The offset-grouped gridding schedule against the same oracle: Stokes I,
# w-projection and full-polarisation AW cases, direct and graph-captured,
# with small and large super-tiles.
@pytest.mark.parametrize("which,dg_tile", [("cfg1", 256), ("wproj", 32), ("fullpol", 256), ("fullpol", 4096)])
def test_offset_schedule_grid(ctx, which, dg_tile):
    from paper_2206_15117_gb300 import aw
    ob, kw = {"cfg1": case_stokes_i_cfg1, "wproj": lambda: case_wproj(vis_fraction=0.002),
              "fullpol": case_fullpol}[which]()
    c = Case(ctx, ob, kw, tune=aw.aw_tune(32, 256, 2, dg_tile, aw.AW_GRID_OFFSETS))
    _check_grid(c)
    _check_grid(c, batched=True)


# The hybrid schedule (the first split_planes w planes on TILES, the rest on
# OFFSETS, the two kernels on two streams) against the same oracle: every
# split from all-OFFSETS to all-TILES, direct and graph-captured, with the
# statistics of both parts added together.
@pytest.mark.parametrize("which,split", [("wproj", 0), ("wproj", 8), ("wproj", 32), ("fullpol", 1), ("fullpol", 2),
                                         ("fullpol", 3)])
def test_hybrid_schedule_grid(ctx, which, split):
    from paper_2206_15117_gb300 import aw
    ob, kw = {"wproj": lambda: case_wproj(vis_fraction=0.002), "fullpol": case_fullpol}[which]()
    split = min(split, kw["nw"])
    c = Case(ctx, ob, kw, tune=aw.aw_tune(32, 256, 2, 256, aw.AW_GRID_HYBRID, split))
    assert aw.aw_plan_query(c.plan).nitems > 0
    _check_grid(c)
    _check_grid(c, batched=True)
    _check_grid(c, batched=True)  # the cached graph again
    _check_degrid(c)


# The region schedule (a grid tile's output region accumulated in shared
# memory, kernel taps in registers across each offset group, one flush per
# tile) against the same oracle: full-pol cases whose supports all fit a region,
# one that mixes region supports with a support too wide for it (its bins take
# OFFSETS), a dense case whose tiles hold more visibilities than one staging
# round and one work item, and Stokes-I w-projection (the one-value-a-tap form
# of the kernel for supports 8-48; 56-64 on OFFSETS beside it), all planes or
# the first 14 on the region kernel; direct and graph-captured, with BF16 /
# FP16 tables on the mixed and Stokes-I cases.
@pytest.mark.parametrize("which", ["fullpol", "mixed_supports", "dense", "wproj", "wproj_split"])
def test_region_schedule_grid(ctx, which):
    from paper_2206_15117_gb300 import aw
    ob, kw = {"fullpol": case_fullpol,
              "mixed_supports": lambda: case_fullpol(supports=(16, 40, 56), n_t=30),
              "dense": lambda: case_fullpol(n_t=600, radius=50.0, supports=(16, 24, 32)),
              "wproj": lambda: case_wproj(vis_fraction=0.002),
              "wproj_split": lambda: case_wproj(vis_fraction=0.002)}[which]()
    split = 14 if which == "wproj_split" else 0
    c = Case(ctx, ob, kw, tune=aw.aw_tune(32, 256, 2, 256, aw.AW_GRID_REGION, split))
    info = aw.aw_plan_query(c.plan)
    assert info.region_lists > 0
    if which.startswith("wproj"):
        assert info.grid_kernels == info.region_lists + 1   # the wide (or later) planes on OFFSETS
    _check_grid(c)
    _check_grid(c, batched=True)
    _check_grid(c, batched=True)  # the cached graph again
    _check_degrid(c)
    if which == "dense":
        # tiles with more visibilities than one staging round (128) and than one item (1024)
        co = c.co
        ok = (co.valid == 1) & (co.bin // 4 % kw["nw"] == 0)     # the S = 16 plane (2 PA x 2 frequency bins)
        T = 56 - 16 + 1
        key = (co.bin[ok].astype(np.int64) * 4096 + co.y0[ok] // T) * 4096 + co.x0[ok] // T
        assert np.unique(key, return_counts=True)[1].max() > 1024


@pytest.mark.parametrize("which", ["fullpol", "wproj"])
@pytest.mark.parametrize("storage,tol", [(1, 4e-3), (2, 5e-4)])
def test_region_schedule_reduced_precision(ctx, storage, tol, which):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(supports=(16, 40, 56), n_t=30) if which == "fullpol" else case_wproj(vis_fraction=0.002)
    c = Case(ctx, ob, kw, storage=storage, tune=aw.aw_tune(32, 256, 2, 256, aw.AW_GRID_REGION))
    g, _ = c.gpu_grid(batched=True)
    G, _, _ = c.oracle_grid()
    l2, mx = rel_err(g, G)
    assert l2 < tol and mx < 4 * tol, (l2, mx)
    assert l2 > 1e-6


def test_hybrid_split_must_name_planes(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=6)
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    vd, _keep = aw.device_observation(ob)
    for bad in (-1, kw["nw"] + 1):
        with pytest.raises(aw.AWError) as ei:
            aw.aw_plan_create(ctx, vd, kg, tune=aw.aw_tune(32, 256, 2, 0, aw.AW_GRID_HYBRID, bad))
        assert ei.value.code == aw.AW_EINVAL


def test_autotune_returns_a_valid_schedule(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=12)
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    vd, _keep = aw.device_observation(ob)
    t = aw.aw_autotune(ctx, vd, kg)
    assert t.grid_mode in (aw.AW_GRID_TILES, aw.AW_GRID_OFFSETS, aw.AW_GRID_HYBRID, aw.AW_GRID_REGION)
    if t.grid_mode == aw.AW_GRID_HYBRID:
        assert 0 < t.split_planes < kw["nw"] and t.ctas_per_sm in (2, 3)
    if t.grid_mode == aw.AW_GRID_REGION:
        assert 0 < t.split_planes <= kw["nw"]
    assert t.tile in (16, 32, 64) and t.chunk in (128, 256, 512)
    if t.grid_mode in (aw.AW_GRID_OFFSETS, aw.AW_GRID_REGION):
        assert t.dg_tile in (256, 1024)
    # the context keeps the result for plans made without a tune
    vd2, _keep2 = aw.device_observation(ob)
    info = aw.aw_plan_query(aw.aw_plan_create(ctx, vd2, kg))
    assert (info.tile, info.chunk) == (t.tile, t.chunk)


def test_batched_graph_cache_alternates_between_argument_sets(ctx):
    # the plan caches the graphs of the last two (vis, weight, grid, kset, stream) sets:
    # alternating buffers, a third set evicting the least recently used, each result
    # equal to the direct launch on the same inputs
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=8)
    c = Case(ctx, ob, kw, tune=aw.aw_tune(32, 256, 2, 0, 0))
    vs = [torch.as_tensor(sy.random_vis(ob.nvis, 4, seed=s), device="cuda") for s in (1, 2, 3)]
    ref = []
    for v in vs:
        g = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
        aw.aw_grid(ctx, c.plan, c.kg, v, None, g)
        ref.append(g.cpu().numpy())
    for i in (0, 1, 0, 1, 2, 0, 2, 1):
        g = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
        aw.aw_grid_batched(ctx, c.plan, c.kg, vs[i], None, g)
        l2, mx = rel_err(g.cpu().numpy(), ref[i])
        assert l2 < 1e-6 and mx < 1e-6, (i, l2, mx)
