"""GPU: per-visibility coordinates (FP64, bit-exact against the oracle) and the
device key sort (a valid, stable sort of the plan's keys)."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from tests.gpu_cases import case_fullpol, case_stokes_i_cfg1, case_wproj, oracle_coords

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _gpu_coords(ctx, ob, kw, flags=None, tune=None):
    from paper_2206_15117_gb300 import aw
    ks = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob, "cuda:0", flags=flags)
    plan = aw.aw_plan_create(ctx, vd, ks, tune=tune)
    n = ob.nvis
    out = {k: torch.empty(n, dtype=torch.int32, device="cuda") for k in ("x0", "y0", "fx", "fy", "bin")}
    out["flip"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    out["valid"] = torch.empty(n, dtype=torch.uint8, device="cuda")
    aw.aw_plan_coords(plan, **out)
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    aw.aw_plan_order(plan, perm)
    torch.cuda.synchronize()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    return res, perm.cpu().numpy().view(np.uint32), aw.aw_plan_query(plan)


@pytest.mark.parametrize("case", ["cfg1", "wproj", "fullpol", "fullpol_flags"])
def test_coordinates_bit_exact(ctx, case):
    flags = None
    if case == "cfg1":
        ob, kw = case_stokes_i_cfg1()
    elif case == "wproj":
        ob, kw = case_wproj(vis_fraction=0.01)
    else:
        ob, kw = case_fullpol(N=128)          # small grid: many visibilities fall outside
        if case == "fullpol_flags":
            flags = (np.random.default_rng(1).random(ob.nvis) < 0.1).astype(np.uint8)
    res, perm, info = _gpu_coords(ctx, ob, kw, flags)
    co = oracle_coords(ob, kw, flags)
    valid = co.valid == 1
    np.testing.assert_array_equal(res["valid"], co.valid)
    for k in ("x0", "y0", "fx", "fy"):
        np.testing.assert_array_equal(res[k][valid], getattr(co, k)[valid])
    np.testing.assert_array_equal(res["bin"], co.bin)
    np.testing.assert_array_equal(res["flip"], co.flip)
    assert info.nvalid == int(valid.sum())
    assert info.nvis == ob.nvis
    if case == "fullpol":
        assert info.n_outside > 0
    if flags is not None:
        assert info.n_flagged > 0


@pytest.mark.parametrize("tile,chunk", [(32, 256), (16, 32), (64, 2048)])
def test_sort_is_stable_key_order(ctx, tile, chunk):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_wproj(vis_fraction=0.005)
    res, perm, info = _gpu_coords(ctx, ob, kw, tune=aw.aw_tune(tile, chunk, 2, 0))
    co = oracle_coords(ob, kw)
    n = ob.nvis
    assert sorted(perm.tolist()) == list(range(n))           # a permutation
    nv = int(co.valid.sum())
    assert np.all(co.valid[perm[:nv]] == 1) and np.all(co.valid[perm[nv:]] == 0)
    # key of the method: (bin, tile y, tile x, y in tile, x in tile)
    ntx = (kw["N"] + tile - 1) // tile
    b = co.bin.astype(np.int64)
    key = ((b * ntx + co.y0 // tile) * ntx + co.x0 // tile) * tile * tile + (co.y0 % tile) * tile + co.x0 % tile
    ks = key[perm[:nv]]
    assert np.all(np.diff(ks) >= 0)
    ties = np.diff(ks) == 0
    assert np.all(np.diff(perm[:nv].astype(np.int64))[ties] > 0)   # stable
    assert info.nitems >= (nv + chunk - 1) // chunk


def test_empty_visibility_set(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_stokes_i_cfg1(time_samples=2)
    ob.row_of_vis = ob.row_of_vis[:0]
    ob.chan_of_vis = ob.chan_of_vis[:0]
    ks = aw.aw_make_kernels(ctx, **kw)
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, ks)
    info = aw.aw_plan_query(plan)
    assert info.nvis == 0 and info.nvalid == 0 and info.nitems == 0
    grid = torch.zeros((1, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
    st = aw.aw_grid(ctx, plan, ks, torch.zeros(1, dtype=torch.complex64, device="cuda"), None, grid,
                    want_stats=True)
    assert st.n_gridded == 0 and st.weight_sum == 0.0
    assert float(grid.abs().max()) == 0.0


def test_invalid_arguments_are_rejected(ctx):
    from paper_2206_15117_gb300 import aw
    with pytest.raises(aw.AWError) as e:
        aw.aw_make_kernels(ctx, N=100, dl=1e-4, OS=4, supports=[7])
    assert e.value.code == aw.AW_EINVAL
    with pytest.raises(aw.AWError) as e:
        aw.aw_make_kernels(ctx, N=128, dl=1e-4, OS=3, supports=[7])   # odd support, odd OS
    assert e.value.code == aw.AW_EINVAL
    with pytest.raises(aw.AWError):
        aw.aw_make_kernels(ctx, N=128, dl=1e-4, OS=4, npol=2, supports=[8])
