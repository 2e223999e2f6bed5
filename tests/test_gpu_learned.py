"""GPU: gridding with the surrogate evaluated inline (aw_grid_learned,
tensor-core MLP inside the gridding kernel) against the FP64 oracle running
the same network at the same continuous coordinates; and its exact-table
fallback for rejected w planes against the oracle's exact gridding."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from oracle import mlp as omlp
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, case_fullpol, oracle_coords, oracle_spec, rel_err, used_bins

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _setup(ctx, n_t=10):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=n_t)
    exact = aw.aw_make_kernels(ctx, **kw)
    scales = dict(D=1.0, norm_supports=list(kw["supports"]), w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                  chi_c=0.0, chi_h=1.5, out_scale=0.02)
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, seed=5, **scales)
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, exact)
    vis = sy.random_vis(ob.nvis, 4, seed=31)
    w = sy.random_weights(ob.nvis, 4, seed=32)
    return ob, kw, exact, sur, plan, vis, w, scales, (vd, keep)


@pytest.mark.parametrize("engine", [0, 1])
def test_inline_surrogate_gridding_matches_oracle(ctx, engine):
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, vis, w, scales, keep = _setup(ctx)
    aw.aw_surrogate_set_engine(sur, engine)
    grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
    st = aw.aw_grid_learned(ctx, plan, sur, exact, torch.as_tensor(vis, device="cuda"),
                            torch.as_tensor(w, device="cuda"), grid, want_stats=True)
    g = grid.cpu().numpy()
    spec = oracle_spec(kw)
    co = oracle_coords(ob, kw)
    p = aw.aw_surrogate_get_params(sur)
    sizes = omlp.layer_sizes(5, 128, 4, 16)
    sc = (scales["D"], scales["norm_supports"], scales["w_max"], scales["f_c"], scales["f_h"], scales["chi_c"],
          scales["chi_h"],
          scales["out_scale"])
    G = omlp.grid_inline(p, sizes, 30.0, sc, spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, co, vis, w)
    l2, mx = rel_err(g, G)
    # FP16 activations between the tensor-core layers: about 2^-11 relative per
    # value, a few 1e-3 after four layers
    assert l2 < 1e-2, (l2, mx)
    assert np.abs(G).max() > 0
    _, ws, _ = oc.grid(oc.make_kernels(spec, bins=used_bins(co)), co, vis, w)
    assert st.weight_sum == pytest.approx(ws, rel=1e-12)


@pytest.mark.parametrize("engine", [0, 1])
def test_rejected_planes_fall_back_to_exact_tables(ctx, engine):
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, vis, w, scales, keep = _setup(ctx)
    aw.aw_surrogate_set_engine(sur, engine)
    learned, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=0.0)   # reject every plane
    assert nrej == aw.aw_kernel_set_info(exact).nbins
    grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
    aw.aw_grid_learned(ctx, plan, sur, exact, torch.as_tensor(vis, device="cuda"), torch.as_tensor(w, device="cuda"),
                       grid)
    co = oracle_coords(ob, kw)
    G, _, _ = oc.grid(oc.make_kernels(oracle_spec(kw), bins=used_bins(co)), co, vis, w)
    l2, mx = rel_err(grid.cpu().numpy(), G)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)


def test_tensor_core_engines_agree(ctx):
    # the two tensor-core engines run the same FP16 network with FP32 accumulation:
    # they differ by FP32 summation order and occasional FP16 roundings of activations
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, vis, w, scales, keep = _setup(ctx, n_t=16)
    out = []
    for engine in (aw.AW_ENGINE_MMA_SYNC, aw.AW_ENGINE_TCGEN05):
        aw.aw_surrogate_set_engine(sur, engine)
        grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
        aw.aw_grid_learned(ctx, plan, sur, exact, torch.as_tensor(vis, device="cuda"),
                           torch.as_tensor(w, device="cuda"), grid)
        out.append(grid.cpu().numpy())
    l2, mx = rel_err(out[1], out[0])
    assert l2 < 2e-3, (l2, mx)
    with pytest.raises(RuntimeError):
        aw.aw_surrogate_set_engine(sur, 7)


@pytest.mark.parametrize("engine", [0, 1])
def test_per_channel_frequency_matches_oracle(ctx, engine):
    # the network fed each visibility's own channel frequency instead of its
    # beam-frequency bin centre (the case has two channels per bin)
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, vis, w, scales, keep = _setup(ctx)
    aw.aw_surrogate_set_engine(sur, engine)
    p = aw.aw_surrogate_get_params(sur)
    sizes = omlp.layer_sizes(5, 128, 4, 16)
    sc = (scales["D"], scales["norm_supports"], scales["w_max"], scales["f_c"], scales["f_h"], scales["chi_c"],
          scales["chi_h"], scales["out_scale"])
    spec = oracle_spec(kw)
    co = oracle_coords(ob, kw)
    out = {}
    for mode in (aw.AW_FREQ_BIN, aw.AW_FREQ_CHANNEL):
        aw.aw_surrogate_set_freq_mode(sur, mode)
        grid = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
        aw.aw_grid_learned(ctx, plan, sur, exact, torch.as_tensor(vis, device="cuda"), torch.as_tensor(w, device="cuda"),
                           grid)
        out[mode] = grid.cpu().numpy()
    G = omlp.grid_inline(p, sizes, 30.0, sc, spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, co, vis, w,
                         per_channel=True)
    l2, mx = rel_err(out[aw.AW_FREQ_CHANNEL], G)
    assert l2 < 1e-2, (l2, mx)
    # the mode matters on this case
    assert rel_err(out[aw.AW_FREQ_BIN], G)[0] > 3 * l2
    with pytest.raises(RuntimeError):
        aw.aw_surrogate_set_freq_mode(sur, 2)


def _setup_degrid(ctx, n_t=10):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=n_t)
    exact = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    scales = dict(D=1.0, norm_supports=list(kw["supports"]), w_max=kw["w_max"], f_c=1.35e9, f_h=0.15e9,
                  chi_c=0.0, chi_h=1.5, out_scale=0.02)
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, seed=6, **scales)
    flags = (np.random.default_rng(40).random(ob.nvis) < 0.05).astype(np.uint8)
    vd, keep = aw.device_observation(ob, flags=flags)
    plan = aw.aw_plan_create(ctx, vd, exact)
    model = sy.random_grid(4, kw["N"], seed=41)
    co = oc.coords(oracle_spec(kw, oc.ROLE_DEGRID), ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin,
                   ob.fbin, flags)
    return ob, kw, exact, sur, plan, model, scales, co, (vd, keep)


@pytest.mark.parametrize("freq_mode", [0, 1])
def test_inline_surrogate_degridding_matches_oracle(ctx, freq_mode):
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, model, scales, co, keep = _setup_degrid(ctx)
    aw.aw_surrogate_set_freq_mode(sur, freq_mode)
    out = torch.full((ob.nvis, 4), complex(3, 3), dtype=torch.complex64, device="cuda")
    aw.aw_degrid_learned(ctx, plan, sur, exact, torch.as_tensor(model, device="cuda"), out)
    got = out.cpu().numpy()
    p = aw.aw_surrogate_get_params(sur)
    sc = (scales["D"], scales["norm_supports"], scales["w_max"], scales["f_c"], scales["f_h"], scales["chi_c"],
          scales["chi_h"], scales["out_scale"])
    ref = omlp.degrid_inline(p, omlp.layer_sizes(5, 128, 4, 16), 30.0, sc, oracle_spec(kw, oc.ROLE_DEGRID), ob.uvw,
                             ob.row_of_vis, ob.chan_of_vis, ob.freq, co, model, per_channel=bool(freq_mode))
    l2, mx = rel_err(got, ref)
    # FP16 activations between the tensor-core layers, as for inline gridding
    assert l2 < 1e-2, (l2, mx)
    assert np.abs(ref).max() > 0
    assert np.all(got[co.valid == 0] == 0) and (co.valid == 0).any()


def test_inline_degridding_rejected_planes_use_exact_tables(ctx):
    from paper_2206_15117_gb300 import aw
    ob, kw, exact, sur, plan, model, scales, co, keep = _setup_degrid(ctx)
    tabs, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=0.0)
    assert nrej == aw.aw_kernel_set_info(exact).nbins
    out = torch.empty((ob.nvis, 4), dtype=torch.complex64, device="cuda")
    aw.aw_degrid_learned(ctx, plan, sur, exact, torch.as_tensor(model, device="cuda"), out)
    ref = oc.degrid(oc.make_kernels(oracle_spec(kw, oc.ROLE_DEGRID), bins=used_bins(co)), co,
                    model.astype(np.complex128))
    l2, mx = rel_err(out.cpu().numpy(), ref)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    # the other engine and a gridding-role fallback are refused
    aw.aw_surrogate_set_engine(sur, aw.AW_ENGINE_MMA_SYNC)
    with pytest.raises(RuntimeError):
        aw.aw_degrid_learned(ctx, plan, sur, exact, torch.as_tensor(model, device="cuda"), out)
    aw.aw_surrogate_set_engine(sur, aw.AW_ENGINE_TCGEN05)
    kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
    with pytest.raises(RuntimeError):
        aw.aw_degrid_learned(ctx, plan, sur, kg, torch.as_tensor(model, device="cuda"), out)
