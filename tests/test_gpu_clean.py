"""GPU parity of the cleaning loop through the C ABI: aw_image_to_grid,
aw_degrid_subtract and aw_psf_sidelobe against the oracle's transforms,
aw_hogbom bit-exact against the oracle's FP32 minor cycle on the same input,
and aw_clean end to end against the oracle's Cotton-Schwab loop."""
import numpy as np
import pytest
import torch

from oracle import clean as ocl
from oracle import core as oc
from tests.gpu_cases import TOL_FP32, case_fullpol, oracle_coords, oracle_spec, rel_err, used_bins
from tests.oracle_cases import small_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


class Setup:
    """One observation on both sides: kernels, plan, oracle coordinates."""

    def __init__(self, ctx, ob, kw):
        from paper_2206_15117_gb300 import aw
        self.ob, self.kw, self.ctx = ob, kw, ctx
        self.kg = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_GRID)
        self.kd = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
        self.vd, self._keep = aw.device_observation(ob)
        self.plan = aw.aw_plan_create(ctx, self.vd, self.kg)
        self.co = oracle_coords(ob, kw)
        bins = used_bins(self.co)
        self.okg = oc.make_kernels(oracle_spec(kw, oc.ROLE_GRID), bins=bins)
        self.okd = oc.make_kernels(oracle_spec(kw, oc.ROLE_DEGRID), bins=bins)


@pytest.fixture(scope="module")
def stokes_i(ctx):
    ob, base = small_case(npol=1, nw=1, S=10, W=7.0, OS=8, N=64, fov_deg=4.0, n_t=24)
    return Setup(ctx, ob, base)


@pytest.fixture(scope="module")
def fullpol(ctx):
    ob, kw = case_fullpol()
    return Setup(ctx, ob, kw)


def test_image_to_grid_matches_oracle(ctx, fullpol):
    from paper_2206_15117_gb300 import aw
    N = fullpol.kw["N"]
    img = np.random.default_rng(5).normal(size=(4, N, N)).astype(np.float32)
    g = torch.empty((4, N, N), dtype=torch.complex64, device="cuda")
    aw.aw_image_to_grid(ctx, fullpol.kd, _cuda(img), g)
    ref = oc.image_to_grid(img.astype(np.float64), fullpol.kw["W"])
    l2, mx = rel_err(g.cpu().numpy(), ref)
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)


@pytest.mark.parametrize("alias", [False, True])
def test_degrid_subtract_matches_oracle(ctx, fullpol, alias):
    from paper_2206_15117_gb300 import aw
    N, nvis = fullpol.kw["N"], fullpol.ob.nvis
    rng = np.random.default_rng(6)
    G = (rng.normal(size=(4, N, N)) + 1j * rng.normal(size=(4, N, N))).astype(np.complex64)
    V = (rng.normal(size=(nvis, 4)) + 1j * rng.normal(size=(nvis, 4))).astype(np.complex64)
    vin = _cuda(V)
    out = vin if alias else torch.empty_like(vin)
    aw.aw_degrid_subtract(ctx, fullpol.plan, fullpol.kd, _cuda(G), vin, out)
    pred = oc.degrid(fullpol.okd, fullpol.co, G.astype(np.complex128))
    ref = V.astype(np.complex128) - pred
    got = out.cpu().numpy()
    scale = max(np.abs(pred).max(), np.abs(V).max())
    assert np.abs(got - ref).max() < TOL_FP32 * scale
    inval = fullpol.co.valid == 0
    assert np.array_equal(got[inval], V[inval])


def test_psf_sidelobe_matches_oracle(ctx, stokes_i):
    from paper_2206_15117_gb300 import aw
    psf, _ = ocl.point_spread_function(stokes_i.okg, stokes_i.co, None, stokes_i.kw["W"])
    assert aw.aw_psf_sidelobe(ctx, _cuda(psf)) == ocl.psf_sidelobe(psf)
    # a sampled PSF of a larger image: main lobe and sidelobes of a sinc^2
    N = 256
    x = (np.arange(N) - N // 2) / 3.7
    s = np.sinc(x)
    big = (np.outer(s, s) ** 2 - 0.01 * np.outer(np.cos(x), np.cos(x))).astype(np.float32)
    big /= big[N // 2, N // 2]
    assert aw.aw_psf_sidelobe(ctx, _cuda(big)) == ocl.psf_sidelobe(big)


def _residual_case(N, npol, seed):
    """PSF-shifted sources plus noise in every Stokes plane, from the generators
    and the oracle's PSF shape (no GPU output)."""
    rng = np.random.default_rng(seed)
    x = (np.arange(N) - N // 2) / 2.3
    s = np.sinc(x)
    psf = (np.outer(s, s) ** 2).astype(np.float32)
    R = np.zeros((npol, N, N))
    for _ in range(12):
        qy, qx = rng.integers(N // 4, 3 * N // 4, 2)
        amp = rng.uniform(0.2, 1.0) * np.array([1.0, 0.1, -0.05, 0.01][:npol])
        R += amp[:, None, None] * np.roll(np.roll(psf, qy - N // 2, 0), qx - N // 2, 1)[None]
    R += 0.002 * rng.normal(size=R.shape)
    return R.astype(np.float32), psf


@pytest.mark.parametrize("N,npol,h,gain,iters", [(64, 1, 12, 0.1, 300), (256, 4, 40, 0.2, 400),
                                                 (256, 4, 127, 0.5, 60), (200, 1, 20, 0.1, 500)])
def test_hogbom_bit_exact_against_the_fp32_oracle(ctx, N, npol, h, gain, iters):
    from paper_2206_15117_gb300 import aw
    R, psf = _residual_case(N, npol, seed=N + npol + h)
    win = ocl.default_window(N)
    Mo, Ro, no = ocl.hogbom(R, psf, gain, 1e-3, iters, h, win)
    r = _cuda(R)
    m = torch.zeros_like(r)
    n = aw.aw_hogbom(ctx, r, _cuda(psf), gain, 1e-3, iters, h, win, m)
    assert n == no
    assert np.array_equal(m.cpu().numpy(), Mo)
    assert np.array_equal(r.cpu().numpy(), Ro)


def test_hogbom_window_edges_and_threshold_stop(ctx):
    from paper_2206_15117_gb300 import aw
    N = 128
    R, psf = _residual_case(N, 1, seed=44)
    win = (3, 70, 125, 121)                      # a window touching the image edge region
    Mo, Ro, no = ocl.hogbom(R, psf, 0.3, 0.05, 10000, 60, win)
    assert 0 < no < 10000                         # stopped by the threshold
    r, m = _cuda(R), torch.zeros((1, N, N), dtype=torch.float32, device="cuda")
    n = aw.aw_hogbom(ctx, r, _cuda(psf), 0.3, 0.05, 10000, 60, win, m)
    assert n == no and np.array_equal(m.cpu().numpy(), Mo) and np.array_equal(r.cpu().numpy(), Ro)


def test_hogbom_rejects_bad_arguments(ctx):
    from paper_2206_15117_gb300 import aw
    N = 64
    r = torch.zeros((1, N, N), dtype=torch.float32, device="cuda")
    p = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    for args in [(0.0, 32, (16, 16, 48, 48)), (0.5, 32, (16, 16, 48, 48)), (0.5, 5, (40, 16, 20, 48)),
                 (0.5, 5, (16, 16, 48, 65))]:
        gain, h, win = args
        with pytest.raises(RuntimeError):
            aw.aw_hogbom(ctx, r, p, gain, 0.0, 10, h, win, r)


def _consistent_vis(s, stokes_model):
    """Observed visibilities = the oracle's prediction of a point-source model."""
    return oc.degrid(s.okd, s.co, oc.image_to_grid(stokes_model, s.kw["W"]))


def _run_both(ctx, s, vis, **cfg):
    from paper_2206_15117_gb300 import aw
    npol, N = s.kw["npol"], s.kw["N"]
    ref = ocl.clean(s.okg, s.okd, s.co, vis, None, s.kw["W"], **cfg)
    model = torch.empty((npol, N, N), dtype=torch.float32, device="cuda")
    resid = torch.empty_like(model)
    psf = torch.empty((N, N), dtype=torch.float32, device="cuda")
    rep = aw.aw_clean(ctx, s.plan, s.kg, s.kd, _cuda(vis.astype(np.complex64)), None, model, resid, psf, **cfg)
    return ref, rep, model.cpu().numpy(), resid.cpu().numpy(), psf.cpu().numpy()


def _inner(a):
    # images are compared on the inner half: the grid correction is small near the
    # edges and scales FP32 rounding there (as for aw_fft_to_image)
    N = a.shape[-1]
    return a[..., N // 4:3 * N // 4, N // 4:3 * N // 4]


def test_clean_stokes_i_matches_oracle(ctx, stokes_i):
    N = stokes_i.kw["N"]
    truth = np.zeros((1, N, N))
    for (y, x, a) in [(28, 30, 1.0), (36, 25, 0.6), (33, 38, -0.4)]:
        truth[0, y, x] = a
    vis = _consistent_vis(stokes_i, truth)
    cfg = dict(n_major=6, max_minor=400, gain=0.2, threshold=1e-3, cycle_factor=1.0, patch_half=16)
    ref, rep, model, resid, psf = _run_both(ctx, stokes_i, vis, **cfg)
    assert np.abs(_inner(psf) - _inner(ref["psf"])).max() < 1e-5
    assert rep.sidelobe == pytest.approx(ref["sidelobe"], rel=1e-5)
    assert rep.n_major == ref["n_major"] and rep.n_minor == sum(ref["minor"])
    assert rep.peak_first == pytest.approx(ref["peaks"][0], rel=1e-5)
    assert rep.peak_last == pytest.approx(ref["peaks"][-1], rel=1e-3, abs=1e-6)
    assert np.abs(model - ref["model"]).max() < 1e-4
    assert np.abs(_inner(resid) - _inner(ref["residual"])).max() < 1e-4 * ref["peaks"][0]


def test_clean_fullpol_matches_oracle(ctx, fullpol):
    N = fullpol.kw["N"]
    truth = np.zeros((4, N, N))
    for (y, x, st) in [(120, 131, (1.0, 0.05, -0.03, 0.005)), (140, 110, (0.5, -0.02, 0.04, 0.0)),
                       (100, 150, (0.3, 0.0, 0.0, 0.0))]:
        truth[:, y, x] = st
    vis = _consistent_vis(fullpol, truth)
    cfg = dict(n_major=4, max_minor=300, gain=0.25, threshold=2e-3, cycle_factor=1.5, patch_half=48)
    ref, rep, model, resid, psf = _run_both(ctx, fullpol, vis, **cfg)
    assert rep.n_major == ref["n_major"] and rep.n_minor == sum(ref["minor"])
    assert rep.peak_first == pytest.approx(ref["peaks"][0], rel=1e-5)
    assert np.abs(model - ref["model"]).max() < 1e-4 * np.abs(ref["model"]).max()
    assert np.abs(_inner(resid) - _inner(ref["residual"])).max() < 1e-4 * ref["peaks"][0]
    # and the loop did its job on the Stokes I point sources
    assert ref["peaks"][-1] < 0.1 * ref["peaks"][0]
