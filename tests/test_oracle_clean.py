"""Pins of the cleaning-loop oracle (Cotton-Schwab major cycle, Hogbom minor
cycle): closed forms and constructed cases, no GPU."""
import math

import numpy as np
import pytest

from oracle import clean as ocl
from oracle import core as oc
from tests.oracle_cases import small_case


def _delta_psf(N):
    p = np.zeros((N, N), np.float32)
    p[N // 2, N // 2] = 1.0
    return p


def test_hogbom_delta_psf_decays_geometrically():
    # one pixel, delta PSF: every iteration multiplies the residual by (1 - g) exactly
    # up to rounding, in every Stokes plane; it stops at the first |I| below the threshold
    N, g, a, t = 32, 0.25, 0.8, 0.01
    R = np.zeros((4, N, N), np.float32)
    R[:, 13, 17] = [a, 0.3, -0.2, 0.05]
    M, Rn, n = ocl.hogbom(R, _delta_psf(N), g, t, 1000, 4, ocl.default_window(N))
    n_expect = math.ceil(math.log(t / a) / math.log(1 - g))
    assert n == n_expect
    decay = (1 - g) ** n
    np.testing.assert_allclose(Rn[:, 13, 17], R[:, 13, 17] * decay, rtol=1e-5)
    np.testing.assert_allclose(M[:, 13, 17], R[:, 13, 17] * (1 - decay), rtol=1e-5)
    Rn[:, 13, 17] = 0
    M[:, 13, 17] = 0
    assert not Rn.any() and not M.any()


def _triangle_psf(N, half):
    x = np.arange(N) - N // 2
    t = np.clip(1.0 - np.abs(x) / half, 0.0, None)
    return np.outer(t, t).astype(np.float32)


def test_hogbom_gain_one_recovers_separated_components_exactly():
    N = 64
    psf = _triangle_psf(N, 4)                         # support |x| < 4, peak 1
    comps = [(20, 22, 0.9), (40, 30, -0.7), (25, 44, 0.5), (44, 44, 0.3)]
    R = np.zeros((1, N, N), np.float64)
    for (y, x, a) in comps:
        R[0, y - 3:y + 4, x - 3:x + 4] += a * psf[N // 2 - 3:N // 2 + 4, N // 2 - 3:N // 2 + 4]
    M, Rn, n = ocl.hogbom(R.astype(np.float32), psf, 1.0, 1e-4, 100, 5, (8, 8, 56, 56))
    assert n == len(comps)
    for (y, x, a) in comps:
        assert M[0, y, x] == np.float32(a)
    assert np.abs(M).sum() == pytest.approx(sum(abs(a) for (_, _, a) in comps), rel=1e-6)
    assert np.abs(Rn).max() < 1e-6


def test_hogbom_patch_truncation_leaves_the_psf_tail():
    # the minor cycle subtracts only the (2h+1)^2 patch: outside it the PSF tail stays
    N, h = 64, 2
    psf = _triangle_psf(N, 6)
    R = np.zeros((1, N, N), np.float32)
    R[0] = np.roll(np.roll(psf, 30 - N // 2, 0), 31 - N // 2, 1)   # unit source at (30, 31)
    M, Rn, n = ocl.hogbom(R, psf, 1.0, 0.5, 1, h, (8, 8, 56, 56))
    assert n == 1 and M[0, 30, 31] == 1.0
    inside = Rn[0, 30 - h:30 + h + 1, 31 - h:31 + h + 1]
    assert np.abs(inside).max() < 1e-7
    tail = Rn[0].copy()
    tail[30 - h:30 + h + 1, 31 - h:31 + h + 1] = 0
    expect = R[0].copy()
    expect[30 - h:30 + h + 1, 31 - h:31 + h + 1] = 0
    assert np.array_equal(tail, expect)


def test_hogbom_ties_go_to_the_lowest_flat_index():
    N = 32
    R = np.zeros((1, N, N), np.float32)
    R[0, 20, 10] = 1.0
    R[0, 12, 21] = -1.0          # same |I|, lower row -> lower flat index
    M, Rn, n = ocl.hogbom(R, _delta_psf(N), 0.5, 0.9, 1, 2, ocl.default_window(N))
    assert n == 1 and M[0, 12, 21] == -0.5 and M[0, 20, 10] == 0.0


def test_psf_sidelobe_of_a_hand_built_psf():
    N = 32
    c = N // 2
    psf = np.zeros((N, N), np.float32)
    psf[c, c] = 1.0
    psf[c, c + 1] = 0.6
    psf[c, c + 2] = 0.2
    psf[c, c + 3] = -0.5        # first non-positive value along +l: main-lobe radius 3
    psf[c + 3, c] = -0.45       # radius 3: inside the main lobe (not > 3)
    psf[c - 4, c + 2] = 0.25    # radius sqrt(20) > 3
    psf[c + 5, c - 5] = -0.3    # the largest |psf| outside the main lobe within N/4
    psf[c + 8, c] = 0.9         # |dy| = N/4: beyond the sidelobe region
    psf[c - 2, c - 9] = -0.8    # |dx| > N/4
    assert ocl.psf_sidelobe(psf) == np.float32(0.3)


def _stokes_i_case():
    ob, base = small_case(npol=1, nw=1, S=10, W=7.0, OS=8, N=64, fov_deg=4.0, n_t=24)
    spec_g = oc.KernelSpec(**base, role=oc.ROLE_GRID)
    spec_d = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    co = oc.coords(spec_g, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin)
    return ob, spec_g, spec_d, co


def test_clean_recovers_point_sources_of_a_consistent_observation():
    # observed visibilities = the method's own prediction of three point sources on
    # pixel centres; Cotton-Schwab cleaning must converge to them
    ob, spec_g, spec_d, co = _stokes_i_case()
    assert co.valid.all()
    N = spec_g.N
    truth = np.zeros((1, N, N))
    srcs = [(28, 30, 1.0), (36, 25, 0.6), (33, 38, -0.4)]
    for (y, x, a) in srcs:
        truth[0, y, x] = a
    ksg, ksd = oc.make_kernels(spec_g), oc.make_kernels(spec_d)
    vis = oc.degrid(ksd, co, oc.image_to_grid(truth, spec_g.W))
    out = ocl.clean(ksg, ksd, co, vis, None, spec_g.W, n_major=6, max_minor=400, gain=0.2,
                    threshold=1e-3, cycle_factor=1.0, patch_half=16)
    assert out["n_major"] >= 2
    peaks = out["peaks"]
    assert peaks[-1] < 0.05 * peaks[0]
    for (y, x, a) in srcs:
        assert out["model"][0, y, x] == pytest.approx(a, abs=0.005)     # on the source pixel
    assert np.abs(out["model"]).sum() == pytest.approx(2.0, abs=0.01)  # and nowhere else
    # the PSF is peak-normalised and its main lobe is excluded from the sidelobe level
    assert out["psf"][N // 2, N // 2] == 1.0
    assert 0.0 < out["sidelobe"] < 1.0


def test_clean_residual_visibilities_are_observed_minus_predicted():
    ob, spec_g, spec_d, co = _stokes_i_case()
    N = spec_g.N
    rng = np.random.default_rng(3)
    vis = rng.normal(size=(co.x0.shape[0], 1)) + 1j * rng.normal(size=(co.x0.shape[0], 1))
    ksg, ksd = oc.make_kernels(spec_g), oc.make_kernels(spec_d)
    out = ocl.clean(ksg, ksd, co, vis, None, spec_g.W, n_major=1, max_minor=5, gain=0.5,
                    threshold=0.0, cycle_factor=0.0, patch_half=8)
    pred = oc.degrid(ksd, co, oc.image_to_grid(out["model"].astype(np.float64), spec_g.W))
    np.testing.assert_allclose(out["residual_vis"], vis - pred, rtol=0, atol=1e-12)
    assert out["minor"] == [5] and np.count_nonzero(out["model"]) <= 5
