"""Pins for the oracle's kernel synthesis (Sec. 3.2: kernels are the FFT of the
Mueller cells after the anti-aliasing function and the w term)."""
import math

import numpy as np
import pytest

from oracle import core as oc


def _spec(**kw):
    base = dict(N=256, dl=math.radians(2.0) / 256, OS=8, W=7.0, npol=1, nw=1, supports=[8])
    base.update(kw)
    return oc.KernelSpec(**base)


def test_taper_kernel_is_real_and_symmetric():
    K = oc.synth_bin(_spec(), 0)[..., 0]            # [oy][ox][jy][jx]
    assert np.abs(K.imag).max() < 1e-15
    # fine offset 0: taps at -3..4 cells; kernel symmetric in d -> K[j] = K[6 - j]
    k0 = K[0, 0, 3, :].real
    np.testing.assert_allclose(k0[:7], k0[:7][::-1], atol=1e-16)
    # separable: psi(l) psi(m) -> outer product
    np.testing.assert_allclose(K[3, 5].real, np.outer(K[3, 0, :, 3].real, K[0, 5, 3, :].real) / K[0, 0, 3, 3].real,
                               rtol=1e-10, atol=1e-16)


def test_zero_offset_taper_kernel_sums_to_one():
    # closed form: the full-period zero-offset taper kernel sums to
    # M^2 psi(0)^2 / M^2 = 1 (Poisson summation of the M-point DFT); a wide
    # support keeps all but the far tails, which shrink as M grows
    for S, tol in ((16, 2e-6), (32, 1e-6), (64, 2e-7)):
        spec = _spec(supports=[S])
        K = oc.synth_bin(spec, 0, offsets_y=[0], offsets_x=[0])[0, 0, :, :, 0]
        assert abs(K.sum() - 1.0) < tol


def test_kernel_follows_pswf_self_reciprocity():
    # the finite Fourier transform of psi_0 is psi_0 itself: the uv kernel at
    # distance d cells is psi_0(2 d / W) up to a constant, for |d| < W/2
    spec = _spec(supports=[64], OS=16)                 # M = 128 image samples
    K = oc.synth_bin(spec, 0)[..., 0].real             # [oy][ox][jy][jx]
    # 1-D profile along x at fy = 0, jy = 31 (d_y = 0): d = (jx - 31) - fx/16
    vals, ds = [], []
    for fx in range(16):
        for jx in range(64):
            vals.append(K[0, fx, 31, jx])
            ds.append((jx - 31) - fx / 16)
    vals, ds = np.array(vals), np.array(ds)
    keep = np.abs(ds) < 2.0
    ref = oc.pswf0(math.pi * 7.0 / 2, 2 * ds[keep] / 7.0)
    ratio = vals[keep] / ref
    # the residual is the Riemann-sum error of the M-sample image (shrinks with M)
    assert np.max(np.abs(ratio / ratio.mean() - 1)) < 1e-4


def test_w_kernel_conjugate_symmetry_and_degrid_role():
    s_pos = _spec(nw=4, w_max=4000.0, supports=[16] * 4)
    s_neg = _spec(nw=4, w_max=-4000.0, supports=[16] * 4)
    Kp = oc.synth_bin(s_pos, 3)
    Kn = oc.synth_bin(s_neg, 3)
    # f(-w) = conj f(w) and f symmetric in l -> K(-w) = conj K(w)
    np.testing.assert_allclose(Kn, np.conj(Kp), atol=1e-14)
    # Stokes I without A term: degrid kernel = conj(grid kernel) = adjoint
    s_deg = _spec(nw=4, w_max=4000.0, supports=[16] * 4, role=oc.ROLE_DEGRID)
    np.testing.assert_allclose(oc.synth_bin(s_deg, 3), np.conj(Kp), atol=1e-14)
    # the w term makes the kernel complex and not separable
    assert np.abs(Kp.imag).max() > 1e-4


def test_fullpol_identity_beam_limit():
    # a beam far wider than the field, no leakage, chi = 0: M^S ~ I, so the
    # grid kernels are the taper kernel times (I / (1 + beta)) T with
    # beta = (eps / 2)^2 (Eq. 6 on a unit diagonal)
    eps = 0.2
    spec = _spec(npol=4, dish_d=1e-4, d_xy=0.0, d_yx=0.0, pa=(0.0,), fbin_freqs=(1.4e9,), eps=eps)
    K = oc.synth_bin(spec, 0)                          # [.., 16]
    Kt = oc.synth_bin(_spec(), 0)[..., 0]
    T = oc.T_CORR_TO_STOKES
    beta = (eps / 2) ** 2
    for s in range(4):
        for c in range(4):
            np.testing.assert_allclose(K[..., s * 4 + c], Kt * T[s, c] / (1 + beta), atol=1e-12)
    spec_d = _spec(npol=4, dish_d=1e-4, d_xy=0.0, d_yx=0.0, pa=(0.0,), fbin_freqs=(1.4e9,),
                   role=oc.ROLE_DEGRID)
    Kd = oc.synth_bin(spec_d, 0)
    Ti = oc.T_STOKES_TO_CORR
    for c in range(4):
        for s in range(4):
            np.testing.assert_allclose(Kd[..., c * 4 + s], Kt * Ti[c, s], atol=1e-12)


def test_adjoint_role_is_conjugate_transpose_of_grid_role():
    kw = dict(npol=4, nw=2, w_max=3000.0, supports=[12, 12], dish_d=12.0, d_xy=0.01j, d_yx=0.02,
              pa=(0.5,), fbin_freqs=(1.3e9,))
    Kg = oc.synth_bin(_spec(**kw), 1)
    Ka = oc.synth_bin(_spec(**kw, role=oc.ROLE_ADJOINT), 1)
    for s in range(4):
        for c in range(4):
            np.testing.assert_allclose(Ka[..., c * 4 + s], np.conj(Kg[..., s * 4 + c]), atol=1e-13)


def test_make_kernels_layout():
    spec = _spec(nw=3, w_max=2000.0, supports=[8, 10, 12])
    ks = oc.make_kernels(spec)
    assert list(ks.bin_support) == [8, 10, 12]
    sizes = [8 * 8 * S * S for S in (8, 10, 12)]
    assert list(ks.offsets) == [0, sizes[0], sizes[0] + sizes[1]]
    np.testing.assert_array_equal(ks.table[ks.offsets[1]:ks.offsets[2]],
                                  oc.synth_bin(spec, 1).reshape(-1))
