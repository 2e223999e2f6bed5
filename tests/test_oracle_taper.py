"""Pins for the oracle's prolate-spheroidal anti-aliasing taper (Sec. 3.2:
kernels are multiplied in the image domain by an anti-aliasing function)."""
import math

import numpy as np
import pytest
import scipy.special

from oracle import core as oc


@pytest.mark.parametrize("W", [5.0, 7.0, 9.0])
def test_pswf_matches_library_routine(W):
    c = math.pi * W / 2
    x = np.linspace(-0.99, 0.99, 41)
    ours = oc.pswf0(c, x)
    ref = scipy.special.pro_ang1(0, 0, c, x)[0] / scipy.special.pro_ang1(0, 0, c, 0.0)[0]
    np.testing.assert_allclose(ours, ref, rtol=1e-9, atol=1e-12)


def test_pswf_is_eigenfunction_of_finite_fourier_transform():
    # int_{-1}^{1} exp(i c x t) psi(t) dt = mu psi(x) for every x
    c = math.pi * 7.0 / 2
    t, wq = np.polynomial.legendre.leggauss(200)
    psi_t = oc.pswf0(c, t)
    x = np.linspace(-0.95, 0.95, 23)
    lhs = np.array([np.sum(wq * np.exp(1j * c * xx * t) * psi_t) for xx in x])
    ratio = lhs / oc.pswf0(c, x)
    assert np.max(np.abs(ratio - ratio[len(x) // 2])) < 1e-9 * abs(ratio[len(x) // 2])


def test_taper_sampling_symmetric_and_edge_zeroed():
    t = oc.taper_samples(7.0, 64)
    assert t[0] == 0.0
    assert t[32] == pytest.approx(1.0)
    np.testing.assert_allclose(t[1:32], t[33:][::-1], rtol=0, atol=1e-15)


def test_grid_correction_is_taper_on_image_pixels():
    N = 128
    c = oc.grid_correction_1d(7.0, N)
    assert c[0] == 0.0 and c[N // 2] == pytest.approx(1.0)
    x = (np.arange(1, N) - N // 2) * 2.0 / N
    np.testing.assert_allclose(c[1:], oc.taper_1d(7.0, x), rtol=1e-14)
