"""Pins of the image-domain mosaic oracle: projection against an independent
vector formulation, interpolation exactness on polynomials, identity and
round trips, and the Eq. 1 combination of co-located fields."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import mosaic as om


def _basis(ra0, dec0):
    # orthonormal (l, m, n) axes of the tangent frame at (ra0, dec0): east, north, centre
    e_l = np.array([-math.sin(ra0), math.cos(ra0), 0.0])
    e_m = np.array([-math.sin(dec0) * math.cos(ra0), -math.sin(dec0) * math.sin(ra0), math.cos(dec0)])
    e_n = np.array([math.cos(dec0) * math.cos(ra0), math.cos(dec0) * math.sin(ra0), math.sin(dec0)])
    return e_l, e_m, e_n


def _unit(ra, dec):
    return np.stack([np.cos(dec) * np.cos(ra), np.cos(dec) * np.sin(ra), np.sin(dec)], -1)


def test_projection_matches_the_vector_formulation():
    rng = np.random.default_rng(0)
    fr = om.frame(1.3, -0.8, 1e-4, 64)
    ra = 1.3 + rng.uniform(-0.05, 0.05, 50)
    dec = -0.8 + rng.uniform(-0.05, 0.05, 50)
    l, m, n = om.radec_to_lmn(fr, ra, dec)
    s = _unit(ra, dec)
    e_l, e_m, e_n = _basis(1.3, -0.8)
    np.testing.assert_allclose(l, s @ e_l, atol=1e-15)
    np.testing.assert_allclose(m, s @ e_m, atol=1e-15)
    np.testing.assert_allclose(n, s @ e_n, atol=1e-15)
    ra2, dec2, ok = om.lm_to_radec(fr, l, m)
    assert ok.all()
    np.testing.assert_allclose(np.angle(np.exp(1j * (ra2 - ra))), 0, atol=1e-13)
    np.testing.assert_allclose(dec2, dec, atol=1e-13)


def test_keys_weights_partition_of_unity_and_interpolate_samples():
    t = np.linspace(0, 0.999, 37)
    w = om.keys_weights(t)
    np.testing.assert_allclose(w.sum(-1), 1.0, atol=1e-14)
    np.testing.assert_allclose(om.keys_weights(np.array([0.0]))[0], [0, 1, 0, 0], atol=1e-15)


def _shifted_frames(dx, dy, N=48):
    src = om.frame(0.7, -0.5, 2e-4, N)
    dst = om.frame(0.7, -0.5, 2e-4, N, cx=N // 2 + dx, cy=N // 2 + dy)
    return src, dst


def test_bilinear_is_exact_on_linear_images_and_cubic_on_quadratics():
    N, dx, dy = 48, 0.37, -0.81
    src, dst = _shifted_frames(dx, dy, N)
    qy, qx = np.mgrid[0:N, 0:N].astype(np.float64)
    lin = 0.3 + 0.02 * qx - 0.05 * qy
    quad = 1.0 + 0.01 * qx - 0.02 * qy + 0.003 * qx * qx - 0.001 * qx * qy + 0.002 * qy * qy
    # the destination pixel q sees the source at q - (dx, dy)
    xs, ys = qx - dx, qy - dy
    out = om.reproject(lin[None], src, dst, om.INTERP_BILINEAR)[0]
    inner = (slice(3, N - 3), slice(3, N - 3))
    np.testing.assert_allclose(out[inner], (0.3 + 0.02 * xs - 0.05 * ys)[inner], atol=1e-11)
    out = om.reproject(quad[None], src, dst, om.INTERP_CUBIC)[0]
    ref = 1.0 + 0.01 * xs - 0.02 * ys + 0.003 * xs * xs - 0.001 * xs * ys + 0.002 * ys * ys
    np.testing.assert_allclose(out[inner], ref[inner], atol=1e-10)


def test_identity_reprojection_returns_the_image():
    N = 40
    fr = om.frame(2.0, 0.3, 3e-4, N)
    img = np.random.default_rng(1).normal(size=(2, N, N))
    for interp in (om.INTERP_BILINEAR, om.INTERP_CUBIC):
        out = om.reproject(img, fr, fr, interp)
        np.testing.assert_allclose(out[:, 2:-2, 2:-2], img[:, 2:-2, 2:-2], atol=1e-9)


def test_stencils_leaving_the_source_are_filled():
    N = 32
    src, dst = _shifted_frames(5.5, 0.0, N)       # the source moves 5.5 pixels left
    out = om.reproject(np.ones((1, N, N)), src, dst, om.INTERP_CUBIC, fill=-7.0)
    assert (out[0, :, :7] == -7.0).all()                           # x stencil leaves on the left
    # rows 0 and N-1 always need a pixel outside; rows 1 and N-2 sit on whole-pixel positions, where the
    # floor of the position (and with it the stencil) may fall either way by rounding: not asserted
    assert (out[0, 0, :] == -7.0).all() and (out[0, -1, :] == -7.0).all()
    np.testing.assert_allclose(out[0, 2:N - 2, 8:], 1.0, atol=1e-14)


def _blob(N, x, y, w=1.5):
    qy, qx = np.mgrid[0:N, 0:N]
    return np.exp(-((qx - x) ** 2 + (qy - y) ** 2) / (2 * w * w))


def test_a_source_lands_where_the_vector_formulation_puts_it():
    N, dl = 128, 2.5e-4
    a = om.frame(0.4, -0.6, dl, N)
    b = om.frame(0.4 + 0.006, -0.6 - 0.004, dl, N)
    ra, dec = 0.4 + 0.003, -0.6 - 0.001
    s = _unit(ra, dec)
    pos = {}
    for name, fr in (("a", a), ("b", b)):
        e_l, e_m, _ = _basis(fr.ra0, fr.dec0)
        pos[name] = (s @ e_l / dl + fr.cx, s @ e_m / dl + fr.cy)
    img = _blob(N, *pos["a"])[None]
    out = om.reproject(img, a, b, om.INTERP_CUBIC)[0]
    qy, qx = np.mgrid[0:N, 0:N]
    wsum = out.sum()
    cx, cy = (out * qx).sum() / wsum, (out * qy).sum() / wsum
    assert abs(cx - pos["b"][0]) < 0.01 and abs(cy - pos["b"][1]) < 0.01
    assert wsum == pytest.approx(img.sum(), rel=1e-3)


def test_round_trip_of_a_smooth_image():
    N = 96
    a = om.frame(1.0, 0.2, 3e-4, N)
    b = om.frame(1.0 - 0.004, 0.2 + 0.002, 3e-4, N)
    img = sum(_blob(N, x, y, 3.0) * amp for (x, y, amp) in [(40, 50, 1.0), (55, 45, -0.5), (48, 60, 0.3)])
    back = om.reproject(om.reproject(img[None], a, b, om.INTERP_CUBIC), b, a, om.INTERP_CUBIC)[0]
    inner = (slice(30, 66), slice(30, 66))
    assert np.abs(back - img)[inner].max() < 0.01 * np.abs(img).max()


def test_combination_of_identical_co_located_fields():
    # Eq. 1 with N identical fields: gamma * N * B * I = I * |B| / max|B| / B = I / max B (B > 0)
    N, nf = 32, 3
    qy, qx = np.mgrid[0:N, 0:N]
    B = np.exp(-((qx - 16) ** 2 + (qy - 16) ** 2) / 200.0)
    I = np.random.default_rng(2).normal(size=(4, N, N))
    gam = oc.mosaic_gamma(np.stack([B] * nf), 0.05)
    out = om.combine(np.stack([I] * nf), np.stack([B] * nf), gam)
    mask = gam > 0
    np.testing.assert_allclose(out[:, mask], I[:, mask] / B.max(), rtol=1e-12)
    assert (out[:, ~mask] == 0).all()
