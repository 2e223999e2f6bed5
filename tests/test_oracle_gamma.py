"""Pins for the oracle's mosaic weighting gamma(l, m) (Sec. 2.2, Eq. 1)."""
import numpy as np
import pytest

from oracle import core as oc


def _beam(N, x0, y0, width):
    y, x = np.mgrid[0:N, 0:N]
    return np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2 * width ** 2))


def test_single_field_closed_form():
    B = _beam(64, 32, 32, 10.0)
    eps = 0.2
    g = oc.mosaic_gamma(B[None], eps)
    keep = B / B.max() >= eps
    np.testing.assert_allclose(g[keep], 1.0 / (B[keep] * B.max()), rtol=1e-12)
    assert np.all(g[~keep] == 0)


def test_colocated_identical_fields_closed_form():
    B = _beam(64, 30, 34, 8.0)
    n = 5
    g = oc.mosaic_gamma(np.stack([B] * n), 0.1)
    keep = B / B.max() >= 0.1
    np.testing.assert_allclose(g[keep], 1.0 / (n * B[keep] * B.max()), rtol=1e-12)


def test_hexagonal_mosaic_properties():
    N = 96
    cen = [(48, 48)] + [(48 + 20 * np.cos(a), 48 + 20 * np.sin(a)) for a in np.arange(6) * np.pi / 3]
    B = np.stack([_beam(N, x, y, 12.0) for x, y in cen])
    g = oc.mosaic_gamma(B, 0.2)
    s = np.sqrt((B ** 2).sum(0))
    keep = s / s.max() >= 0.2
    # gamma * sum B^2 = the normalised pattern (pbp) where unmasked
    np.testing.assert_allclose(g[keep] * (B ** 2).sum(0)[keep], s[keep] / s.max(), rtol=1e-12)
    assert g[~keep].max() == 0
