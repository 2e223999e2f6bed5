"""Oracle of the image-domain mosaic round trip (Sec. 2.2): image-plane
reprojection between phase centres, the Eq. 1 combination, plainly, in FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring): no product code imports
this module.

Sec. 2.2 makes an image of each mosaic field at its own phase centre,
reprojects the images to a common phase position to form the mosaic, and
reprojects the model back to each field before degridding.  The paper does not
write the projection or the interpolation out; the readings:

* Frames are orthographic (SIN) projections about a phase centre (ra0, dec0):
  a sky direction (ra, dec) has direction cosines
      l = cos dec sin(ra - ra0)
      m = sin dec cos dec0 - cos dec sin dec0 cos(ra - ra0)
      n = sin dec sin dec0 + cos dec cos dec0 cos(ra - ra0)
  and pixel (qx, qy) of a frame sits at l = (qx - cx) dl, m = (qy - cy) dl
  (cx = cy = N/2 for the imaging frames of this repository).
* An output pixel is mapped to its sky direction (inverse projection, FP64),
  then into the source frame; the value there is interpolated: bilinear (2 x 2
  pixels) or Keys cubic convolution with a = -1/2 (4 x 4 pixels).  Where the
  stencil leaves the source image, or the direction is not on the visible
  hemisphere of either frame (n <= 0, or l^2 + m^2 > 1), the output is `fill`.
* Combination (Eq. 1): mosaic = gamma * sum_f B_f * I_f over the fields, with
  every image already in the common frame; gamma is mosaic_gamma's.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

INTERP_BILINEAR = 0
INTERP_CUBIC = 1


@dataclass(frozen=True)
class Frame:
    ra0: float
    dec0: float
    dl: float
    N: int
    cx: float
    cy: float


def frame(ra0, dec0, dl, N, cx=None, cy=None) -> Frame:
    return Frame(float(ra0), float(dec0), float(dl), int(N), float(N // 2 if cx is None else cx),
                 float(N // 2 if cy is None else cy))


def lm_to_radec(fr: Frame, l, m):
    """Inverse SIN projection; returns (ra, dec, ok) with ok False off the sphere."""
    l = np.asarray(l, np.float64)
    m = np.asarray(m, np.float64)
    r2 = l * l + m * m
    ok = r2 <= 1.0
    n = np.sqrt(np.where(ok, 1.0 - r2, 0.0))
    sd0, cd0 = np.sin(fr.dec0), np.cos(fr.dec0)
    dec = np.arcsin(np.clip(m * cd0 + n * sd0, -1.0, 1.0))
    ra = fr.ra0 + np.arctan2(l, n * cd0 - m * sd0)
    return ra, dec, ok


def radec_to_lmn(fr: Frame, ra, dec):
    d = np.asarray(ra, np.float64) - fr.ra0
    sd, cd = np.sin(dec), np.cos(dec)
    sd0, cd0 = np.sin(fr.dec0), np.cos(fr.dec0)
    l = cd * np.sin(d)
    m = sd * cd0 - cd * sd0 * np.cos(d)
    n = sd * sd0 + cd * cd0 * np.cos(d)
    return l, m, n


def keys_weights(t: np.ndarray) -> np.ndarray:
    """Keys cubic convolution weights (a = -1/2) of the 4 samples at offsets
    -1, 0, 1, 2 from floor(x), for t = x - floor(x) in [0, 1)."""
    a = -0.5
    s = np.stack([1.0 + t, t, 1.0 - t, 2.0 - t], axis=-1)
    near = (a + 2) * s ** 3 - (a + 3) * s ** 2 + 1
    far = a * s ** 3 - 5 * a * s ** 2 + 8 * a * s - 4 * a
    return np.where(s <= 1.0, near, far)


def source_positions(src: Frame, dst: Frame):
    """Fractional source-frame pixel of every destination pixel, and validity."""
    qy, qx = np.mgrid[0:dst.N, 0:dst.N].astype(np.float64)
    ra, dec, ok = lm_to_radec(dst, (qx - dst.cx) * dst.dl, (qy - dst.cy) * dst.dl)
    l, m, n = radec_to_lmn(src, ra, dec)
    ok &= n > 0
    return l / src.dl + src.cx, m / src.dl + src.cy, ok


def reproject(image: np.ndarray, src: Frame, dst: Frame, interp: int = INTERP_BILINEAR, fill: float = 0.0):
    """image [nplane][src.N][src.N] -> [nplane][dst.N][dst.N] (FP64)."""
    img = np.asarray(image, np.float64)
    nplane = img.shape[0]
    x, y, ok = source_positions(src, dst)
    x0 = np.floor(x)
    y0 = np.floor(y)
    tx, ty = x - x0, y - y0
    if interp == INTERP_BILINEAR:
        offs = np.array([0, 1])
        wx = np.stack([1.0 - tx, tx], -1)
        wy = np.stack([1.0 - ty, ty], -1)
    else:
        offs = np.array([-1, 0, 1, 2])
        wx = keys_weights(tx)
        wy = keys_weights(ty)
    xi = x0[..., None].astype(np.int64) + offs
    yi = y0[..., None].astype(np.int64) + offs
    inside = ok & (xi.min(-1) >= 0) & (xi.max(-1) < src.N) & (yi.min(-1) >= 0) & (yi.max(-1) < src.N)
    xi = np.clip(xi, 0, src.N - 1)
    yi = np.clip(yi, 0, src.N - 1)
    out = np.zeros((nplane, dst.N, dst.N))
    for a in range(len(offs)):
        for b in range(len(offs)):
            w = wy[..., a] * wx[..., b]
            out += w[None] * img[:, yi[..., a], xi[..., b]]
    out[:, ~inside] = fill
    return out


def combine(images: np.ndarray, beams: np.ndarray, gamma: np.ndarray) -> np.ndarray:
    """Eq. 1: gamma * sum_f B_f * I_f.  images [nfield][nplane][N][N], beams
    [nfield][N][N], gamma [N][N]."""
    images = np.asarray(images, np.float64)
    beams = np.asarray(beams, np.float64)
    return np.asarray(gamma, np.float64)[None] * np.einsum("fyx,fpyx->pyx", beams, images)
