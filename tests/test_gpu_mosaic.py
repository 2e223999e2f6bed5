"""GPU parity of the image-domain mosaic calls through the C ABI: aw_reproject
(bilinear, Keys cubic) and aw_mosaic_combine against the FP64 oracle on the
same seeded images."""
import math

import numpy as np
import pytest
import torch

from oracle import core as oc
from oracle import mosaic as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _image(N, nplane, seed):
    rng = np.random.default_rng(seed)
    qy, qx = np.mgrid[0:N, 0:N]
    img = np.zeros((nplane, N, N))
    for _ in range(15):
        x, y = rng.uniform(0, N, 2)
        w = rng.uniform(1.0, 6.0)
        img += rng.normal(size=(nplane, 1, 1)) * np.exp(-((qx - x) ** 2 + (qy - y) ** 2) / (2 * w * w))[None]
    img += 0.01 * rng.normal(size=img.shape)
    return img.astype(np.float32)


def _compare(ctx, img, src, dst, interp, fill=0.0):
    from paper_2206_15117_gb300 import aw
    out = torch.empty((img.shape[0], dst.N, dst.N), dtype=torch.float32, device="cuda")
    aw.aw_reproject(ctx, _cuda(img), aw.sky_frame(src.ra0, src.dec0, src.dl, src.N, src.cx, src.cy), out,
                    aw.sky_frame(dst.ra0, dst.dec0, dst.dl, dst.N, dst.cx, dst.cy), interp, fill)
    got = out.cpu().numpy()
    ref = om.reproject(img.astype(np.float64), src, dst, interp, fill)
    # positions within rounding of a whole pixel may pick either stencil; their value is
    # continuous (compared), but at the image border the fill decision is not: skip those
    x, y, _ = om.source_positions(src, dst)
    amb = (np.abs(x - np.rint(x)) < 1e-6) | (np.abs(y - np.rint(y)) < 1e-6)
    filled_ref = ref == fill
    border = amb & ((np.abs(x - 1) < 1.5) | (np.abs(x - (src.N - 2)) < 1.5) | (np.abs(y - 1) < 1.5) |
                    (np.abs(y - (src.N - 2)) < 1.5))
    keep = ~border
    assert np.array_equal((got == fill)[:, keep], filled_ref[:, keep])
    scale = np.abs(img).max()
    assert np.abs(got - ref)[:, keep].max() < 1e-5 * scale
    return got, ref, keep


@pytest.mark.parametrize("interp", [0, 1])
def test_reproject_between_mosaic_fields_matches_oracle(ctx, interp):
    # two fields of a hexagonal mosaic, 1 deg apart, 3 deg images (scaled down to 256^2)
    N = 256
    dl = math.radians(3.0) / N
    dec0 = math.radians(-45.0)
    a = om.frame(1.1, dec0, dl, N)
    b = om.frame(1.1 + math.radians(1.0) / math.cos(dec0), dec0 + math.radians(0.2), dl, N)
    img = _image(N, 4, seed=3)
    got, ref, keep = _compare(ctx, img, a, b, interp)
    assert (ref != 0).sum() > 0.3 * ref.size            # a real overlap
    # and a larger destination frame (the mosaic) with a different pixel size
    m = om.frame(1.1 + 0.01, dec0 - 0.004, dl * 0.75, 400)
    _compare(ctx, img, a, m, interp, fill=-1.0)


@pytest.mark.parametrize("interp", [0, 1])
def test_reproject_pure_shift_and_identity(ctx, interp):
    N = 96
    src = om.frame(0.7, -0.5, 2e-4, N)
    img = _image(N, 2, seed=4)
    _compare(ctx, img, src, om.frame(0.7, -0.5, 2e-4, N, cx=N // 2 + 0.37, cy=N // 2 - 2.81), interp)
    got, ref, keep = _compare(ctx, img, src, src, interp)
    inner = (slice(None), slice(2, N - 2), slice(2, N - 2))
    assert np.abs(got[inner] - img[inner]).max() < 1e-5 * np.abs(img).max()


def test_mosaic_combine_matches_oracle(ctx):
    from paper_2206_15117_gb300 import aw
    N, nf = 128, 7
    rng = np.random.default_rng(5)
    imgs = rng.normal(size=(nf, 4, N, N)).astype(np.float32)
    beams = rng.uniform(0, 1, size=(nf, N, N)).astype(np.float32)
    gam = oc.mosaic_gamma(beams.astype(np.float64), 0.1).astype(np.float32)
    out = torch.empty((4, N, N), dtype=torch.float32, device="cuda")
    aw.aw_mosaic_combine(ctx, _cuda(imgs), _cuda(beams), _cuda(gam), out)
    ref = om.combine(imgs, beams, gam)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5 * np.abs(ref).max()


def test_reproject_rejects_bad_frames(ctx):
    from paper_2206_15117_gb300 import aw
    x = torch.zeros((1, 16, 16), dtype=torch.float32, device="cuda")
    good = aw.sky_frame(0.0, 0.0, 1e-3, 16)
    for bad in (aw.sky_frame(0.0, 0.0, 0.0, 16), aw.sky_frame(0.0, float("nan"), 1e-3, 16),
                aw.sky_frame(0.0, 0.0, 1e-3, 2)):
        with pytest.raises(RuntimeError):
            aw.aw_reproject(ctx, x, bad, x, good)
    with pytest.raises(RuntimeError):
        aw.aw_reproject(ctx, x, good, x, good, interp=5)
