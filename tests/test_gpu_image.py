"""GPU parity of aw_fft_to_image (cuFFT + the library's shift/grid-correction
kernels) and mosaic_gamma (Eq. 1) against the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import TOL_FP32, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


@pytest.mark.parametrize("npol,N", [(1, 512), (4, 256), (1, 2048)])
def test_fft_to_image(ctx, npol, N):
    from paper_2206_15117_gb300 import aw
    kw = dict(N=N, dl=math.radians(2.0) / N, OS=4, W=7.0, npol=npol, nw=1, supports=[8],
              pa=[0.0], fbin_freqs=[1.4e9])
    ks = aw.aw_make_kernels(ctx, **kw, role=aw.AW_ROLE_DEGRID)
    G = sy.random_grid(npol, N, seed=N + npol)
    wsum = 1234.5
    img = torch.empty((npol, N, N), dtype=torch.float32, device="cuda")
    aw.aw_fft_to_image(ctx, ks, torch.as_tensor(G, device="cuda"), wsum, img)
    ref = oc.fft_to_image(G.astype(np.complex128), 7.0, wsum)
    got = img.cpu().numpy()
    # the grid correction divides by psi(l) psi(m) (about 1e-4 at the edge),
    # which amplifies FP32 FFT rounding there: the inner half is compared at
    # the FP32 tolerance, the whole image with the correction taken back out
    q = slice(N // 4, 3 * N // 4)
    l2, mx = rel_err(got[:, q, q], ref[:, q, q])
    assert l2 < TOL_FP32 and mx < TOL_FP32, (l2, mx)
    c = oc.grid_correction_1d(7.0, N)
    corr = (c[:, None] * c[None, :])[None]
    l2, mx = rel_err(got * corr, ref * corr)
    assert l2 < TOL_FP32, l2
    assert np.all(got[:, 0, :] == 0) and np.all(got[:, :, 0] == 0)


def test_mosaic_gamma(ctx):
    from paper_2206_15117_gb300 import aw
    N = 512
    rng = np.random.default_rng(3)
    y, x = np.mgrid[0:N, 0:N]
    cen = [(N / 2, N / 2)] + [(N / 2 + 90 * math.cos(a), N / 2 + 90 * math.sin(a)) for a in np.arange(6) * math.pi / 3]
    B = np.stack([np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * 60.0 ** 2)) for cx, cy in cen]).astype(np.float32)
    B *= rng.uniform(0.9, 1.1, (7, 1, 1)).astype(np.float32)
    gam = torch.empty((N, N), dtype=torch.float32, device="cuda")
    aw.mosaic_gamma(ctx, torch.as_tensor(B, device="cuda"), 0.2, gam)
    ref = oc.mosaic_gamma(B.astype(np.float64), 0.2)
    got = gam.cpu().numpy()
    s = np.sqrt((B.astype(np.float64) ** 2).sum(0))
    pbp = s / s.max()
    far = np.abs(pbp - 0.2) > 1e-5          # away from the mask edge (FP32 vs FP64 decision)
    np.testing.assert_allclose(got[far], ref[far], rtol=1e-5, atol=0)
    assert np.all(got[pbp < 0.2 - 1e-5] == 0)
