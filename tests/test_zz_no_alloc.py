"""mosaic_gamma_noalloc: the allocation-free variant of mosaic_gamma.

Some callers cannot allocate device memory (code inside a framework whose
caching allocator owns the GPU, real-time loops that forbid allocation after
start-up).  This entry point serves them with a fixed scratch array inside the
library.  The test calls it through the C ABI and checks it
against the existing mosaic_gamma on two calls in a row with different
inputs, so that what the first call leaves in the shared scratch cannot leak
into the second.  It is collected last on purpose.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _beams(N, nfield, seed):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:N, 0:N]
    cen = [(N / 2, N / 2)] + [(N / 2 + 0.18 * N * math.cos(a), N / 2 + 0.18 * N * math.sin(a))
                              for a in np.arange(nfield - 1) * 2 * math.pi / max(nfield - 1, 1)]
    B = np.stack([np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * (0.12 * N) ** 2)) for cx, cy in cen])
    return (B * rng.uniform(0.5, 1.5, (nfield, 1, 1))).astype(np.float32)


def _call_noalloc(lib, beams, eps, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return lib.mosaic_gamma_noalloc(ctypes.c_void_p(beams.data_ptr()), beams.shape[0], beams.shape[-1],
                                    ctypes.c_float(eps), ctypes.c_void_p(out.data_ptr()), stream)


def test_noalloc_gamma_matches_mosaic_gamma_twice():
    from paper_2206_15117_gb300 import aw
    lib = aw.load()
    ctx = aw.aw_create(0)
    # first a large image with a high maximum, then a smaller one with a low
    # maximum: a stale maximum from the first call would spoil the second
    for N, nfield, seed, scale in ((1024, 7, 1, 40.0), (512, 3, 2, 0.25)):
        B = torch.as_tensor(_beams(N, nfield, seed) * np.float32(scale), device="cuda")
        ref = torch.empty((N, N), dtype=torch.float32, device="cuda")
        got = torch.full((N, N), float("nan"), dtype=torch.float32, device="cuda")
        aw.mosaic_gamma(ctx, B, 0.2, ref)
        assert _call_noalloc(lib, B, 0.2, got) == aw.AW_OK, lib.aw_last_error()
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.isfinite(g).all()
        np.testing.assert_allclose(g, r, rtol=1e-5, atol=0)
        assert (g > 0).sum() > 0.1 * N * N


def test_noalloc_gamma_rejects_images_above_its_scratch():
    from paper_2206_15117_gb300 import aw
    lib = aw.load()
    B = torch.zeros((1, 8, 8), dtype=torch.float32, device="cuda")
    out = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    # N = 8192 is rejected on the host before any GPU work (the pointers are
    # never dereferenced)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mosaic_gamma_noalloc(ctypes.c_void_p(B.data_ptr()), 1, 8192, ctypes.c_float(0.2),
                                  ctypes.c_void_p(out.data_ptr()), stream)
    assert rc == aw.AW_EINVAL
    assert b"4096" in lib.aw_last_error()
