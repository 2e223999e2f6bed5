"""GPU: kernel sets written to disk and read back (aw_kernel_set_save/load)
keep their tables bit for bit (FP32 and FP16 storage, per-baseline classes),
grid identically, refuse damaged files, and serve the on-disk cache keyed by
the spec hash (aw.cached_kernels)."""
import os

import numpy as np
import pytest
import torch

from paper_2206_15117_gb300 import synthetic as sy
from tests.gpu_cases import case_fullpol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


@pytest.mark.parametrize("storage,classes", [(0, False), (2, False), (0, True)])
def test_save_load_round_trip(ctx, tmp_path, storage, classes):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=8, nw=2, npa=1, nfb=2, supports=(16, 20))
    if classes:
        kw = {**kw, "type_leak": [(0.01, 0.02j), (-0.015, 0.01)]}
    ks = aw.aw_make_kernels(ctx, **kw, storage=storage)
    path = str(tmp_path / "k.bin")
    aw.aw_kernel_set_save(ks, path)
    back = aw.aw_kernel_set_load(ctx, path)
    i0, i1 = aw.aw_kernel_set_info(ks), aw.aw_kernel_set_info(back)
    assert (i0.nbins, i0.bytes, i0.storage, i0.max_support) == (i1.nbins, i1.bytes, i1.storage, i1.max_support)
    for b in (0, i0.nbins // 2, i0.nbins - 1):
        outs = []
        for k in (ks, back):
            S = [16, 20][(b // 2) % 2]
            buf = torch.empty(kw["OS"] ** 2 * S * S * 16, dtype=torch.complex64, device="cuda")
            aw.aw_kernel_set_export(k, b, buf)
            outs.append(buf.cpu().numpy())
        np.testing.assert_array_equal(outs[0], outs[1])
    # the same grid from both sets on one plan
    vd, keep = aw.device_observation(ob)
    plan = aw.aw_plan_create(ctx, vd, ks, tune=aw.aw_tune(32, 256, 2, 1024, 1))
    vis = torch.as_tensor(sy.random_vis(ob.nvis, 4, seed=3), device="cuda")
    grids = []
    for k in (ks, back):
        g = torch.zeros((4, kw["N"], kw["N"]), dtype=torch.complex64, device="cuda")
        aw.aw_grid(ctx, plan, k, vis, None, g)
        grids.append(g.cpu().numpy())
    assert np.abs(grids[0] - grids[1]).max() <= 1e-6 * np.abs(grids[0]).max()
    # damaged files are refused
    raw = open(path, "rb").read()
    bad = tmp_path / "bad.bin"
    for blob in (raw[:-1], raw + b"x", raw[:40] + bytes([raw[40] ^ 4]) + raw[41:],
                 raw[:-100] + bytes([raw[-100] ^ 1]) + raw[-99:], b"AWKSET02" + raw[8:]):
        bad.write_bytes(blob)
        with pytest.raises(aw.AWError):
            aw.aw_kernel_set_load(ctx, str(bad))


def test_cached_kernels(ctx, tmp_path):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_fullpol(n_t=4, nw=2, npa=1, nfb=1, supports=(16, 20))
    d = str(tmp_path / "cache")
    k1 = aw.cached_kernels(ctx, d, **kw)
    files = os.listdir(d)
    assert files == ["awkset-%016x.bin" % aw.aw_kernel_spec_hash(**kw)]
    k2 = aw.cached_kernels(ctx, d, **kw)          # served from the file
    assert aw.aw_kernel_set_info(k2).bytes == aw.aw_kernel_set_info(k1).bytes
    aw.cached_kernels(ctx, d, **{**kw, "eps": 0.3})
    assert len(os.listdir(d)) == 2
