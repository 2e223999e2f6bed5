"""GPU: the learned kernel surrogate's own kernels (forward, backward, Adam
training, table evaluation with per-w-plane rejection) against the FP64 MLP
oracle and the exact kernels."""
import math

import numpy as np
import pytest
import torch

from oracle import core as oc
from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


@pytest.mark.parametrize("npol,width,omega0", [(4, 32, 30.0), (1, 16, 1.0)])
def test_forward_and_gradient_match_fp64_oracle(ctx, npol, width, omega0):
    from paper_2206_15117_gb300 import aw
    sur = aw.aw_surrogate_create(ctx, npol=npol, width=width, n_hidden=4, omega0=omega0, seed=3)
    p = aw.aw_surrogate_get_params(sur).astype(np.float64)
    sizes = omlp.layer_sizes(5, width, 4, npol * npol)
    assert p.size == omlp.n_params(sizes) == aw.aw_surrogate_nparams(sur)
    rng = np.random.default_rng(5)
    B = 300
    X = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    T = rng.standard_normal((B, 2 * npol * npol)).astype(np.float32)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    Y = torch.empty((B, 2 * npol * npol), dtype=torch.float32, device="cuda")
    aw.aw_surrogate_forward(ctx, sur, Xd, Y)
    g = torch.empty(p.size, dtype=torch.float32, device="cuda")
    loss = aw.aw_surrogate_loss_grad(ctx, sur, Xd, Td, g)
    Yr, cache = omlp.forward(p, sizes, X.astype(np.float64), omega0)
    gr = omlp.backward(p, sizes, cache, Yr, T.astype(np.float64), omega0)
    y = Y.cpu().numpy()
    assert np.abs(y - Yr).max() < 2e-4 * max(1.0, np.abs(Yr).max())
    assert loss == pytest.approx(omlp.loss(Yr, T.astype(np.float64)), rel=1e-4)
    gg = g.cpu().numpy()
    assert np.linalg.norm(gg - gr) < 1e-3 * np.linalg.norm(gr)
    # every layer separately (a transposed or dropped term shows here)
    off = 0
    for i in range(len(sizes) - 1):
        n = sizes[i + 1] * sizes[i] + sizes[i + 1]
        a, b = gg[off:off + n], gr[off:off + n]
        assert np.linalg.norm(a - b) < 2e-3 * np.linalg.norm(b) + 1e-7, i
        off += n


def _wproj_spec():
    N = 512
    return dict(N=N, dl=math.radians(2.0) / N, OS=8, W=7.0, npol=1, nw=4, w_max=2000.0,
                supports=[8, 8, 12, 16])


def _export_all(aw, ks, kw):
    out = []
    for b, S in enumerate(kw["supports"]):
        t = torch.empty(kw["OS"] ** 2 * S * S, dtype=torch.complex64, device="cuda")
        aw.aw_kernel_set_export(ks, b, t)
        out.append(t.cpu().numpy())
    return out


def test_training_learns_the_kernels_and_rejects_per_plane(ctx):
    from paper_2206_15117_gb300 import aw
    kw = _wproj_spec()
    exact = aw.aw_make_kernels(ctx, **kw)
    ex = _export_all(aw, exact, kw)
    kmax = max(np.abs(e).max() for e in ex)
    sur = aw.aw_surrogate_create(ctx, npol=1, width=64, n_hidden=4, omega0=30.0, D=1.0, norm_supports=kw["supports"], w_max=kw["w_max"],
                                 f_c=1.4e9, f_h=0.2e9, chi_c=0.0, chi_h=1.5, out_scale=float(kmax), seed=11)
    rep = aw.aw_surrogate_train(ctx, sur, exact, steps=600, batch=8192, lr=1e-3, lr_final=1e-5, seed=3)
    assert rep.steps == 600 and rep.loss_last < 0.05 * rep.loss_first, (rep.loss_first, rep.loss_last)
    # tables: per-bin error against the oracle's exact kernels
    learned, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=1e9)
    assert nrej == 0
    got = _export_all(aw, learned, kw)
    spec = oc.KernelSpec(**kw)
    for b in range(spec.nbins):
        ref = oc.synth_bin(spec, b).reshape(-1)
        rel = np.linalg.norm(got[b] - ref) / np.linalg.norm(ref)
        assert rel == pytest.approx(float(err[b]), rel=0.05, abs=1e-4)
        assert rel < 0.2
    # a threshold below the smallest error rejects every plane: exact tables back
    learned2, err2, nrej2 = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=0.0)
    assert nrej2 == spec.nbins
    for a, b in zip(_export_all(aw, learned2, kw), ex):
        np.testing.assert_array_equal(a, b)
    # what the network buys: its parameters against the tables it replaces
    nbytes_net = aw.aw_surrogate_nparams(sur) * 2          # FP16 weights
    assert nbytes_net < aw.aw_kernel_set_info(exact).bytes


def test_save_and_load_round_trip(ctx, tmp_path):
    # parameters, configuration, per-plane rejection and engine survive a file round trip bit-exactly
    from paper_2206_15117_gb300 import aw
    sur = aw.aw_surrogate_create(ctx, npol=4, width=32, n_hidden=4, omega0=30.0, seed=11, D=1.5,
                                 norm_supports=[16, 24, 32], w_max=500.0, f_c=1.3e9, f_h=0.1e9,
                                 chi_c=0.2, chi_h=1.1, out_scale=0.03)
    rng = np.random.default_rng(12)
    p = (rng.standard_normal(aw.aw_surrogate_nparams(sur)) * 0.1).astype(np.float32)
    aw.aw_surrogate_set_params(sur, p)
    aw.aw_surrogate_set_engine(sur, aw.AW_ENGINE_MMA_SYNC)
    path = str(tmp_path / "sur.bin")
    aw.aw_surrogate_save(sur, path)
    back = aw.aw_surrogate_load(ctx, path)
    np.testing.assert_array_equal(aw.aw_surrogate_get_params(back), p)
    X = torch.as_tensor(rng.uniform(-1, 1, (257, 5)).astype(np.float32), device="cuda")
    Y0 = torch.empty((257, 32), dtype=torch.float32, device="cuda")
    Y1 = torch.empty_like(Y0)
    aw.aw_surrogate_forward(ctx, sur, X, Y0)
    aw.aw_surrogate_forward(ctx, back, X, Y1)
    torch.cuda.synchronize()
    assert torch.equal(Y0, Y1)
    # a second save of the loaded surrogate gives the same bytes
    path2 = str(tmp_path / "sur2.bin")
    aw.aw_surrogate_save(back, path2)
    raw = open(path, "rb").read()
    assert raw == open(path2, "rb").read()
    assert raw[:8] == b"AWSURR01"
    # damaged files are refused
    bad = tmp_path / "bad.bin"
    for blob in (raw[:-9], raw + b"\0", b"XXXXXXXX" + raw[8:], raw[:100] + bytes([raw[100] ^ 1]) + raw[101:]):
        bad.write_bytes(blob)
        with pytest.raises(RuntimeError):
            aw.aw_surrogate_load(ctx, str(bad))
    with pytest.raises(RuntimeError):
        aw.aw_surrogate_load(ctx, str(tmp_path / "missing.bin"))
