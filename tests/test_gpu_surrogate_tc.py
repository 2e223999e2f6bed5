"""GPU: training the learned kernel surrogate on the tensor cores (width 128:
every layer but the first as tcgen05.mma with FP16 operands and FP32
accumulation, weight gradients as GEMMs over the batch).  The loss and the
gradient of every layer are compared with the FP64 MLP oracle (itself pinned
by central finite differences); the bound is set by FP16 operands (11
significand bits: activations, weights and output errors each rounded once,
about 5e-4 relative per value, a few such roundings along each path), stated
per layer below.  Then the path must train: the loss falls on a small exact
kernel set, as with the FP32 engine."""
import math

import numpy as np
import pytest
import torch

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

# relative L2 bound on each layer's gradient (weights and biases together)
TOL_LAYER = 2e-2
TOL_ALL = 1e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


@pytest.mark.parametrize("npol,n_hidden", [(4, 4), (1, 3), (4, 2)])
def test_tensor_core_gradient_matches_fp64_oracle(ctx, npol, n_hidden):
    from paper_2206_15117_gb300 import aw
    omega0 = 30.0
    sur = aw.aw_surrogate_create(ctx, npol=npol, width=128, n_hidden=n_hidden, omega0=omega0, seed=7)
    p = aw.aw_surrogate_get_params(sur).astype(np.float64)
    sizes = omlp.layer_sizes(5, 128, n_hidden, npol * npol)
    rng = np.random.default_rng(9)
    B = 384
    X = rng.uniform(-1, 1, (B, 5)).astype(np.float32)
    T = (0.5 * rng.standard_normal((B, 2 * npol * npol))).astype(np.float32)
    Xd, Td = torch.as_tensor(X, device="cuda"), torch.as_tensor(T, device="cuda")
    g = torch.empty(p.size, dtype=torch.float32, device="cuda")
    loss = aw.aw_surrogate_loss_grad(ctx, sur, Xd, Td, g)
    Yr, cache = omlp.forward(p, sizes, X.astype(np.float64), omega0)
    gr = omlp.backward(p, sizes, cache, Yr, T.astype(np.float64), omega0)
    assert loss == pytest.approx(omlp.loss(Yr, T.astype(np.float64)), rel=5e-3)
    gg = g.cpu().numpy()
    assert np.isfinite(gg).all()
    assert np.linalg.norm(gg - gr) < TOL_ALL * np.linalg.norm(gr)
    off = 0
    for i in range(len(sizes) - 1):
        n = sizes[i + 1] * sizes[i] + sizes[i + 1]
        a, b = gg[off:off + n], gr[off:off + n]
        assert np.linalg.norm(a - b) < TOL_LAYER * np.linalg.norm(b) + 1e-9, (i, np.linalg.norm(a - b) / np.linalg.norm(b))
        off += n
    assert off == p.size
    # the FP32 engine on the same network gives the same gradient to its own (tighter) precision
    aw.aw_surrogate_set_train_engine(sur, aw.AW_TRAIN_FP32)
    g32 = torch.empty_like(g)
    aw.aw_surrogate_loss_grad(ctx, sur, Xd, Td, g32)
    assert np.linalg.norm(g32.cpu().numpy() - gr) < 1e-3 * np.linalg.norm(gr)


def test_tensor_core_training_learns_the_kernels(ctx):
    from paper_2206_15117_gb300 import aw
    N = 512
    kw = dict(N=N, dl=math.radians(2.0) / N, OS=8, W=7.0, npol=1, nw=4, w_max=2000.0, supports=[8, 8, 12, 16])
    exact = aw.aw_make_kernels(ctx, **kw)
    kmax = 0.0
    for b, S in enumerate(kw["supports"]):
        t = torch.empty(kw["OS"] ** 2 * S * S, dtype=torch.complex64, device="cuda")
        aw.aw_kernel_set_export(exact, b, t)
        kmax = max(kmax, float(t.abs().max()))
    sur = aw.aw_surrogate_create(ctx, npol=1, width=128, n_hidden=4, omega0=30.0, D=1.0, norm_supports=kw["supports"],
                                 w_max=kw["w_max"], f_c=1.4e9, f_h=0.2e9, chi_c=0.0, chi_h=1.5, out_scale=kmax, seed=11)
    rep = aw.aw_surrogate_train(ctx, sur, exact, steps=600, batch=8192, lr=1e-3, lr_final=1e-5, seed=3)
    assert rep.steps == 600 and rep.loss_last < 0.05 * rep.loss_first, (rep.loss_first, rep.loss_last)
    _, err, nrej = aw.aw_surrogate_tables(ctx, sur, exact, reject_rel=1e9)
    assert nrej == 0 and float(np.max(err)) < 0.2, err


def test_train_engine_is_checked(ctx):
    from paper_2206_15117_gb300 import aw
    sur = aw.aw_surrogate_create(ctx, npol=4, width=128, n_hidden=4, omega0=30.0, seed=1)
    with pytest.raises(aw.AWError):
        aw.aw_surrogate_set_train_engine(sur, 7)
