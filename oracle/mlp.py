"""FP64 oracle of the learned kernel surrogate: a SIREN-style coordinate MLP.

TEST INFRASTRUCTURE ONLY.  The surrogate maps continuous kernel coordinates
to the P complex Mueller kernel values of one tap, standing in for the
per-bin FFT synthesis of Sec. 3.2 (the kernels it learns are the uv
transforms of the Mueller cells times the anti-aliasing function and the w
term).  Definitions shared with the CUDA path (written separately there):

* features (5): x = [d_u / s, d_v / s, 2 w / w_max - 1, (f - f_c) / f_h,
  (chi - chi_c) / chi_h], with (d_u, d_v) the grid-minus-visibility offset of
  the tap in cells and s = D (S(w)/2 + 1), S(w) = norm_supports[floor(w n /
  w_max)] (clamped) for a fixed layout of n normalisation planes;
* layers: sizes [5, H, H, H, H, 2P]; the first four apply
  h = sin(omega0 * (W h_prev + b)), the last is linear;
* parameters: one flat vector, per layer W [out][in] row-major then b [out];
* loss: L = (1/B) sum_b sum_j (y_bj - t_bj)^2;
* Adam (Kingma & Ba): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
  p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).

Pinned by central finite differences in tests/test_oracle_mlp.py.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def layer_sizes(n_in: int = 5, width: int = 128, n_hidden: int = 4, P: int = 16) -> List[int]:
    return [n_in] + [width] * n_hidden + [2 * P]


def n_params(sizes: Sequence[int]) -> int:
    return sum(sizes[i + 1] * sizes[i] + sizes[i + 1] for i in range(len(sizes) - 1))


def unpack(params: np.ndarray, sizes: Sequence[int]) -> List[Tuple[np.ndarray, np.ndarray]]:
    out, pos = [], 0
    for i in range(len(sizes) - 1):
        n_in, n_out = sizes[i], sizes[i + 1]
        W = params[pos:pos + n_out * n_in].reshape(n_out, n_in)
        pos += n_out * n_in
        b = params[pos:pos + n_out]
        pos += n_out
        out.append((W, b))
    return out


def forward(params: np.ndarray, sizes: Sequence[int], X: np.ndarray, omega0: float):
    """Returns (Y [B][2P], cache of pre-activations and activations)."""
    layers = unpack(np.asarray(params, np.float64), sizes)
    h = np.asarray(X, np.float64)
    acts, pres = [h], []
    for li, (W, b) in enumerate(layers):
        z = h @ W.T + b
        pres.append(z)
        if li < len(layers) - 1:
            h = np.sin(omega0 * z)
        else:
            h = z
        acts.append(h)
    return h, (acts, pres)


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    return float(np.sum((Y - T) ** 2) / Y.shape[0])


def backward(params: np.ndarray, sizes: Sequence[int], cache, Y: np.ndarray, T: np.ndarray,
             omega0: float) -> np.ndarray:
    """Analytic gradient of loss(Y, T) with respect to the flat parameters."""
    layers = unpack(np.asarray(params, np.float64), sizes)
    acts, pres = cache
    B = Y.shape[0]
    grads = []
    dz = 2.0 * (Y - T) / B
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        h_prev = acts[li]
        dW = dz.T @ h_prev
        db = dz.sum(axis=0)
        grads.append((dW, db))
        if li > 0:
            dh = dz @ W
            dz = dh * omega0 * np.cos(omega0 * pres[li - 1])
    flat = []
    for dW, db in reversed(grads):
        flat.append(dW.reshape(-1))
        flat.append(db)
    return np.concatenate(flat)


def adam_step(params, grads, m, v, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8):
    m = b1 * m + (1 - b1) * grads
    v = b2 * v + (1 - b2) * grads * grads
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def features(du, dv, w, f, chi, D, norm_supports, w_max, f_c, f_h, chi_c, chi_h) -> np.ndarray:
    du = np.asarray(du, np.float64)
    w = np.asarray(w, np.float64)
    ns = np.asarray(norm_supports)
    pn = np.clip(np.floor(w * len(ns) / w_max).astype(np.int64), 0, len(ns) - 1)
    s = D * (ns[pn] // 2 + 1)
    return np.stack([du / s, np.asarray(dv) / s, 2.0 * w / w_max - 1.0,
                     (np.asarray(f) - f_c) / f_h, (np.asarray(chi) - chi_c) / chi_h], axis=-1)


def _fp16_rounded(params, sizes, fp16_layers):
    """FP64 parameters with the weights of the tensor-core layers (all but the
    first) rounded to FP16 when fp16_layers, as the GPU stores them."""
    p = np.array(params, np.float64)
    if fp16_layers:
        pos = sizes[0] * sizes[1] + sizes[1]
        for li in range(1, len(sizes) - 1):
            n_in, n_out = sizes[li], sizes[li + 1]
            p[pos:pos + n_out * n_in] = p[pos:pos + n_out * n_in].astype(np.float16).astype(np.float64)
            pos += n_out * n_in + n_out
    return p


def _inline_kernels(p, sizes, omega0, scales, spec, uvw, row_of_vis, chan_of_vis, freq, co, per_channel):
    """For every valid visibility k (in index order): (k, K) with K the network's
    kernel [S][S][npol][npol] at the taps of its footprint.  Tap (jy, jx) lies at
    d = (x0 + jx) - X cells from the visibility's exact position X = u N dl + N/2
    (u after the w >= 0 flip; no oversampling grid); the features use its exact
    |w|, the centre of its parallactic-angle bin and the centre of its
    beam-frequency bin (per_channel: its own channel frequency); the network's
    2P outputs times out_scale are the P Mueller values."""
    from . import core as oc
    D, norm_supports, w_max, f_c, f_h, chi_c, chi_h, out_scale = scales
    npol, N = spec.npol, spec.N
    f = np.asarray(freq, np.float64)[chan_of_vis] / oc.C_LIGHT
    uvwl = np.asarray(uvw, np.float64)[row_of_vis] * f[:, None]
    for k in np.flatnonzero(co.valid == 1):
        u, vv, ww = uvwl[k]
        if co.flip[k]:
            u, vv, ww = -u, -vv, -ww
        X = u * (N * spec.dl) + N // 2
        Y = vv * (N * spec.dl) + N // 2
        b = co.bin[k]
        pidx = spec.plane_of(b)
        a = (b // spec.nfb) % spec.npa
        S = spec.supports[pidx]
        jy, jx = np.meshgrid(np.arange(S), np.arange(S), indexing="ij")
        du = (co.x0[k] + jx.ravel()) - X
        dv = (co.y0[k] + jy.ravel()) - Y
        nf = du.size
        fb = b % spec.nfb
        fq = freq[chan_of_vis[k]] if per_channel else spec.fbin_freqs[fb]
        Xf = features(du, dv, np.full(nf, ww), np.full(nf, fq), np.full(nf, spec.pa[a]),
                      D, norm_supports, w_max, f_c, f_h, chi_c, chi_h)
        out, _ = forward(p, sizes, Xf, omega0)
        K = (out[:, 0::2] + 1j * out[:, 1::2]) * out_scale          # [taps][P]
        yield k, K.reshape(S, S, npol, npol)


def grid_inline(params, sizes, omega0, scales, spec, uvw, row_of_vis, chan_of_vis, freq, co, vis, weight=None,
                fp16_layers=True, per_channel=False):
    """Gridding with the surrogate evaluated at every (visibility, tap) point
    (see _inline_kernels): G[s][y0 + jy][x0 + jx] += sum_c K_{s,c} w'_c V'_c,
    with V', w' the flipped visibility and weights (V' = P conj V for w < 0).
    `scales` = (D, norm_supports, w_max, f_c, f_h, chi_c, chi_h, out_scale).
    """
    npol, N = spec.npol, spec.N
    p = _fp16_rounded(params, sizes, fp16_layers)
    G = np.zeros((npol, N, N), np.complex128)
    v = np.asarray(vis, np.complex128).reshape(-1, npol)
    w = np.ones(v.shape, np.float64) if weight is None else np.asarray(weight, np.float64).reshape(-1, npol)
    for k, K in _inline_kernels(p, sizes, omega0, scales, spec, uvw, row_of_vis, chan_of_vis, freq, co,
                                per_channel):
        vk, wk = v[k].copy(), w[k].copy()
        if co.flip[k]:
            vk = np.conj(vk)
            if npol == 4:
                vk = vk[[0, 2, 1, 3]]
                wk = wk[[0, 2, 1, 3]]
        S = K.shape[0]
        contrib = np.einsum("yxsc,c->syx", K, wk * vk)              # K [jy][jx][s][c]
        G[:, co.y0[k]:co.y0[k] + S, co.x0[k]:co.x0[k] + S] += contrib
    return G


def degrid_inline(params, sizes, omega0, scales, spec, uvw, row_of_vis, chan_of_vis, freq, co, G,
                  fp16_layers=True, per_channel=False):
    """Degridding with the surrogate (trained on degridding kernels) evaluated
    at every (visibility, tap) point (see _inline_kernels):
    V_c = sum_taps sum_s K_{c,s} G_s[y0 + jy][x0 + jx], then P conj(V) for a
    visibility flipped to w >= 0; invalid visibilities give 0.  Returns
    complex128 [nvis][npol]."""
    npol = spec.npol
    p = _fp16_rounded(params, sizes, fp16_layers)
    G = np.asarray(G, np.complex128)
    out = np.zeros((co.x0.shape[0], npol), np.complex128)
    for k, K in _inline_kernels(p, sizes, omega0, scales, spec, uvw, row_of_vis, chan_of_vis, freq, co,
                                per_channel):
        S = K.shape[0]
        win = G[:, co.y0[k]:co.y0[k] + S, co.x0[k]:co.x0[k] + S]   # [s][jy][jx]
        vk = np.einsum("yxcs,syx->c", K, win)                       # K [jy][jx][c][s]
        if co.flip[k]:
            vk = np.conj(vk)
            if npol == 4:
                vk = vk[[0, 2, 1, 3]]
        out[k] = vk
    return out
