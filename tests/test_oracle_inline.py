"""Pins of the oracle's inline surrogate gridding and degridding (the network
evaluated at every visibility-tap point): with the network replaced by an
analytic kernel K_{s,c}(d) = M_{s,c} g(d_u, d_v), inline gridding equals a
direct sum over every footprint cell written with explicit loops, and inline
degridding with the conjugate-transposed kernel is its adjoint (flipped
samples included)."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import mlp as omlp
from paper_2206_15117_gb300 import synthetic as sy

NPOL = 4


def _g(du, dv):
    return np.exp(-0.5 * (du * du + dv * dv) / 9.0)


def _case():
    ob = sy.small_observation(n_ant=8, radius_m=60.0, n_t=10, freq=(1.3e9, 1.4e9))
    N = 64
    spec = oc.KernelSpec(N=N, dl=math.radians(4.0) / N, OS=8, npol=NPOL, nw=4, w_max=ob.w_max, supports=[8, 8, 10, 12])
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    # D = 1 and a zero normalisation support make the first two features the raw cell offsets
    scales = (1.0, [0], ob.w_max, 1.35e9, 0.1e9, 0.0, 1.0, 1.0)
    return ob, spec, co, scales


def _patched_forward(M):
    """A stand-in for the network: outputs (re, im) of M_m g(x0, x1) for m = 0..P-1."""
    Mf = np.asarray(M).reshape(-1)

    def fwd(p, sizes, X, omega0):
        g = _g(X[:, 0], X[:, 1])
        K = g[:, None] * Mf[None, :]
        out = np.empty((X.shape[0], 2 * Mf.size))
        out[:, 0::2] = K.real
        out[:, 1::2] = K.imag
        return out, None
    return fwd


def test_inline_gridding_equals_the_direct_footprint_sum(monkeypatch):
    ob, spec, co, scales = _case()
    rng = np.random.default_rng(0)
    M = rng.standard_normal((NPOL, NPOL)) + 1j * rng.standard_normal((NPOL, NPOL))    # [s][c]
    monkeypatch.setattr(omlp, "forward", _patched_forward(M))
    v = rng.standard_normal((ob.nvis, NPOL)) + 1j * rng.standard_normal((ob.nvis, NPOL))
    w = rng.uniform(0.5, 1.5, (ob.nvis, NPOL))
    G = omlp.grid_inline(np.zeros(1), [5, 8], 1.0, scales, spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq,
                         co, v, w, fp16_layers=False)
    N = spec.N
    ref = np.zeros((NPOL, N, N), np.complex128)
    assert co.flip.any() and (co.flip == 0).any()
    for k in range(ob.nvis):
        if not co.valid[k]:
            continue
        lam = oc.C_LIGHT / ob.freq[ob.chan_of_vis[k]]
        u, vv, ww = ob.uvw[ob.row_of_vis[k]] / lam
        vk, wk = v[k].copy(), w[k].copy()
        if ww < 0:
            u, vv = -u, -vv
            vk = np.conj(vk)[[0, 2, 1, 3]]
            wk = wk[[0, 2, 1, 3]]
        X = u * N * spec.dl + N / 2
        Y = vv * N * spec.dl + N / 2
        S = spec.supports[spec.plane_of(co.bin[k])]
        for y in range(co.y0[k], co.y0[k] + S):
            for x in range(co.x0[k], co.x0[k] + S):
                gv = _g(x - X, y - Y)
                for s in range(NPOL):
                    for c in range(NPOL):
                        ref[s, y, x] += M[s, c] * gv * wk[c] * vk[c]
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


def test_inline_degridding_is_the_adjoint_of_inline_gridding(monkeypatch):
    ob, spec, co, scales = _case()
    rng = np.random.default_rng(1)
    M = rng.standard_normal((NPOL, NPOL)) + 1j * rng.standard_normal((NPOL, NPOL))    # gridding [s][c]
    v = rng.standard_normal((ob.nvis, NPOL)) + 1j * rng.standard_normal((ob.nvis, NPOL))
    x = rng.standard_normal((NPOL, spec.N, spec.N)) + 1j * rng.standard_normal((NPOL, spec.N, spec.N))
    args = (np.zeros(1), [5, 8], 1.0, scales, spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, co)
    monkeypatch.setattr(omlp, "forward", _patched_forward(M))
    G = omlp.grid_inline(*args, v, fp16_layers=False)
    # degridding kernel [c][s] = conj(gridding kernel [s][c])
    monkeypatch.setattr(omlp, "forward", _patched_forward(np.conj(M).T))
    Dx = omlp.degrid_inline(*args, x, fp16_layers=False)
    lhs, rhs = np.vdot(G, x), np.vdot(v, Dx)
    # real inner product: the flip makes both maps real-linear
    assert abs(lhs.real - rhs.real) < 1e-12 * abs(lhs)
    keep = co.flip == 0
    v0 = np.where(keep[:, None], v, 0)
    monkeypatch.setattr(omlp, "forward", _patched_forward(M))
    G0 = omlp.grid_inline(*args, v0, fp16_layers=False)
    assert abs(np.vdot(G0, x) - np.vdot(v0, Dx)) < 1e-12 * abs(np.vdot(G0, x))
    assert np.all(Dx[co.valid == 0] == 0)
