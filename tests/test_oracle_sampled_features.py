"""Pins of two oracle functions the full-size and learned-kernel parity tests
lean on:

* `core.degrid_sampled` (degridding of chosen visibilities one by one, each
  with only its own kernel block synthesised) must equal the tabulated C-loop
  degridder `core.degrid` (itself pinned by the adjoint identity and the
  direct DFT) on every visibility, flipped samples included;
* `mlp.features` (the surrogate's five inputs: tap offset over the
  normalisation scale of the w plane |w| falls in, w, frequency and
  parallactic angle, each mapped to [-1, 1]) is checked at hand-computed
  points: on plane boundaries, past w_max (clamped to the last plane), at the
  edges of the frequency and angle ranges; and inline gridding with a
  stand-in network that uses all five features is checked against an
  explicit loop that forms the features by hand.
"""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import mlp as omlp
from paper_2206_15117_gb300 import synthetic as sy
from tests.oracle_cases import small_case


@pytest.mark.parametrize("npol", [1, 4])
def test_degrid_sampled_equals_the_tabulated_degridder(npol):
    ob, base = small_case(npol=npol, nw=3, S=10, N=64, n_t=16)
    base["supports"] = [8, 10, 12]
    spec = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    assert co.flip.any() and (co.flip == 0).any()
    assert len(set(spec.plane_of(co.bin[co.valid == 1]).tolist())) == 3
    rng = np.random.default_rng(11)
    G = rng.standard_normal((npol, spec.N, spec.N)) + 1j * rng.standard_normal((npol, spec.N, spec.N))
    ref = oc.degrid(oc.make_kernels(spec), co, G)
    # every visibility, in a shuffled order (the result follows idx)
    idx = rng.permutation(co.x0.shape[0])
    got = oc.degrid_sampled(spec, G, co, idx)
    assert np.abs(got - ref[idx]).max() <= 1e-12 * np.abs(ref).max()
    # the flipped samples are where a wrong P conj() would show
    fl = co.flip[idx] == 1
    assert np.abs(got[fl]).max() > 0.1 * np.abs(ref).max()


def test_degrid_sampled_catches_a_planted_transpose(monkeypatch):
    """The pin above fails if degrid_sampled applied K[c][s] as K[s][c]."""
    ob, base = small_case(npol=4, nw=2, S=8, N=64, n_t=8)
    spec = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    G = np.random.default_rng(3).standard_normal((4, spec.N, spec.N)) + 0j
    ref = oc.degrid(oc.make_kernels(spec), co, G)
    real_synth = oc.synth_bin

    def transposed(spec_, b, offsets_y=None, offsets_x=None):
        K = real_synth(spec_, b, offsets_y=offsets_y, offsets_x=offsets_x)
        return K.reshape(K.shape[:4] + (4, 4)).swapaxes(-1, -2).reshape(K.shape[:4] + (16,))
    monkeypatch.setattr(oc, "synth_bin", transposed)
    got = oc.degrid_sampled(spec, G, co, np.arange(co.x0.shape[0]))
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


# ---------------------------------------------------------------- features

D, NS, WMAX = 1.5, [8, 12, 16, 20], 400.0
FC, FH, CC, CH = 1.35e9, 0.1e9, 0.2, 0.5


def _feat(du, dv, w, f, chi):
    return omlp.features(np.asarray([du], float), np.asarray([dv], float), np.asarray([w], float),
                         np.asarray([f], float), np.asarray([chi], float), D, NS, WMAX, FC, FH, CC, CH)[0]


@pytest.mark.parametrize("w, plane", [
    (0.0, 0), (99.999, 0),      # inside the first quarter of [0, w_max)
    (100.0, 1),                 # exactly on the first boundary: the upper plane
    (200.0, 2), (299.0, 2),
    (300.0, 3), (399.999, 3),
    (400.0, 3), (1e4, 3),       # at and past w_max: clamped to the last plane
])
def test_features_pick_the_normalisation_plane_of_w(w, plane):
    # the normalisation scale is D (S / 2 + 1) with S the support of that plane
    s = D * (NS[plane] / 2 + 1)
    x = _feat(3.0, -2.0, w, FC, CC)
    assert x[0] == pytest.approx(3.0 / s, rel=1e-15)
    assert x[1] == pytest.approx(-2.0 / s, rel=1e-15)
    assert x[2] == pytest.approx(2 * w / WMAX - 1, rel=1e-15, abs=1e-15)


def test_features_map_the_ranges_to_plus_minus_one():
    lo = _feat(0.0, 0.0, 0.0, FC - FH, CC - CH)
    hi = _feat(0.0, 0.0, WMAX, FC + FH, CC + CH)
    mid = _feat(0.0, 0.0, WMAX / 2, FC, CC)
    np.testing.assert_allclose(lo[2:], [-1.0, -1.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(hi[2:], [1.0, 1.0, 1.0], atol=1e-15)
    np.testing.assert_allclose(mid[2:], [0.0, 0.0, 0.0], atol=1e-15)
    # hand values: f = 1.30 GHz, chi = 0.45 rad, w = 50
    x = _feat(-5.0, 7.5, 50.0, 1.30e9, 0.45)
    s = D * (8 / 2 + 1)
    np.testing.assert_allclose(x, [-5.0 / s, 7.5 / s, -0.75, -0.5, 0.5], rtol=1e-14)


def test_features_of_odd_supports_use_the_floor_of_half():
    # S = 7: S // 2 + 1 = 4
    x = omlp.features(np.array([4.0]), np.array([0.0]), np.array([0.0]), np.array([FC]), np.array([CC]),
                      2.0, [7], WMAX, FC, FH, CC, CH)[0]
    assert x[0] == pytest.approx(4.0 / (2.0 * 4))


def _stand_in(X):
    """A network stand-in whose 2P outputs use all five features: K_m =
    M_m g(x0, x1) (1 + 0.3 x2 + 0.5 x3 - 0.7 x4)."""
    g = np.exp(-0.5 * (X[:, 0] ** 2 + X[:, 1] ** 2) / 0.09)
    return g * (1.0 + 0.3 * X[:, 2] + 0.5 * X[:, 3] - 0.7 * X[:, 4])


@pytest.mark.parametrize("per_channel", [False, True])
def test_inline_gridding_uses_w_frequency_and_angle_features(monkeypatch, per_channel):
    NPOL = 4
    ob = sy.small_observation(n_ant=8, radius_m=60.0, n_t=12, freq=(1.25e9, 1.3e9, 1.4e9, 1.45e9),
                              npa=2, nfb=2, z_spread_m=25.0)
    N = 64
    sup = [8, 10, 12, 14]
    spec = oc.KernelSpec(N=N, dl=math.radians(4.0) / N, OS=8, npol=NPOL, nw=4, w_max=ob.w_max, supports=sup,
                         pa=tuple(ob.pa_centres), fbin_freqs=tuple(ob.fbin_freqs))
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, ob.pa_bin, ob.fbin)
    norm = [9, 13]                         # two normalisation planes over [0, w_max)
    Dn, fc, fh, cc, ch = 1.25, 1.35e9, 0.12e9, float(np.mean(ob.pa_centres)), 0.8
    scales = (Dn, norm, ob.w_max, fc, fh, cc, ch, 1.0)
    rng = np.random.default_rng(4)
    M = rng.standard_normal((NPOL, NPOL)) + 1j * rng.standard_normal((NPOL, NPOL))
    Mf = M.reshape(-1)

    def fwd(p, sizes, X, omega0):
        K = _stand_in(X)[:, None] * Mf[None, :]
        out = np.empty((X.shape[0], 2 * Mf.size))
        out[:, 0::2], out[:, 1::2] = K.real, K.imag
        return out, None
    monkeypatch.setattr(omlp, "forward", fwd)
    v = rng.standard_normal((ob.nvis, NPOL)) + 1j * rng.standard_normal((ob.nvis, NPOL))
    G = omlp.grid_inline(np.zeros(1), [5, 8], 1.0, scales, spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq,
                         co, v, None, fp16_layers=False, per_channel=per_channel)
    ref = np.zeros((NPOL, N, N), np.complex128)
    valid = np.flatnonzero(co.valid == 1)
    assert co.flip[valid].any() and (co.flip[valid] == 0).any()
    seen_planes = set()
    for k in valid:
        lam = oc.C_LIGHT / ob.freq[ob.chan_of_vis[k]]
        u, vv, ww = ob.uvw[ob.row_of_vis[k]] / lam
        vk = v[k].copy()
        if ww < 0:
            u, vv, ww = -u, -vv, -ww
            vk = np.conj(vk)[[0, 2, 1, 3]]
        X = u * N * spec.dl + N / 2
        Y = vv * N * spec.dl + N / 2
        # normalisation plane by explicit comparison with the plane edges
        q = 0
        while q + 1 < len(norm) and ww >= (q + 1) * ob.w_max / len(norm):
            q += 1
        seen_planes.add(q)
        s = Dn * (norm[q] // 2 + 1)
        fq = ob.freq[ob.chan_of_vis[k]] if per_channel else ob.fbin_freqs[ob.fbin[ob.chan_of_vis[k]]]
        chi = ob.pa_centres[ob.pa_bin[ob.row_of_vis[k]]]
        x2, x3, x4 = 2 * ww / ob.w_max - 1, (fq - fc) / fh, (chi - cc) / ch
        S = sup[spec.plane_of(co.bin[k])]
        for y in range(co.y0[k], co.y0[k] + S):
            for x in range(co.x0[k], co.x0[k] + S):
                g = math.exp(-0.5 * (((x - X) / s) ** 2 + ((y - Y) / s) ** 2) / 0.09)
                kv = g * (1.0 + 0.3 * x2 + 0.5 * x3 - 0.7 * x4)
                for si in range(NPOL):
                    for c in range(NPOL):
                        ref[si, y, x] += M[si, c] * kv * vk[c]
    assert seen_planes == {0, 1}
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()
