"""Pins for the oracle's coordinates, gridding, degridding and uv->image step
against brute force and the mathematics (Eq. 2 evaluated directly, the
adjoint identity, a point source at the phase centre, Hermitian symmetry)."""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import core as oc
from tests.oracle_cases import all_pixels_lm, quantised_uvw, small_case


def _setup(npol=1, role=oc.ROLE_GRID, **kw):
    ob, base = small_case(npol=npol, **kw)
    spec = oc.KernelSpec(**base, role=role)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    return ob, base, spec, co


def _sources(N, rng, n=6, spread=14):
    qx = rng.integers(N // 2 - spread, N // 2 + spread, n)
    qy = rng.integers(N // 2 - spread, N // 2 + spread, n)
    return qx, qy


@pytest.mark.parametrize("W,S,tol", [(7.0, 12, 1e-4), (9.0, 16, 5e-6)])
def test_stokes_i_grid_and_degrid_match_direct_dft(W, S, tol):
    # the direct sum of Eq. 2 at the coordinates the method quantises to (the
    # oversampled uv cell and the w-plane centre); what is left is the
    # anti-aliasing error of the truncated kernel, which shrinks with W and S
    ob, base, spec, co = _setup(W=W, S=S)
    assert co.valid.all() and co.flip.any() and (co.flip == 0).any()
    N, dl = spec.N, spec.dl
    rng = np.random.default_rng(1)
    qx, qy = _sources(N, rng)
    I = rng.uniform(0.1, 1, qx.size)
    uq = quantised_uvw(spec, co)
    V = oc.dft_predict(uq, oc.pixel_lm(N, dl, qx, qy), I + 0j)
    vin = np.where(co.flip == 1, np.conj(V), V)            # as observed (before the flip)
    ks = oc.make_kernels(spec)
    G, ws, nbad = oc.grid(ks, co, vin)
    assert nbad == 0 and ws == pytest.approx(ob.nvis)
    img = oc.fft_to_image(G, W, ws)[0]
    D = oc.dft_adjoint(uq, V, all_pixels_lm(N, dl)).real.reshape(N, N) / ws
    inner = slice(N // 4, 3 * N // 4)
    assert np.abs(img - D)[inner, inner].max() < tol * np.abs(D).max()
    model = np.zeros((1, N, N))
    np.add.at(model[0], (qy, qx), I)
    ksd = oc.make_kernels(oc.KernelSpec(**base, role=oc.ROLE_DEGRID))
    Vd = oc.degrid(ksd, co, oc.image_to_grid(model, W))[:, 0]
    assert np.abs(Vd - vin).max() < 2 * tol * np.abs(V).max()


def _mueller_at(spec, lm):
    l, m = lm[:, 0], lm[:, 1]
    J = oc.jones(l, m, spec.fbin_freqs[0], spec.pa[0], spec.dish_d, spec.d_xy, spec.d_yx)
    return oc.mueller_from_jones(J)


def test_fullpol_degrid_matches_direct_mueller_dft():
    # Eq. 2 with the Mueller matrix and Eq. 4: V_c = sum_pix (M T^-1)_{c,s} I_s e^{-2 pi i b.s}
    ob, base, spec, co = _setup(npol=4, role=oc.ROLE_DEGRID, W=9.0, S=16)
    N, dl = spec.N, spec.dl
    rng = np.random.default_rng(2)
    qx, qy = _sources(N, rng, n=4, spread=10)
    lm = oc.pixel_lm(N, dl, qx, qy)
    stokes = np.stack([rng.uniform(0.5, 1, 4), rng.uniform(-0.1, 0.1, 4),
                       rng.uniform(-0.1, 0.1, 4), rng.uniform(-0.01, 0.01, 4)], 1)
    A = _mueller_at(spec, lm) @ oc.T_STOKES_TO_CORR               # [src][c][s]
    brightness = np.einsum("pcs,ps->pc", A, stokes)                # per source, per correlation
    uq = quantised_uvw(spec, co)
    Vq = np.stack([oc.dft_predict(uq, lm, brightness[:, c]) for c in range(4)], 1)
    # undo the flip: V_obs = P conj(V at the flipped coordinate)
    Vobs = Vq.copy()
    fl = co.flip == 1
    Vobs[fl] = np.conj(Vq[fl][:, [0, 2, 1, 3]])
    model = np.zeros((4, N, N))
    for s in range(4):
        np.add.at(model[s], (qy, qx), stokes[:, s])
    ks = oc.make_kernels(spec)
    Vd = oc.degrid(ks, co, oc.image_to_grid(model, spec.W))
    assert np.abs(Vd - Vobs).max() < 2e-4 * np.abs(Vobs).max()


def test_fullpol_grid_matches_direct_adjoint_with_inverse_mueller():
    # gridding with the regularised inverse: I_s(l) = sum_c ((M^S)'^-1 T)_{s,c}(l) D_c(l),
    # D_c the direct dirty image of correlation c (Sec. 3.2-3.3)
    ob, base, spec, co = _setup(npol=4, role=oc.ROLE_GRID, W=9.0, S=16)
    N, dl = spec.N, spec.dl
    rng = np.random.default_rng(4)
    vobs = rng.standard_normal((ob.nvis, 4)) + 1j * rng.standard_normal((ob.nvis, 4))
    ks = oc.make_kernels(spec)
    G, ws, _ = oc.grid(ks, co, vobs)
    img = oc.fft_to_image(G, spec.W, ws)
    # direct: flip as the method does, then the adjoint DFT per correlation
    v = vobs.copy()
    fl = co.flip == 1
    v[fl] = np.conj(vobs[fl][:, [0, 2, 1, 3]])
    uq = quantised_uvw(spec, co)
    inner = np.arange(N // 4, 3 * N // 4, 3)
    QX, QY = np.meshgrid(inner, inner)
    lm = oc.pixel_lm(N, dl, QX.ravel(), QY.ravel())
    D = np.stack([oc.dft_adjoint(uq, v[:, c], lm) for c in range(4)], 1) / ws   # [pix][c]
    # the regularised inverse needs max|B_p| over the synthesis image: the beam centre
    MS = oc.mueller_stokes(_mueller_at(spec, lm))
    MS0 = oc.mueller_stokes(_mueller_at(spec, np.zeros((1, 2))))[0]
    MSr = MS.copy()
    for p in range(4):
        MSr[:, p, p] = oc.regularise_beam(MS[:, p, p], spec.eps, Bmax=abs(MS0[p, p]))
    Ginv = oc.invert4(MSr) @ oc.T_CORR_TO_STOKES
    expect = np.einsum("psc,pc->ps", Ginv, D).real
    got = img[:, QY.ravel(), QX.ravel()].T
    assert np.abs(got - expect).max() < 2e-4 * np.abs(expect).max()


@pytest.mark.parametrize("npol", [1, 4])
def test_adjoint_identity(npol):
    # <Grid v, x> = <v, Degrid_adjoint x>.  The w < 0 flip conjugates, so
    # gridding is real-linear: the identity holds for the real inner product
    # Re<a, b>, and for the complex one on visibilities that are not flipped.
    ob, base, spec, co = _setup(npol=npol, W=7.0, S=12)
    rng = np.random.default_rng(9)
    v = rng.standard_normal((ob.nvis, npol)) + 1j * rng.standard_normal((ob.nvis, npol))
    x = rng.standard_normal((npol, spec.N, spec.N)) + 1j * rng.standard_normal((npol, spec.N, spec.N))
    ks = oc.make_kernels(spec)
    ka = oc.make_kernels(oc.KernelSpec(**base, role=oc.ROLE_ADJOINT))
    G, _, _ = oc.grid(ks, co, v)
    Dx = oc.degrid(ka, co, x)
    lhs, rhs = np.vdot(G, x), np.vdot(v, Dx)
    assert co.flip.any()
    assert abs(lhs.real - rhs.real) < 1e-12 * abs(lhs)
    keep = co.flip == 0
    v0 = np.where(keep[:, None], v, 0)
    G0, _, _ = oc.grid(ks, co, v0)
    lhs0, rhs0 = np.vdot(G0, x), np.vdot(v0, Dx)
    assert abs(lhs0 - rhs0) < 1e-12 * abs(lhs0)


def test_point_source_at_phase_centre():
    # Eq. 2: a point source at the phase centre gives V = S for every (u, v, w)
    ob, base, spec, co = _setup(W=9.0, S=16)
    S_jy = 2.5
    model = np.zeros((1, spec.N, spec.N))
    model[0, spec.N // 2, spec.N // 2] = S_jy
    ksd = oc.make_kernels(oc.KernelSpec(**base, role=oc.ROLE_DEGRID))
    V = oc.degrid(ksd, co, oc.image_to_grid(model, spec.W))[:, 0]
    assert np.abs(V - S_jy).max() < 1e-5 * S_jy
    # and gridding constant visibilities gives a dirty-image peak of S at the centre
    G, ws, _ = oc.grid(oc.make_kernels(spec), co, np.full(ob.nvis, S_jy + 0j))
    img = oc.fft_to_image(G, spec.W, ws)[0]
    assert img[spec.N // 2, spec.N // 2] == pytest.approx(S_jy, rel=1e-5)
    assert np.unravel_index(np.argmax(img), img.shape) == (spec.N // 2, spec.N // 2)


def test_dirty_image_of_hermitian_data_is_real():
    # w = 0 (no flip): grid V(b) and V(-b) = conj V(b) -> Hermitian grid -> real
    # image.  A visibility exactly half way between two footprint choices
    # (fine offset 0) has no mirror-symmetric footprint, so those are dropped.
    ob, base = small_case(nw=1)
    ob.uvw[:, 2] = 0.0
    uvw2 = np.concatenate([ob.uvw, -ob.uvw])
    nrow = ob.uvw.shape[0]
    row = np.concatenate([ob.row_of_vis, ob.row_of_vis + nrow]).astype(np.uint32)
    chan = np.concatenate([ob.chan_of_vis, ob.chan_of_vis])
    spec = oc.KernelSpec(**base)
    co = oc.coords(spec, uvw2, row, chan, ob.freq)
    assert co.valid.all() and not co.flip.any()
    n = ob.nvis
    tie = (co.fx[:n] == 0) | (co.fy[:n] == 0) | (co.fx[n:] == 0) | (co.fy[n:] == 0)
    assert tie.sum() < n // 4
    rng = np.random.default_rng(13)
    v = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    v[tie] = 0
    G, ws, _ = oc.grid(oc.make_kernels(spec), co, np.concatenate([v, np.conj(v)]))
    img = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(G[0])))
    assert np.abs(img.imag).max() < 1e-12 * np.abs(img.real).max()
    # the footprints of a visibility and its mirror image are mirror images
    keep = ~tie
    S = spec.supports[0]
    assert np.all(co.x0[:n][keep] + co.x0[n:][keep] + S - 1 == spec.N)


def test_coordinates_round_like_exact_arithmetic():
    ob, base, spec, co = _setup()
    OS, N = spec.OS, spec.N
    uscale = Fraction(N) * Fraction(spec.dl) * OS
    c = Fraction(oc.C_LIGHT)
    ties = 0
    for k in range(0, ob.nvis, 7):
        r, ch = int(ob.row_of_vis[k]), int(ob.chan_of_vis[k])
        f = Fraction(ob.freq[ch]) / c
        u = Fraction(ob.uvw[r, 0]) * f
        w = Fraction(ob.uvw[r, 2]) * f
        if w < 0:
            u = -u
        x = u * uscale + Fraction(N // 2) * OS
        frac = x - math.floor(x)
        if abs(frac - Fraction(1, 2)) < Fraction(1, 10 ** 6):
            ties += 1
            continue
        Xi = math.floor(x + Fraction(1, 2))
        rho = (spec.supports[0] - 2) * OS // 2
        assert co.x0[k] * OS + rho + co.fx[k] == Xi
        assert 0 <= co.fx[k] < OS
        # the footprint holds the S cells nearest the visibility
        S = spec.supports[0]
        cells = co.x0[k] + np.arange(S)
        dist = np.abs(cells - Fraction(Xi, OS))
        assert max(dist) <= Fraction(S, 2)
    assert ties < 3


def test_skip_rule_flags_and_w_planes():
    ob, base = small_case(nw=4, S=12)
    spec = oc.KernelSpec(**base)
    N, dl, OS = spec.N, spec.dl, spec.OS
    du = 1.0 / (N * dl)
    f = 1.4e9
    lam = oc.C_LIGHT / f
    # a visibility on cell X has footprint X - 5 .. X + 6 (S = 12, fine offset 0):
    # it just fits for X = 5 and X = N - 7 and just does not for 4 and N - 6
    def uvw_for_cell(cell):
        return (cell - N // 2) * du * lam
    rows = np.array([[uvw_for_cell(5), 0.0, 1.0], [uvw_for_cell(4), 0.0, 1.0],
                     [uvw_for_cell(N - 7), 0.0, 1.0], [uvw_for_cell(N - 6), 0.0, 1.0],
                     [0.0, 0.0, -10.0 * lam], [0.0, 0.0, spec.w_max * 10 * lam]])
    row = np.arange(rows.shape[0], dtype=np.uint32)
    chan = np.zeros(rows.shape[0], np.uint16)
    flags = np.array([0, 0, 0, 0, 0, 1], np.uint8)
    co = oc.coords(spec, rows, row, chan, np.array([f]), flags=flags)
    assert list(co.valid) == [1, 0, 1, 0, 1, 0]
    assert co.flip[4] == 1 and co.flip[0] == 0
    assert co.bin[4] == 0                      # |w| = 10 -> first plane
    assert co.bin[5] == spec.nw - 1            # clamped to the last plane


def test_nonfinite_visibilities_are_skipped_and_counted():
    ob, base, spec, co = _setup()
    rng = np.random.default_rng(3)
    v = rng.standard_normal(ob.nvis) + 1j * rng.standard_normal(ob.nvis)
    v_bad = v.copy()
    v_bad[[3, 10]] = np.nan
    ks = oc.make_kernels(spec)
    G1, ws1, nb1 = oc.grid(ks, co, v_bad)
    v_zero = v.copy()
    v_zero[[3, 10]] = 0
    valid2 = co.valid.copy()
    G2, _, _ = oc.grid(ks, co, v_zero)
    assert nb1 == 2
    assert ws1 == pytest.approx(ob.nvis - 2)
    np.testing.assert_allclose(G1, G2, atol=1e-12)
