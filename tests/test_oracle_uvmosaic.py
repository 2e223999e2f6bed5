"""Pins of the UV-domain mosaic pieces of the oracle (Sec. 2.2): phase
rotation against direct prediction at both phase centres, the beam-weighted
gridding role as the exact adjoint of degridding, and the pointing offset of
the beam against the direct Mueller sum."""
import math

import numpy as np
import pytest

from oracle import core as oc
from oracle import mosaic as om
from paper_2206_15117_gb300 import synthetic as sy
from tests.oracle_cases import quantised_uvw, small_case


def _small_obs():
    return sy.small_observation(n_ant=8, radius_m=60.0, n_t=10, freq=(1.3e9, 1.4e9))


def test_phase_rotation_equals_prediction_at_the_new_centre():
    # V about centre A, rotated to centre B, equals the direct sum about B with the
    # rotated baselines (sky directions from the trigonometric projection formulas)
    ob = _small_obs()
    A = (1.0, math.radians(-45.0))
    B = (1.0 + math.radians(1.0) / math.cos(A[1]), A[1] + math.radians(0.4))
    rng = np.random.default_rng(0)
    ra = A[0] + rng.uniform(-0.02, 0.02, 5)
    dec = A[1] + rng.uniform(-0.02, 0.02, 5)
    flux = rng.uniform(0.2, 1.0, 5) + 0j
    fa, fb = om.frame(*A, 1e-4, 8), om.frame(*B, 1e-4, 8)
    la, ma, _ = om.radec_to_lmn(fa, ra, dec)
    lb, mb, _ = om.radec_to_lmn(fb, ra, dec)
    uvw_a = ob.uvw
    uvw_b, _ = oc.phase_rotate(uvw_a, ob.row_of_vis, ob.chan_of_vis, ob.freq, np.zeros(ob.nvis), A, B)
    Va = oc.dft_predict(oc.uvw_lambda(uvw_a, ob.row_of_vis, ob.chan_of_vis, ob.freq), np.stack([la, ma], 1), flux)
    Vb = oc.dft_predict(oc.uvw_lambda(uvw_b, ob.row_of_vis, ob.chan_of_vis, ob.freq), np.stack([lb, mb], 1), flux)
    _, Vrot = oc.phase_rotate(uvw_a, ob.row_of_vis, ob.chan_of_vis, ob.freq, Va, A, B)
    np.testing.assert_allclose(Vrot, Vb, atol=1e-9 * np.abs(Vb).max())
    # baseline lengths are kept
    np.testing.assert_allclose(np.linalg.norm(uvw_b, axis=1), np.linalg.norm(uvw_a, axis=1), rtol=1e-14)


def test_phase_rotation_round_trip():
    ob = _small_obs()
    A, B = (0.3, -0.7), (0.31, -0.69)
    v = np.random.default_rng(1).normal(size=(ob.nvis, 4)) + 0j
    uvw_b, vb = oc.phase_rotate(ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, v, A, B)
    uvw_a, va = oc.phase_rotate(uvw_b, ob.row_of_vis, ob.chan_of_vis, ob.freq, vb, B, A)
    np.testing.assert_allclose(uvw_a, ob.uvw, atol=1e-9)
    np.testing.assert_allclose(va, v, atol=1e-12)


@pytest.mark.parametrize("npol", [1, 4])
def test_beam_role_is_the_adjoint_of_degridding(npol):
    # <Grid_beam v, x> = <v, Degrid x> (real inner product; complex on unflipped)
    ob, base = small_case(npol=npol, S=12)
    base = {**base, "point_l": 0.01, "point_m": -0.007}
    spec = oc.KernelSpec(**base, role=oc.ROLE_BEAM)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    rng = np.random.default_rng(3)
    v = rng.standard_normal((ob.nvis, npol)) + 1j * rng.standard_normal((ob.nvis, npol))
    x = rng.standard_normal((npol, spec.N, spec.N)) + 1j * rng.standard_normal((npol, spec.N, spec.N))
    kb = oc.make_kernels(spec)
    kd = oc.make_kernels(oc.KernelSpec(**base, role=oc.ROLE_DEGRID))
    G, _, _ = oc.grid(kb, co, v)
    Dx = oc.degrid(kd, co, x)
    lhs, rhs = np.vdot(G, x), np.vdot(v, Dx)
    assert co.flip.any()
    assert abs(lhs.real - rhs.real) < 1e-12 * abs(lhs)
    keep = co.flip == 0
    v0 = np.where(keep[:, None], v, 0)
    G0, _, _ = oc.grid(kb, co, v0)
    assert abs(np.vdot(G0, x) - np.vdot(v0, Dx)) < 1e-12 * abs(np.vdot(G0, x))


def test_offset_beam_degridding_matches_the_direct_mueller_sum():
    # Eq. 2 with the beam centred on the pointing (l_p, m_p) instead of the phase centre
    ob, base = small_case(npol=4, W=9.0, S=16)
    lp, mp = 2.5 * base["dl"] * 4, -1.5 * base["dl"] * 4
    base = {**base, "point_l": lp, "point_m": mp}
    spec = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    N, dl = spec.N, spec.dl
    rng = np.random.default_rng(2)
    qx = rng.integers(N // 2 - 10, N // 2 + 10, 4)
    qy = rng.integers(N // 2 - 10, N // 2 + 10, 4)
    lm = oc.pixel_lm(N, dl, qx, qy)
    stokes = np.stack([rng.uniform(0.5, 1, 4), rng.uniform(-0.1, 0.1, 4),
                       rng.uniform(-0.1, 0.1, 4), rng.uniform(-0.01, 0.01, 4)], 1)
    J = oc.jones(lm[:, 0] - lp, lm[:, 1] - mp, spec.fbin_freqs[0], spec.pa[0], spec.dish_d, spec.d_xy, spec.d_yx)
    A = oc.mueller_from_jones(J) @ oc.T_STOKES_TO_CORR
    bright = np.einsum("pcs,ps->pc", A, stokes)
    uq = quantised_uvw(spec, co)
    Vq = np.stack([oc.dft_predict(uq, lm, bright[:, c]) for c in range(4)], 1)
    Vobs = Vq.copy()
    fl = co.flip == 1
    Vobs[fl] = np.conj(Vq[fl][:, [0, 2, 1, 3]])
    model = np.zeros((4, N, N))
    for s in range(4):
        np.add.at(model[s], (qy, qx), stokes[:, s])
    Vd = oc.degrid(oc.make_kernels(spec), co, oc.image_to_grid(model, spec.W))
    assert np.abs(Vd - Vobs).max() < 2e-4 * np.abs(Vobs).max()
    # the offset matters: the centred beam gives a different answer
    Vc = oc.degrid(oc.make_kernels(oc.KernelSpec(**{**base, "point_l": 0.0, "point_m": 0.0},
                                                 role=oc.ROLE_DEGRID)), co, oc.image_to_grid(model, spec.W))
    assert np.abs(Vc - Vobs).max() > 10 * np.abs(Vd - Vobs).max()
