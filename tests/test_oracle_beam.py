"""Pins for the oracle's Jones/Mueller/Stokes algebra (Sec. 3.2, Eq. 2-5)
and for the null regularisation of Eq. 6 (Sec. 3.3, Fig. 1)."""
import math
import os

import numpy as np
import pytest

from oracle import core as oc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig1_eq6.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            vals[parts[0]] = parts[1:]
    return vals


def _sinc2(x):
    return np.sinc(x) ** 2


def _sinc2_first_sidelobe():
    # brute force: maximum of sinc^2 between its first and second nulls
    x = np.linspace(1.0, 2.0, 2_000_001)
    return float(_sinc2(x).max())


def _one_sig_fig(x):
    e = math.floor(math.log10(abs(x)))
    return round(x / 10 ** e) * 10 ** e


def test_fig1_divergence_values_printed_in_paper():
    g = _golden()
    eps = float(g["eps"][0])
    B = np.array([1.0, _sinc2_first_sidelobe()])
    assert B[1] == pytest.approx(0.04719, abs=1e-5)
    # the beam as a function of angle: its maximum is 1 (sinc^2(0))
    Bp = oc.regularise_beam(B, eps, Bmax=1.0)
    div = np.abs(1.0 / Bp - 1.0 / B) / np.abs(1.0 / B)
    assert _one_sig_fig(div[0]) == pytest.approx(float(g["centre"][1]))
    assert _one_sig_fig(div[1]) == pytest.approx(float(g["first_sidelobe"][1]))
    assert div[0] == pytest.approx(9.999e-5, rel=1e-3)
    assert div[1] == pytest.approx(4.30e-2, rel=1e-2)


def test_eq6_max_of_inverse_closed_form():
    # 1/|B'| = |B| / (|B|^2 + beta) peaks at |B| = sqrt(beta) with 1/(eps max|B|)
    eps, Bmax = 0.2, 0.8
    x = np.linspace(1e-6, Bmax, 400001)
    B = np.concatenate([x, [Bmax]]) * np.exp(0.3j)
    inv = 1.0 / np.abs(oc.regularise_beam(B, eps, Bmax=Bmax))
    assert inv.max() == pytest.approx(1.0 / (eps * Bmax), rel=1e-6)
    beta = (eps / 2 * Bmax) ** 2
    assert abs(np.abs(B[np.argmax(inv)]) - math.sqrt(beta)) < 1e-5


def test_eq6_keeps_phase_and_large_values():
    eps = 0.2
    rng = np.random.default_rng(3)
    B = rng.uniform(0.5, 1.0, 50) * np.exp(1j * rng.uniform(-3, 3, 50))
    Bp = oc.regularise_beam(B, eps, Bmax=1.0)
    np.testing.assert_allclose(np.angle(Bp), np.angle(B), atol=1e-14)
    beta = (eps / 2) ** 2
    np.testing.assert_allclose(np.abs(Bp), np.abs(B) + beta / np.abs(B), rtol=1e-14)
    # the maximum over the pattern comes from the data when not given
    np.testing.assert_allclose(oc.regularise_beam(B, eps), oc.regularise_beam(B, eps, Bmax=np.abs(B).max()))


def test_eq6_null_gives_zero_inverse():
    Bp = oc.regularise_beam(np.array([0.0, 1.0]), 0.2)
    assert np.isfinite(Bp).all()
    assert abs(1.0 / Bp[0]) < 1e-10


def test_stokes_matrices_are_inverse_and_match_eq4():
    np.testing.assert_allclose(oc.T_CORR_TO_STOKES @ oc.T_STOKES_TO_CORR, np.eye(4), atol=1e-15)
    # Eq. 4 rows for I, Q and V as printed; U read as (XY + YX) / 2
    XX, XY, YX, YY = 1.3 + 0.1j, 0.2 - 0.4j, 0.7 + 0.3j, 0.5 - 0.2j
    I, Q, U, V = oc.T_CORR_TO_STOKES @ np.array([XX, XY, YX, YY])
    assert I == pytest.approx((XX + YY) / 2)
    assert Q == pytest.approx((XX - YY) / 2)
    assert V == pytest.approx(1j * (YX - XY) / 2)
    assert U == pytest.approx((XY + YX) / 2)


def test_unpolarised_and_pure_u_sources():
    corr = np.array([2.0, 0.0, 0.0, 2.0])  # unpolarised: XX = YY, no cross terms
    s = oc.T_CORR_TO_STOKES @ corr
    np.testing.assert_allclose(s, [2.0, 0, 0, 0], atol=1e-15)
    c = oc.T_STOKES_TO_CORR @ np.array([0, 0, 0.7, 0])   # pure U
    np.testing.assert_allclose(c, [0, 0.7, 0.7, 0], atol=1e-15)
    c = oc.T_STOKES_TO_CORR @ np.array([0, 0, 0, 0.3])   # pure V
    np.testing.assert_allclose(c, [0, 0.3j, -0.3j, 0], atol=1e-15)


def _random_jones(rng):
    return rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))


def test_kronecker_mixed_product_and_identity():
    rng = np.random.default_rng(5)
    J1, J2 = _random_jones(rng), _random_jones(rng)
    lhs = oc.mueller_from_jones(J1 @ J2)
    rhs = oc.mueller_from_jones(J1) @ oc.mueller_from_jones(J2)
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)
    np.testing.assert_allclose(oc.mueller_from_jones(np.eye(2)), np.eye(4), atol=0)
    np.testing.assert_allclose(oc.mueller_stokes(np.eye(4, dtype=complex)), np.eye(4), atol=1e-15)
    # entry (ab, cd) = J_ac conj(J_bd) (the coherency <e_a e_b*> transforms this way)
    M = oc.mueller_from_jones(J1)
    for a in range(2):
        for b in range(2):
            for c in range(2):
                for d in range(2):
                    assert M[2 * a + b, 2 * c + d] == pytest.approx(J1[a, c] * np.conj(J1[b, d]))


def test_stokes_mueller_is_real_for_any_jones():
    # real Stokes in -> real Stokes out: a wrong sign or factor i in Eq. 4 breaks this
    rng = np.random.default_rng(7)
    for _ in range(10):
        MS = oc.mueller_stokes(oc.mueller_from_jones(_random_jones(rng)))
        assert np.abs(MS.imag).max() < 1e-12 * np.abs(MS).max()


def test_invert4_matches_library_inverse():
    rng = np.random.default_rng(11)
    A = rng.standard_normal((30, 4, 4)) + 1j * rng.standard_normal((30, 4, 4))
    A[0] = np.array([[0, 1, 0, 0], [1, 0, 0, 0], [0, 0, 0, 2], [0, 0, 3j, 0]])  # needs pivoting
    np.testing.assert_allclose(oc.invert4(A), np.linalg.inv(A), rtol=1e-10, atol=1e-12)


def test_airy_voltage_pattern():
    freq, D = 1.4e9, 12.0
    lam = oc.C_LIGHT / freq
    # first null of 2 J1(x)/x at x = 3.8317..., i.e. sin r = 1.21967 lambda / D
    r0 = 3.8317059702075125 * lam / (math.pi * D)
    E = oc.airy_voltage(np.array([0.0, r0]), np.array([0.0, 0.0]), freq, D)
    assert E[0] == 1.0
    assert abs(E[1]) < 1e-12
    # half-power of the power pattern E^2 at x = 1.6163...
    rh = 1.616339948310703 * lam / (math.pi * D)
    Eh = oc.airy_voltage(np.array([rh / math.sqrt(2)]), np.array([rh / math.sqrt(2)]), freq, D)
    assert Eh[0] ** 2 == pytest.approx(0.5, rel=1e-9)


def test_jones_structure():
    l = np.array([0.0]); m = np.array([0.0])
    J = oc.jones(l, m, 1.4e9, 0.0, 12.0, 0.01j, -0.02)[0]
    np.testing.assert_allclose(J, [[1, 0.01j], [-0.02, 1]])
    chi = 0.4
    J = oc.jones(l, m, 1.4e9, chi, 12.0, 0.0, 0.0)[0]
    np.testing.assert_allclose(J, [[math.cos(chi), -math.sin(chi)], [math.sin(chi), math.cos(chi)]])
    # a feed rotation by chi rotates (Q, U) by 2 chi and leaves I, V alone
    MS = oc.mueller_stokes(oc.mueller_from_jones(J)).real
    c2, s2 = math.cos(2 * chi), math.sin(2 * chi)
    expect = np.array([[1, 0, 0, 0], [0, c2, -s2, 0], [0, s2, c2, 0], [0, 0, 0, 1]])
    assert np.allclose(MS, expect, atol=1e-12) or np.allclose(MS, expect.T, atol=1e-12)
