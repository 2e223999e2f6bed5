"""Pins of the per-baseline Mueller kernels of the oracle (Sec. 2.1 and the
baseline averaging of Sec. 3.2 undone): antennas of several types with their
own leakage terms, one kernel class per ordered type pair.

* Degridding a model with the class kernels equals the direct Mueller sum
  V_ij = sum_src (J_i kron conj J_j) T^-1 S exp(-2 pi i (u l + v m + w (n-1)))
  at each visibility's own baseline, flipped samples included (their class
  swaps the two types).
* Identical types reduce to the baseline-averaged kernels.
* The beam-weighted gridding role stays the exact adjoint of degridding.
* The gridding role inverts each class's own Stokes Mueller matrix.
"""
import numpy as np
import pytest

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy
from tests.oracle_cases import quantised_uvw, small_case

TYPE_LEAK = [(0.10 * np.exp(0.3j), 0.08 * np.exp(-0.5j)),
             (-0.12 + 0.0j, 0.05j),
             (0.03 + 0.02j, -0.09 + 0.0j)]
N_ANT = 10
ANT_TYPE = np.array([0, 1, 2, 0, 1, 2, 2, 1, 0, 1])


def _case(role, S=16, W=9.0):
    ob, base = small_case(npol=4, W=W, S=S)
    base = {**base, "type_leak": TYPE_LEAK}
    spec = oc.KernelSpec(**base, role=role)
    rt = sy.row_antenna_types(N_ANT, ob.uvw.shape[0], ANT_TYPE)
    co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, row_types=rt)
    return ob, base, spec, rt, co


def test_bin_layout():
    spec = oc.KernelSpec(N=64, dl=1e-3, OS=4, npol=4, nw=3, w_max=10.0, supports=[8, 10, 12],
                         pa=(0.0, 0.5), fbin_freqs=(1.3e9, 1.4e9), type_leak=TYPE_LEAK)
    assert spec.nclass == 9 and spec.nbins == 9 * 3 * 2 * 2
    b = ((7 * 3 + 2) * 2 + 1) * 2 + 0
    assert spec.decode_bin(b) == (7, 2, 1, 0)
    assert spec.plane_of(b) == 2
    assert spec.leakages(7) == (TYPE_LEAK[2], TYPE_LEAK[1])


def test_degridding_matches_the_direct_per_baseline_mueller_sum():
    ob, base, spec, rt, co = _case(oc.ROLE_DEGRID)
    N, dl = spec.N, spec.dl
    types = rt[ob.row_of_vis]
    # the case exercises flipped samples on baselines between different types
    assert np.any((co.flip == 1) & (types[:, 0] != types[:, 1]))
    assert np.any((co.flip == 0) & (types[:, 0] != types[:, 1]))
    rng = np.random.default_rng(4)
    qx = rng.integers(N // 2 - 10, N // 2 + 10, 4)
    qy = rng.integers(N // 2 - 10, N // 2 + 10, 4)
    lm = oc.pixel_lm(N, dl, qx, qy)
    stokes = np.stack([rng.uniform(0.5, 1, 4), rng.uniform(-0.2, 0.2, 4),
                       rng.uniform(-0.2, 0.2, 4), rng.uniform(-0.02, 0.02, 4)], 1)
    # every sample at its own baseline's coordinates: the flip undone
    uq = quantised_uvw(spec, co)
    u_own = np.where(co.flip[:, None] == 1, -uq, uq)
    Vobs = np.zeros((ob.nvis, 4), np.complex128)
    f0, chi = spec.fbin_freqs[0], spec.pa[0]
    for ti in range(3):
        for tj in range(3):
            sel = (types[:, 0] == ti) & (types[:, 1] == tj)
            if not sel.any():
                continue
            Ji = oc.jones(lm[:, 0], lm[:, 1], f0, chi, spec.dish_d, *TYPE_LEAK[ti])
            Jj = oc.jones(lm[:, 0], lm[:, 1], f0, chi, spec.dish_d, *TYPE_LEAK[tj])
            bright = np.einsum("pcs,ps->pc", oc.mueller_from_jones(Ji, Jj) @ oc.T_STOKES_TO_CORR, stokes)
            for c in range(4):
                Vobs[sel, c] = oc.dft_predict(u_own[sel], lm, bright[:, c])
    model = np.zeros((4, N, N))
    for s in range(4):
        np.add.at(model[s], (qy, qx), stokes[:, s])
    Vd = oc.degrid(oc.make_kernels(spec), co, oc.image_to_grid(model, spec.W))
    err = np.abs(Vd - Vobs).max()
    assert err < 1e-5 * np.abs(Vobs).max(), err
    # the classes matter: baseline-averaged kernels with the mean leakage miss
    # the per-baseline cross-hand terms by far more
    mean = tuple(np.mean([t[q] for t in TYPE_LEAK]) for q in range(2))
    avg = oc.KernelSpec(**{**base, "type_leak": (), "d_xy": mean[0], "d_yx": mean[1]}, role=oc.ROLE_DEGRID)
    co_avg = oc.coords(avg, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    Va = oc.degrid(oc.make_kernels(avg), co_avg, oc.image_to_grid(model, spec.W))
    assert np.abs(Va - Vobs).max() > 20 * err
    # and so does the swap of a flipped sample's types
    co_ns = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, row_types=rt)
    per = spec.nw * spec.npa * spec.nfb
    k = co_ns.bin // per
    ti, tj = k // 3, k % 3
    fl = co_ns.flip == 1
    co_ns.bin = np.where(fl, (tj * 3 + ti) * per + co_ns.bin % per, co_ns.bin).astype(np.int32)
    Vns = oc.degrid(oc.make_kernels(spec), co_ns, oc.image_to_grid(model, spec.W))
    assert np.abs(Vns - Vobs).max() > 20 * err


@pytest.mark.parametrize("role", [oc.ROLE_GRID, oc.ROLE_DEGRID, oc.ROLE_BEAM])
def test_identical_types_reduce_to_baseline_averaged_kernels(role):
    _, base = small_case(npol=4, nw=2, S=8, OS=4)
    d = (base["d_xy"], base["d_yx"])
    one = oc.KernelSpec(**base, role=role)
    many = oc.KernelSpec(**{**base, "type_leak": [d, d]}, role=role)
    per = one.nbins
    for b in (0, per - 1):
        ref = oc.synth_bin(one, b)
        for k in (1, 3):
            np.testing.assert_allclose(oc.synth_bin(many, k * per + b), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_beam_role_with_classes_is_the_adjoint_of_degridding():
    ob, base, spec, rt, co = _case(oc.ROLE_BEAM, S=12, W=7.0)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((ob.nvis, 4)) + 1j * rng.standard_normal((ob.nvis, 4))
    x = rng.standard_normal((4, spec.N, spec.N)) + 1j * rng.standard_normal((4, spec.N, spec.N))
    kb = oc.make_kernels(spec)
    kd = oc.make_kernels(oc.KernelSpec(**base, role=oc.ROLE_DEGRID))
    G, _, _ = oc.grid(kb, co, v)
    Dx = oc.degrid(kd, co, x)
    lhs, rhs = np.vdot(G, x), np.vdot(v, Dx)
    assert abs(lhs.real - rhs.real) < 1e-12 * abs(lhs)


def test_gridding_role_inverts_each_class_mueller_matrix():
    # image domain: grid function x degrid function = psi^4 (M^S')^-1 M^S,
    # the identity up to the Eq. 6 regularisation where the beam is strong
    _, base = small_case(npol=4, nw=1, S=16, OS=4, eps=1e-4)
    base = {**base, "type_leak": TYPE_LEAK}
    g = oc.KernelSpec(**base, role=oc.ROLE_GRID)
    d = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    M = g.image_size(0)
    t = oc.taper_samples(g.W, M)
    psi4 = (t[None, :] * t[:, None]) ** 2
    c = slice(M // 2 - 2, M // 2 + 3)
    for k in (0, 5, 7):
        fg = oc.cell_functions(g, 0, 0, 0, k).reshape(4, 4, M, M)      # [s][c]
        fd = oc.cell_functions(d, 0, 0, 0, k).reshape(4, 4, M, M)      # [c][s]
        prod = np.einsum("scyx,ctyx->styx", fg, fd)[:, :, c, c]
        eye = np.eye(4)[:, :, None, None] * psi4[None, None, c, c]
        assert np.abs(prod - eye).max() < 1e-3, k
        # and not another class's inverse
        fo = oc.cell_functions(d, 0, 0, 0, 1 if k != 1 else 2).reshape(4, 4, M, M)
        wrong = np.einsum("scyx,ctyx->styx", fg, fo)[:, :, c, c]
        assert np.abs(wrong - eye).max() > 1e-2


def test_per_channel_kernels_remove_the_frequency_averaging():
    # one beam-frequency bin per channel: degridding equals the direct Mueller
    # sum with each visibility's beam at its own channel frequency; the single
    # band-averaged bin does not
    ob, base = small_case(npol=4, W=9.0, S=16)
    per_chan = oc.KernelSpec(**{**base, "fbin_freqs": tuple(ob.freq)}, role=oc.ROLE_DEGRID)
    averaged = oc.KernelSpec(**base, role=oc.ROLE_DEGRID)
    fbin = np.arange(ob.freq.size, dtype=np.uint8)
    co = oc.coords(per_chan, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, fbin=fbin)
    co_avg = oc.coords(averaged, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    N, dl = per_chan.N, per_chan.dl
    rng = np.random.default_rng(6)
    qx = rng.integers(N // 2 - 20, N // 2 + 20, 4)
    qy = rng.integers(N // 2 - 20, N // 2 + 20, 4)
    lm = oc.pixel_lm(N, dl, qx, qy)
    stokes = np.stack([rng.uniform(0.5, 1, 4), rng.uniform(-0.2, 0.2, 4),
                       rng.uniform(-0.2, 0.2, 4), rng.uniform(-0.02, 0.02, 4)], 1)
    uq = quantised_uvw(per_chan, co)
    u_own = np.where(co.flip[:, None] == 1, -uq, uq)
    Vobs = np.zeros((ob.nvis, 4), np.complex128)
    for c, nu in enumerate(ob.freq):
        sel = ob.chan_of_vis == c
        J = oc.jones(lm[:, 0], lm[:, 1], nu, per_chan.pa[0], per_chan.dish_d, per_chan.d_xy, per_chan.d_yx)
        bright = np.einsum("pcs,ps->pc", oc.mueller_from_jones(J) @ oc.T_STOKES_TO_CORR, stokes)
        for k in range(4):
            Vobs[sel, k] = oc.dft_predict(u_own[sel], lm, bright[:, k])
    model = np.zeros((4, N, N))
    for s in range(4):
        np.add.at(model[s], (qy, qx), stokes[:, s])
    G = oc.image_to_grid(model, per_chan.W)
    err = np.abs(oc.degrid(oc.make_kernels(per_chan), co, G) - Vobs).max()
    err_avg = np.abs(oc.degrid(oc.make_kernels(averaged), co_avg, G) - Vobs).max()
    assert err < 1e-5 * np.abs(Vobs).max(), err
    assert err_avg > 20 * err, (err, err_avg)
