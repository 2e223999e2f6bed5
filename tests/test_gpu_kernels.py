"""GPU: kernel synthesis (aw_make_kernels, cuFFT in FP64 + the library's
Mueller/Eq. 6 kernels) against the oracle's direct DFT of the same image
functions; storage conversion to BF16/FP16."""
import numpy as np
import pytest
import torch

from oracle import core as oc
from tests.gpu_cases import case_fullpol, case_stokes_i_cfg1, case_wproj

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2206_15117_gb300 import aw
    return aw.aw_create(0)


def _export(ks, b, S, OS, P):
    from paper_2206_15117_gb300 import aw
    out = torch.empty(OS * OS * S * S * P, dtype=torch.complex64, device="cuda")
    aw.aw_kernel_set_export(ks, b, out)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(OS, OS, S, S, P)


@pytest.mark.parametrize("case,role", [("cfg1", 0), ("wproj", 0), ("wproj", 1),
                                       ("fullpol", 0), ("fullpol", 1), ("fullpol", 2)])
def test_synthesis_matches_oracle(ctx, case, role):
    from paper_2206_15117_gb300 import aw
    if case == "cfg1":
        ob, kw = case_stokes_i_cfg1(time_samples=2)
    elif case == "wproj":
        ob, kw = case_wproj(vis_fraction=1e-4, nw=8, N=512)
    else:
        ob, kw = case_fullpol()
    ks = aw.aw_make_kernels(ctx, **kw, role=role)
    info = aw.aw_kernel_set_info(ks)
    spec = oc.KernelSpec(**kw, role=role)
    assert info.nbins == spec.nbins
    P = spec.npol ** 2
    bins = range(spec.nbins) if spec.nbins <= 4 else [0, spec.nbins // 2, spec.nbins - 1]
    for b in bins:
        p = b // (spec.npa * spec.nfb)
        S = spec.supports[p]
        got = _export(ks, b, S, spec.OS, P)
        ref = oc.synth_bin(spec, b)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-6, (b, err)


@pytest.mark.parametrize("storage,tol", [(1, 2.0 ** -8), (2, 2.0 ** -11)])
def test_reduced_storage_rounds_the_fp32_tables(ctx, storage, tol):
    from paper_2206_15117_gb300 import aw
    ob, kw = case_wproj(vis_fraction=1e-4, nw=4, N=512)
    k32 = aw.aw_make_kernels(ctx, **kw)
    k16 = aw.aw_make_kernels(ctx, **kw, storage=storage)
    assert aw.aw_kernel_set_info(k16).bytes * 2 == aw.aw_kernel_set_info(k32).bytes
    S = kw["supports"][3]
    a = _export(k32, 3, S, kw["OS"], 1)
    b = _export(k16, 3, S, kw["OS"], 1)
    # each component rounded to nearest: |b - a| <= tol |a| (normal range), tiny values absolute
    for comp in (np.real, np.imag):
        d = np.abs(comp(b) - comp(a))
        assert np.all(d <= tol * np.abs(comp(a)) + 1e-6 * np.abs(a).max())
