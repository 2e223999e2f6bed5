"""Host sanitizers on the oracle's C part: coordinates, gridding, degridding
and the direct DFT run under AddressSanitizer and UndefinedBehaviorSanitizer
(errors fatal) in a child process, on small cases that include samples
outside the grid, flipped samples, flags, non-finite values and an empty set."""
import os
import subprocess
import sys
import textwrap

import pytest

from oracle import build as ob

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    try:
        p = subprocess.check_output(["gcc", "-print-file-name=" + name], text=True).strip()
    except (OSError, subprocess.CalledProcessError):
        return None
    return p if os.path.isabs(p) and os.path.exists(p) else None


SCRIPT = textwrap.dedent('''
    import math, sys
    import numpy as np
    sys.path.insert(0, %r)
    from oracle import core as oc
    from paper_2206_15117_gb300 import synthetic as sy
    ob = sy.small_observation(n_ant=8, radius_m=60.0, n_t=8, freq=(1.3e9, 1.4e9))
    for npol, N in ((1, 32), (4, 48)):
        spec = oc.KernelSpec(N=N, dl=math.radians(4.0) / N, OS=4, npol=npol, nw=3, w_max=ob.w_max,
                             supports=[6, 8, 10], dish_d=4.0, d_xy=0.01j, d_yx=-0.01j)
        flags = (np.arange(ob.nvis) %% 7 == 0).astype(np.uint8)
        co = oc.coords(spec, ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq, flags=flags)
        assert (co.valid == 0).any() and co.flip.any()
        rng = np.random.default_rng(0)
        v = rng.standard_normal((ob.nvis, npol)) + 1j * rng.standard_normal((ob.nvis, npol))
        v[3, 0] = np.nan
        ks = oc.make_kernels(spec)
        G, ws, nbad = oc.grid(ks, co, v)
        assert nbad >= 1
        kd = oc.make_kernels(oc.KernelSpec(**{**spec.__dict__, "role": oc.ROLE_DEGRID}))
        V = oc.degrid(kd, co, G)
        assert np.isfinite(V).all()
        # an empty visibility set
        e = np.zeros(0, np.uint32)
        co0 = oc.coords(spec, ob.uvw, e, e.astype(np.uint16), ob.freq)
        G0, ws0, _ = oc.grid(ks, co0, np.zeros((0, npol), complex))
        assert ws0 == 0 and not G0.any()
        assert oc.degrid(kd, co0, G).shape == (0, npol)
    lm = np.array([[0.001, -0.002], [0.0, 0.0]])
    uvwl = oc.uvw_lambda(ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq)
    D = oc.dft_predict(uvwl, lm, np.array([1.0, 0.5]) + 0j)
    A = oc.dft_adjoint(uvwl, D, lm)
    assert np.isfinite(A).all()
    assert oc._c()._name.endswith("_aw_oracle_san.so"), oc._c()._name
    print("sanitized oracle ok")
''') % ROOT


def test_oracle_c_code_under_asan_and_ubsan():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc sanitizer runtimes not installed")
    ob.build(sanitize=True)
    env = dict(os.environ, AW_ORACLE_SANITIZE="1", LD_PRELOAD=asan + " " + ubsan,
               ASAN_OPTIONS="detect_leaks=0:abort_on_error=0:exitcode=23",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1:exitcode=24")
    r = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "sanitized oracle ok" in r.stdout
    assert "AddressSanitizer" not in r.stderr and "runtime error" not in r.stderr, r.stderr[-4000:]
