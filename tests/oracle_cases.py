"""Small seeded cases shared by the oracle pin tests (host only)."""
import math

import numpy as np

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy


def small_case(npol=1, nw=8, S=12, W=7.0, OS=8, N=64, fov_deg=4.0, dish=4.0, leak=0.05,
               eps=0.2, n_t=24, chi=0.3):
    ob = sy.small_observation(n_ant=10, radius_m=35.0, n_t=n_t, freq=(1.3e9, 1.4e9))
    dl = math.radians(fov_deg) / N
    base = dict(N=N, dl=dl, OS=OS, W=W, npol=npol, nw=nw, w_max=ob.w_max if nw > 1 else 0.0,
                supports=[S] * nw, pa=(chi,), fbin_freqs=(1.35e9,), dish_d=dish,
                d_xy=leak * np.exp(0.7j), d_yx=leak * np.exp(-1.1j), eps=eps)
    return ob, base


def quantised_uvw(spec, co):
    """Visibility coordinates after the method's own quantisation: the
    oversampled uv position it was gridded at and the centre of its w plane."""
    du = 1.0 / (spec.N * spec.dl)
    p = spec.plane_of(co.bin)
    rho = (np.asarray(spec.supports)[p] - 2) * spec.OS // 2
    u = ((co.x0 * spec.OS + rho + co.fx) / spec.OS - spec.N // 2) * du
    v = ((co.y0 * spec.OS + rho + co.fy) / spec.OS - spec.N // 2) * du
    w = np.array([spec.w_centre(int(x)) for x in p])
    return np.stack([u, v, w], 1)


def all_pixels_lm(N, dl):
    qq = np.arange(N)
    QX, QY = np.meshgrid(qq, qq)
    return oc.pixel_lm(N, dl, QX.ravel(), QY.ravel())
