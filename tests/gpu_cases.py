"""Seeded cases for the GPU parity tests: each case is run through the C ABI
(libaw) and through the FP64 oracle on the same generator output."""
import math

import numpy as np

from oracle import core as oc
from paper_2206_15117_gb300 import synthetic as sy

# Tolerance for the FP32 path against the FP64 oracle (relative to the
# reference's L2 norm, and max-abs relative to its largest magnitude).
TOL_FP32 = 1e-5


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    l2 = np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)
    mx = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300) if b.size else 0.0
    return float(l2), float(mx)


def case_stokes_i_cfg1(time_samples=200):
    """Configuration 1 geometry (36 antennas, 1 channel, 512^2, 7x7 PSWF, OS 4)."""
    ob = sy.observation(1, time_samples=time_samples)
    return ob, sy.config_spec(1, ob)


def case_wproj(vis_fraction=0.002, nw=32, N=2048):
    """Configuration 2 geometry subset: 32 w planes, supports 8..64, OS 8."""
    ob = sy.observation(2, vis_fraction=vis_fraction)
    g = sy.grid_geometry(2)
    kw = dict(N=N, dl=g["dl"] * 2048 / N, OS=g["OS"], W=7.0, npol=1, nw=nw, w_max=ob.w_max,
              supports=sy.w_supports(nw))
    return ob, kw


def case_fullpol(N=256, nw=3, npa=2, nfb=2, n_t=40, n_ant=16, radius=180.0, supports=(16, 20, 24)):
    """Full-polarisation AW on a small grid: Airy beam, 1 % leakage, Eq. 6."""
    ob = sy.small_observation(n_ant=n_ant, radius_m=radius, n_t=n_t, freq=(1.2e9, 1.3e9, 1.4e9, 1.5e9),
                              npa=npa, nfb=nfb, seed=sy.BASE_SEED + 300)
    dl = math.radians(3.0) / N
    kw = dict(N=N, dl=dl, OS=8, W=7.0, npol=4, nw=nw, w_max=ob.w_max, supports=list(supports),
              pa=list(ob.pa_centres), fbin_freqs=list(ob.fbin_freqs), dish_d=12.0,
              d_xy=0.01 * np.exp(0.4j), d_yx=0.01 * np.exp(-1.3j), eps=0.2)
    return ob, kw


def oracle_spec(kw, role=oc.ROLE_GRID):
    return oc.KernelSpec(**kw, role=role)


def oracle_coords(ob, kw, flags=None):
    return oc.coords(oracle_spec(kw), ob.uvw, ob.row_of_vis, ob.chan_of_vis, ob.freq,
                     ob.pa_bin, ob.fbin, flags)


def used_bins(co):
    return sorted(set(int(b) for b in np.unique(co.bin[co.valid == 1])))
