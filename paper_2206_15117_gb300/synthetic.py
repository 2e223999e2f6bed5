"""Seeded synthetic inputs shaped like the paper's ASKAP observations.

This module is the only thing the CUDA path and the FP64 oracle have in
common: it draws geometry and random numbers and holds none of the gridding
method's arithmetic.  The paper's measurement sets (ASKAP, ALMA; Sec. 2.1,
Sec. 2.3) are not available, so these arrays stand in for them:

* 36 antennas uniform in a disk of 1.5 km radius (ENU, flat), latitude
  -26.7 deg, phase centre at declination -45 deg;
* earth-rotation uvw in metres over hour angles -4 h .. +4 h, 630 baselines;
* channels, per-channel visibility subsets (flagging), parallactic angles;
* point-source sky models (flux U(0.1, 1) Jy) and complex Gaussian
  visibility values.

Every generator takes an explicit seed; the base seed is 2206_15117 plus the
configuration number.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

BASE_SEED = 2206_15117
C_LIGHT = 299792458.0
LAT_DEG = -26.7
DEC_DEG = -45.0


def antenna_enu(n_ant: int, radius_m: float, rng: np.random.Generator) -> np.ndarray:
    r = radius_m * np.sqrt(rng.random(n_ant))
    th = 2 * math.pi * rng.random(n_ant)
    return np.stack([r * np.cos(th), r * np.sin(th), np.zeros(n_ant)], axis=1)


def baselines_xyz(enu: np.ndarray, lat_rad: float) -> np.ndarray:
    """Baseline vectors (i < j) rotated from local ENU to equatorial XYZ."""
    i, j = np.triu_indices(enu.shape[0], k=1)
    d = enu[j] - enu[i]
    e, n, u = d[:, 0], d[:, 1], d[:, 2]
    X = -math.sin(lat_rad) * n + math.cos(lat_rad) * u
    Y = e
    Z = math.cos(lat_rad) * n + math.sin(lat_rad) * u
    return np.stack([X, Y, Z], axis=1)


def earth_rotation_uvw(bxyz: np.ndarray, ha_rad: np.ndarray, dec_rad: float) -> np.ndarray:
    """uvw [n_ha * n_bl][3] in metres, rows ordered time-major."""
    sH = np.sin(ha_rad)[:, None]
    cH = np.cos(ha_rad)[:, None]
    sd, cd = math.sin(dec_rad), math.cos(dec_rad)
    X, Y, Z = bxyz[:, 0][None, :], bxyz[:, 1][None, :], bxyz[:, 2][None, :]
    u = sH * X + cH * Y
    v = -sd * cH * X + sd * sH * Y + cd * Z
    w = cd * cH * X - cd * sH * Y + sd * Z
    return np.stack([u, v, w], axis=-1).reshape(-1, 3)


def parallactic_angle(ha_rad: np.ndarray, lat_rad: float, dec_rad: float) -> np.ndarray:
    return np.arctan2(np.sin(ha_rad) * math.cos(lat_rad),
                      math.sin(lat_rad) * math.cos(dec_rad)
                      - math.cos(lat_rad) * math.sin(dec_rad) * np.cos(ha_rad))


@dataclasses.dataclass
class Observation:
    """One synthetic observation (all arrays numpy, host)."""
    uvw: np.ndarray            # f64 [nrow][3] metres
    freq: np.ndarray           # f64 [nchan] Hz
    row_of_vis: np.ndarray     # u32 [nvis]
    chan_of_vis: np.ndarray    # u16 [nvis]
    pa_bin: np.ndarray         # u8 [nrow]
    fbin: np.ndarray           # u8 [nchan]
    pa_centres: np.ndarray     # f64 [npa] rad
    fbin_freqs: np.ndarray     # f64 [nfb] Hz
    w_max: float               # max |w| over all visibilities, wavelengths
    sources: np.ndarray        # f64 [nsrc][3]: l, m, flux (Jy)
    params: Dict

    @property
    def nvis(self) -> int:
        return int(self.row_of_vis.shape[0])


def mosaic_offsets(n_fields: int = 7, sep_deg: float = 1.0):
    """Hexagonal pointing offsets (east, north) in degrees: the centre and six
    neighbours at `sep_deg`."""
    out = [(0.0, 0.0)]
    for k in range(n_fields - 1):
        a = k * math.pi / 3.0
        out.append((sep_deg * math.cos(a), sep_deg * math.sin(a)))
    return out


def _common_array(rng, n_t: int, ha_hours: float = 4.0, offset_deg=(0.0, 0.0)):
    enu = antenna_enu(36, 1500.0, rng)
    lat = math.radians(LAT_DEG)
    dec = math.radians(DEC_DEG + offset_deg[1])
    # an eastward pointing offset shifts the hour angle by -offset / cos(dec)
    dha = -math.radians(offset_deg[0]) / math.cos(math.radians(DEC_DEG))
    ha = np.linspace(-ha_hours, ha_hours, n_t) * (math.pi / 12.0) + dha
    bxyz = baselines_xyz(enu, lat)
    uvw = earth_rotation_uvw(bxyz, ha, dec)
    pa_row = np.repeat(parallactic_angle(ha, lat, dec), bxyz.shape[0])
    return uvw, pa_row


def _sources(rng, n: int, half_width_deg: float) -> np.ndarray:
    hw = math.radians(half_width_deg)
    l = rng.uniform(-hw, hw, n)
    m = rng.uniform(-hw, hw, n)
    s = rng.uniform(0.1, 1.0, n)
    return np.stack([l, m, s], axis=1)


def _bins(values: np.ndarray, nbins: int):
    lo, hi = float(values.min()), float(values.max())
    width = (hi - lo) / nbins if hi > lo else 1.0
    idx = np.clip(np.floor((values - lo) / width), 0, nbins - 1).astype(np.uint8)
    centres = lo + (np.arange(nbins) + 0.5) * width
    return idx, centres


def _w_max(uvw: np.ndarray, freq: np.ndarray) -> float:
    return float(np.max(np.abs(uvw[:, 2])) * np.max(freq) / C_LIGHT) * (1.0 + 1e-9)


def observation(cfg: int, *, time_samples: Optional[int] = None, vis_fraction: float = 1.0,
                seed: Optional[int] = None, field: int = 0) -> Observation:
    """Geometry of configuration `cfg` (1, 2, 3 or 5).

    cfg 1: 200 time samples, one channel at 1.4 GHz (126,000 visibilities).
    cfg 2: 2000 time samples x 16 channels 1.2-1.5 GHz (20,160,000).
    cfg 3: 2000 time samples, 288 channels 1.200-1.487 GHz at 1 MHz, each
           channel keeps a random row subset of U[50k, 400k] rows (flagging);
           8 parallactic-angle bins, 4 beam-frequency bins.
    cfg 5: per field, config 2's array/band with 993 samples x 16 channels
           (10.0M visibilities), phase centre at the field's hexagonal offset.
    `vis_fraction` < 1 keeps a seeded random subset of the visibilities.
    """
    rng = np.random.default_rng(BASE_SEED + cfg if seed is None else seed)
    if cfg == 1:
        n_t = time_samples or 200
        uvw, pa_row = _common_array(rng, n_t)
        freq = np.array([1.4e9])
        nrow = uvw.shape[0]
        row = np.arange(nrow, dtype=np.uint32)
        chan = np.zeros(nrow, dtype=np.uint16)
        src = _sources(rng, 20, 0.5)
        npa, nfb = 1, 1
    elif cfg in (2, 5):
        n_t = time_samples or (2000 if cfg == 2 else 993)
        off = mosaic_offsets()[field] if cfg == 5 else (0.0, 0.0)
        uvw, pa_row = _common_array(rng, n_t, offset_deg=off)
        freq = np.linspace(1.2e9, 1.5e9, 16)
        nrow = uvw.shape[0]
        row = np.tile(np.arange(nrow, dtype=np.uint32), freq.size)
        chan = np.repeat(np.arange(freq.size, dtype=np.uint16), nrow)
        src = _sources(rng, 20, 1.5)
        npa, nfb = (1, 1) if cfg == 2 else (8, 4)
    elif cfg == 3:
        n_t = time_samples or 2000
        uvw, pa_row = _common_array(rng, n_t)
        freq = 1.200e9 + 1.0e6 * np.arange(288)
        nrow = uvw.shape[0]
        scale = nrow / 1_260_000.0
        counts = rng.integers(int(50_000 * scale), int(400_000 * scale) + 1, size=freq.size)
        rows: List[np.ndarray] = []
        chans: List[np.ndarray] = []
        for c, n_c in enumerate(counts):
            sel = np.sort(rng.choice(nrow, size=int(n_c), replace=False)).astype(np.uint32)
            rows.append(sel)
            chans.append(np.full(sel.size, c, dtype=np.uint16))
        row = np.concatenate(rows)
        chan = np.concatenate(chans)
        src = _sources(rng, 20, 1.5)
        npa, nfb = 8, 4
    else:
        raise ValueError("unknown configuration %r" % cfg)
    if vis_fraction < 1.0:
        keep = np.sort(rng.choice(row.size, size=max(1, int(round(row.size * vis_fraction))),
                                  replace=False))
        row, chan = row[keep], chan[keep]
    pa_bin, pa_centres = _bins(pa_row, npa)
    if nfb > 1:
        fb = (np.arange(freq.size) * nfb // freq.size).astype(np.uint8)
        fcent = np.array([freq[fb == b].mean() for b in range(nfb)])
    else:
        fb = np.zeros(freq.size, np.uint8)
        fcent = np.array([float(freq.mean())])
    return Observation(uvw=uvw, freq=freq, row_of_vis=row.astype(np.uint32),
                       chan_of_vis=chan.astype(np.uint16), pa_bin=pa_bin, fbin=fb,
                       pa_centres=pa_centres, fbin_freqs=fcent, w_max=_w_max(uvw, freq),
                       sources=src, params={"cfg": cfg, "n_t": n_t})


def random_vis(n: int, npol: int, sigma: float = 1.0, seed: int = BASE_SEED) -> np.ndarray:
    """Complex Gaussian visibility values, complex64 [n][npol]."""
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n, npol), dtype=np.float32)
    im = rng.standard_normal((n, npol), dtype=np.float32)
    return ((re + 1j * im) * np.float32(sigma)).astype(np.complex64)


def random_weights(n: int, npol: int, seed: int = BASE_SEED + 7) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.5, 1.5, (n, npol)).astype(np.float32)


def grid_geometry(cfg: int) -> Dict:
    """Grid size, cell and oversampling of configuration `cfg`."""
    if cfg == 1:
        return {"N": 512, "dl": math.radians(1.0) / 512, "OS": 4, "W": 7.0}
    if cfg in (2, 4, 5):
        return {"N": 2048, "dl": math.radians(3.0) / 2048, "OS": 8, "W": 7.0}
    if cfg == 3:
        return {"N": 4096, "dl": math.radians(3.0) / 4096, "OS": 8, "W": 7.0}
    raise ValueError(cfg)


# leakage of the configurations' feeds: 1 % with fixed phases
LEAK_XY, LEAK_YX = 0.01 * complex(math.cos(0.4), math.sin(0.4)), 0.01 * complex(math.cos(-1.3), math.sin(-1.3))


def config_spec(cfg: int, ob: "Observation") -> Dict:
    """Kernel-set arguments (the fields of aw_kernel_spec) of configuration
    `cfg` for its observation `ob`:
      1: Stokes I, no w or A term, 7-cell PSWF kernel, OS 4, 512^2;
      2, 4: Stokes I w-projection, 32 planes, supports 8..64, OS 8, 2048^2
         (4 is 2 with BF16 / FP16 tables: pass storage separately);
      3: full-pol AW, 32 planes, supports 16..72, the observation's PA and
         beam-frequency bins, 12 m Airy beam, 1 % leakage, eps 0.2, 4096^2;
      5: full-pol AW of one mosaic field, 32 planes, supports 8..64, 2048^2."""
    g = grid_geometry(cfg)
    base = dict(N=g["N"], dl=g["dl"], OS=g["OS"], W=g["W"])
    if cfg == 1:
        return dict(base, npol=1, nw=1, supports=[7])
    if cfg in (2, 4):
        return dict(base, npol=1, nw=32, w_max=ob.w_max, supports=w_supports(32))
    if cfg in (3, 5):
        return dict(base, npol=4, nw=32, w_max=ob.w_max, supports=w_supports(32, extra=8 if cfg == 3 else 0),
                    pa=list(ob.pa_centres), fbin_freqs=list(ob.fbin_freqs), dish_d=12.0, d_xy=LEAK_XY,
                    d_yx=LEAK_YX, eps=0.2)
    raise ValueError(cfg)


def w_supports(nw: int, extra: int = 0) -> List[int]:
    """Full kernel width per w plane: S_p = 8 max(1, round(8 w_p / w_max)) + extra,
    w_p = (p + 1/2) w_max / nw (8..64 cells for 32 planes; +8 for AW)."""
    out = []
    for p in range(nw):
        r = int(math.floor(8.0 * (p + 0.5) / nw + 0.5))
        out.append(8 * max(1, r) + extra)
    return out


def small_observation(n_ant: int = 8, radius_m: float = 40.0, n_t: int = 8,
                      freq=(1.4e9,), ha_hours: float = 4.0, seed: int = BASE_SEED + 100,
                      z_spread_m: float = 0.0, npa: int = 1, nfb: int = 1) -> Observation:
    """A tiny array for brute-force checks (uv extent of a few hundred
    wavelengths).  `z_spread_m` gives antennas random heights so that w is
    not tied to (u, v)."""
    rng = np.random.default_rng(seed)
    enu = antenna_enu(n_ant, radius_m, rng)
    if z_spread_m:
        enu[:, 2] = rng.uniform(-z_spread_m, z_spread_m, n_ant)
    lat = math.radians(LAT_DEG)
    dec = math.radians(DEC_DEG)
    ha = np.linspace(-ha_hours, ha_hours, n_t) * (math.pi / 12.0)
    bxyz = baselines_xyz(enu, lat)
    uvw = earth_rotation_uvw(bxyz, ha, dec)
    freq = np.asarray(freq, dtype=np.float64)
    nrow = uvw.shape[0]
    row = np.tile(np.arange(nrow, dtype=np.uint32), freq.size)
    chan = np.repeat(np.arange(freq.size, dtype=np.uint16), nrow)
    pa_row = np.repeat(parallactic_angle(ha, lat, dec), bxyz.shape[0])
    pa_bin, pa_centres = _bins(pa_row, npa)
    fb = (np.arange(freq.size) * nfb // max(freq.size, 1)).astype(np.uint8)
    fcent = np.array([freq[fb == b].mean() if np.any(fb == b) else freq.mean() for b in range(nfb)])
    return Observation(uvw=uvw, freq=freq, row_of_vis=row, chan_of_vis=chan, pa_bin=pa_bin,
                       fbin=fb, pa_centres=pa_centres, fbin_freqs=fcent, w_max=_w_max(uvw, freq),
                       sources=np.zeros((0, 3)), params={"n_t": n_t})


def row_antenna_types(n_ant: int, nrow: int, ant_type: np.ndarray) -> np.ndarray:
    """uint8 [nrow][2]: the types of the two antennas (i < j) of each row, for
    rows ordered time-major over the baselines of triu_indices(n_ant, 1)."""
    i, j = np.triu_indices(n_ant, k=1)
    bl = np.arange(nrow) % i.size
    t = np.asarray(ant_type, np.uint8)
    return np.stack([t[i[bl]], t[j[bl]]], axis=1)


def random_grid(npol: int, N: int, seed: int = BASE_SEED + 11, scale: float = 1.0) -> np.ndarray:
    """A complex64 uv grid [npol][N][N] of Gaussian values (a model grid)."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((npol, N, N), dtype=np.float32) + 1j * rng.standard_normal((npol, N, N), dtype=np.float32)
    return (g * np.float32(scale)).astype(np.complex64)
