"""Oracle of the cleaning loop: Cotton-Schwab major cycles (Sec. 2.1) around a
Hogbom minor cycle (named in Sec. 4), plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring): no product code imports
this module.

The paper names the algorithm and its controls (number of clean cycles, loop
gain, cycle factor, threshold) without writing them out; the steps below are
the textbook method with these readings:

* The minor cycle works on the Stokes I plane: the peak of |I| inside the clean
  window picks the pixel, and the component at that pixel is the loop gain
  times the residual of every Stokes plane there.  It is removed with a
  truncated point-spread function (a square patch of half-width h around the
  peak); the major cycle then recomputes the residual exactly from the
  visibilities, which is what makes the truncation harmless.
* Ties of |I| go to the lowest flat pixel index (row-major).  The minor cycle
  runs in FP32 with one rounding per multiply and per subtraction, so that a
  kernel doing the same FP32 operations makes the same argmax decisions.
* Point-spread function: the Stokes I image of unit Stokes I visibilities
  (XX = YY = 1, XY = YX = 0; or 1 for a single correlation) gridded with the
  same weights and kernels, divided by its value at the phase centre.
* Cycle threshold: max(threshold, cycle_factor * sidelobe * peak), with peak the
  largest |I| of the residual in the window at the start of the major cycle and
  sidelobe the largest |psf| outside the main lobe and within N/4 pixels of the
  centre on both axes (|dx|, |dy| < N/4).  The main lobe is the disk around the
  centre whose radius r0 is the first pixel distance x > 0 along +l with
  psf[c][c + x] <= 0 (c = N / 2).  The N/4 limit keeps the outer image out of
  the level: with A-projection the image of unit visibilities carries the
  inverse beam and the grid correction, which grow towards the edge.
* Major cycle k: residual image from the residual visibilities; stop when its
  peak is below the threshold; otherwise run the minor cycle, predict the model
  (image -> grid -> degrid) and subtract it from the observed visibilities.
"""
from __future__ import annotations

from typing import Dict, Optional, Sequence, Tuple

import numpy as np

from . import core


def default_window(N: int) -> Tuple[int, int, int, int]:
    """Inner half of the image (x0, y0, x1, y1), half-open."""
    return (N // 4, N // 4, 3 * N // 4, 3 * N // 4)


def psf_sidelobe(psf: np.ndarray) -> np.float32:
    """Largest |psf| outside the main lobe, |dx|, |dy| < N/4 (module docstring)."""
    psf = np.asarray(psf, dtype=np.float32)
    N = psf.shape[0]
    c = N // 2
    r0 = N // 2
    for x in range(1, N - c):
        if psf[c, c + x] <= 0:
            r0 = x
            break
    qy, qx = np.mgrid[0:N, 0:N]
    outside = ((qx - c) ** 2 + (qy - c) ** 2 > r0 * r0) & (np.abs(qx - c) < N // 4) & (np.abs(qy - c) < N // 4)
    if not outside.any():
        return np.float32(0.0)
    return np.float32(np.abs(psf[outside]).max())


def peak_abs(image_I: np.ndarray, window: Sequence[int]) -> np.float32:
    x0, y0, x1, y1 = window
    return np.float32(np.abs(np.asarray(image_I, np.float32)[y0:y1, x0:x1]).max())


def hogbom(residual: np.ndarray, psf: np.ndarray, gain: float, threshold: float, max_iter: int,
           patch_half: int, window: Sequence[int], model: Optional[np.ndarray] = None):
    """Hogbom minor cycle in FP32.  residual [npol][N][N], psf [N][N] with its
    peak at (N/2, N/2).  Returns (model, residual, iterations)."""
    R = np.array(residual, dtype=np.float32, copy=True)
    npol, N, _ = R.shape
    P = np.asarray(psf, dtype=np.float32)
    M = np.zeros_like(R) if model is None else np.array(model, dtype=np.float32, copy=True)
    g = np.float32(gain)
    thr = np.float32(threshold)
    h = int(patch_half)
    if not 0 <= h < N // 2:
        raise ValueError("patch_half must be in [0, N/2)")
    x0, y0, x1, y1 = window
    c = N // 2
    n = 0
    while n < max_iter:
        sub = np.abs(R[0, y0:y1, x0:x1])
        k = int(np.argmax(sub))                      # first maximum in row-major order
        py, px = y0 + k // (x1 - x0), x0 + k % (x1 - x0)
        if np.abs(R[0, py, px]) < thr:
            break
        comp = g * R[:, py, px]                      # FP32 products
        M[:, py, px] = M[:, py, px] + comp
        ya, yb = max(0, py - h), min(N, py + h + 1)
        xa, xb = max(0, px - h), min(N, px + h + 1)
        patch = P[c + ya - py:c + yb - py, c + xa - px:c + xb - px]
        R[:, ya:yb, xa:xb] = R[:, ya:yb, xa:xb] - comp[:, None, None] * patch[None]
        n += 1
    return M, R, n


def unit_stokes_i(nvis: int, npol: int) -> np.ndarray:
    u = np.zeros((nvis, npol), dtype=np.complex128)
    u[:, 0] = 1.0
    if npol == 4:
        u[:, 3] = 1.0
    return u


def point_spread_function(ks_grid, co, weight, W: float) -> Tuple[np.ndarray, float]:
    """Stokes I image of unit Stokes I visibilities, peak-normalised (FP32)."""
    npol = ks_grid.spec.npol
    N = ks_grid.spec.N
    G, ws, _ = core.grid(ks_grid, co, unit_stokes_i(co.x0.shape[0], npol), weight)
    img = core.fft_to_image(G, W, ws)[0]
    return (img / img[N // 2, N // 2]).astype(np.float32), ws


def clean(ks_grid, ks_degrid, co, vis: np.ndarray, weight: Optional[np.ndarray], W: float, n_major: int,
          max_minor: int, gain: float, threshold: float, cycle_factor: float, patch_half: int,
          window: Optional[Sequence[int]] = None) -> Dict:
    """Cotton-Schwab cleaning with FP64 transforms and the FP32 minor cycle."""
    npol = ks_grid.spec.npol
    N = ks_grid.spec.N
    win = tuple(window) if window is not None else default_window(N)
    vis = np.asarray(vis, dtype=np.complex128).reshape(-1, npol)
    psf, _ = point_spread_function(ks_grid, co, weight, W)
    side = psf_sidelobe(psf)
    model = np.zeros((npol, N, N), dtype=np.float32)
    res_vis = vis.copy()
    peaks, minors = [], []
    R = None
    done = 0
    for _ in range(n_major):
        G, ws, _ = core.grid(ks_grid, co, res_vis, weight)
        R = core.fft_to_image(G, W, ws).astype(np.float32)
        peak = peak_abs(R[0], win)
        peaks.append(float(peak))
        if peak < np.float32(threshold):
            break
        thr = max(np.float32(threshold), np.float32(cycle_factor) * side * peak)
        model, R, n = hogbom(R, psf, gain, thr, max_minor, patch_half, win, model)
        minors.append(n)
        done += 1
        pred = core.degrid(ks_degrid, co, core.image_to_grid(model.astype(np.float64), W))
        res_vis = vis - pred
    else:
        G, ws, _ = core.grid(ks_grid, co, res_vis, weight)
        R = core.fft_to_image(G, W, ws).astype(np.float32)
        peaks.append(float(peak_abs(R[0], win)))
    return {"model": model, "residual": R, "psf": psf, "sidelobe": float(side), "peaks": peaks,
            "minor": minors, "n_major": done, "residual_vis": res_vis}
