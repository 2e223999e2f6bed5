"""FP64 oracle: the AW-projection gridding method of arXiv:2206.15117, plainly.

TEST INFRASTRUCTURE ONLY (see the package docstring): no product code imports
this module.

Conventions (the paper is silent on these; the readings are listed with the
design notes of the repository):

* Grid of N x N cells, image cell dl radians, field F = N * dl, uv cell
  du = 1 / F wavelengths.  Grid index g has u = (g - N/2) du; image index q has
  l = (q - N/2) dl.
* Degridding (model -> visibilities) uses exp(-2 pi i (u l + v m + w (n-1)));
  gridding is its adjoint (exp(+...)).  Eq. 2 prints the opposite sign; it
  only mirrors the image.
* Correlations in the order XX, XY, YX, YY; Stokes in the order I, Q, U, V.
* A kernel table for one bin is an array [OS][OS][S][S][P] of complex values,
  P = npol * npol, with Mueller index m = out * npol + in.  A visibility at
  oversampled coordinate Xi covers the S cells nearest to it, x0 .. x0 + S - 1,
  with x0 = floor((Xi - rho) / OS), rho = (S - 2) OS / 2, and fine offset
  fx = Xi - rho - x0 OS in [0, OS).  Tap jx lies d = jx OS - rho - fx
  oversampled units from the visibility (grid minus visibility); the table
  holds the uv kernel there.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np
import scipy.special

from . import build as _build

C_LIGHT = 299792458.0

# ----------------------------------------------------------------------------
# Prolate-spheroidal anti-aliasing taper (Sec. 3.2: kernels are "first
# multiplied in the image domain by an anti-aliasing function")
# ----------------------------------------------------------------------------


def pswf0_coefficients(c: float, nterms: int = 48) -> np.ndarray:
    """Legendre coefficients of the zeroth prolate spheroidal wave function.

    psi_0(x) = sum_k beta_k * Pbar_{2k}(x), Pbar_n = sqrt(n + 1/2) P_n, is the
    eigenvector of smallest eigenvalue of the operator
    -(1-x^2) d2/dx2 + 2x d/dx + c^2 x^2, which is tridiagonal in the even
    normalised Legendre basis (x^2 Pbar_n expands into Pbar_{n-2}, Pbar_n,
    Pbar_{n+2}).  Pinned against scipy.special.pro_ang1 and against the finite
    Fourier transform eigen-equation in the tests.
    """
    n = 2 * np.arange(nterms, dtype=np.float64)
    diag = n * (n + 1) + c * c * (2 * n * (n + 1) - 1) / ((2 * n + 3) * (2 * n - 1))
    nn = n[:-1]
    off = c * c * (nn + 2) * (nn + 1) / ((2 * nn + 3) * np.sqrt((2 * nn + 1) * (2 * nn + 5)))
    A = np.diag(diag) + np.diag(off, 1) + np.diag(off, -1)
    evals, evecs = np.linalg.eigh(A)
    beta = evecs[:, 0]
    # psi_0(0) > 0
    p0 = legendre_even_at_zero(nterms)
    if float(np.dot(beta, p0)) < 0:
        beta = -beta
    return beta


def legendre_even_at_zero(nterms: int) -> np.ndarray:
    """Pbar_{2k}(0) = sqrt(2k + 1/2) * P_{2k}(0)."""
    out = np.empty(nterms)
    for k in range(nterms):
        out[k] = math.sqrt(2 * k + 0.5) * scipy.special.eval_legendre(2 * k, 0.0)
    return out


def pswf0(c: float, x: np.ndarray, nterms: int = 48) -> np.ndarray:
    """psi_0(c, x) for |x| <= 1, normalised so psi_0(0) = 1."""
    beta = pswf0_coefficients(c, nterms)
    x = np.asarray(x, dtype=np.float64)
    val = np.zeros_like(x)
    for k in range(nterms):
        val = val + beta[k] * math.sqrt(2 * k + 0.5) * scipy.special.eval_legendre(2 * k, x)
    v0 = float(np.dot(beta, legendre_even_at_zero(nterms)))
    return val / v0


def taper_1d(W: float, x: np.ndarray) -> np.ndarray:
    """Image-domain taper psi(x), x = 2 l / F in [-1, 1): the PSWF with
    c = pi W / 2, whose uv transform is concentrated on W cells."""
    return pswf0(math.pi * W / 2.0, x)


def taper_samples(W: float, M: int) -> np.ndarray:
    """Taper on the M image samples l_p = (p - M/2) F / M, p in [0, M).

    The sample at p = 0 (l = -F/2, the Nyquist edge) is set to zero so that
    the sampled function is symmetric about l = 0 (reading of the paper).
    """
    p = np.arange(M)
    x = (p - M // 2) * 2.0 / M
    t = taper_1d(W, x)
    t[0] = 0.0
    return t


def grid_correction_1d(W: float, N: int) -> np.ndarray:
    """Grid correction c(q) = psi(2 l_q / F) at image pixels q, psi(0) = 1.

    Pixel q = 0 (l = -F/2) gets 0 and is written as 0 in the image."""
    q = np.arange(N)
    x = (q - N // 2) * 2.0 / N
    c = taper_1d(W, x)
    c[0] = 0.0
    return c


# ----------------------------------------------------------------------------
# Beam, Jones and Mueller matrices (Sec. 3.2, Eq. 2-5) and Eq. 6
# ----------------------------------------------------------------------------

# Eq. 4 with the U row read as (XY + YX) / 2: correlation vector -> Stokes
T_CORR_TO_STOKES = np.array([
    [0.5, 0.0, 0.0, 0.5],
    [0.5, 0.0, 0.0, -0.5],
    [0.0, 0.5, 0.5, 0.0],
    [0.0, -0.5j, 0.5j, 0.0],
], dtype=np.complex128)

# Inverse of the above: XX = I + Q, XY = U + iV, YX = U - iV, YY = I - Q
T_STOKES_TO_CORR = np.array([
    [1.0, 1.0, 0.0, 0.0],
    [0.0, 0.0, 1.0, 1.0j],
    [0.0, 0.0, 1.0, -1.0j],
    [1.0, -1.0, 0.0, 0.0],
], dtype=np.complex128)


def airy_voltage(l: np.ndarray, m: np.ndarray, freq_hz: float, dish_d: float) -> np.ndarray:
    """Airy-disk voltage pattern E = 2 J1(x) / x, x = pi D sin(r) / lambda,
    sin(r) = sqrt(l^2 + m^2) (a rotationally symmetric beam, Sec. 3.1)."""
    lam = C_LIGHT / freq_hz
    x = math.pi * dish_d * np.sqrt(l * l + m * m) / lam
    out = np.ones_like(x)
    nz = x != 0.0
    out[nz] = 2.0 * scipy.special.j1(x[nz]) / x[nz]
    return out


def jones(l: np.ndarray, m: np.ndarray, freq_hz: float, chi: float, dish_d: float,
          d_xy: complex, d_yx: complex) -> np.ndarray:
    """Antenna Jones matrix J = E(l, m) * [[1, d_xy], [d_yx, 1]] * R(chi).

    Shape (..., 2, 2).  R(chi) rotates the feeds by the parallactic angle."""
    E = airy_voltage(l, m, freq_hz, dish_d)
    D = np.array([[1.0, d_xy], [d_yx, 1.0]], dtype=np.complex128)
    R = np.array([[math.cos(chi), -math.sin(chi)], [math.sin(chi), math.cos(chi)]])
    DR = D @ R
    return E[..., None, None] * DR


def mueller_from_jones(J: np.ndarray, J2: Optional[np.ndarray] = None) -> np.ndarray:
    """M = J kron conj(J2) (Eq. 2-3 text; the conjugate on the second factor
    is the reading for correlations <e_a e_b*>): the Mueller matrix of a
    baseline whose first antenna has Jones matrix J and second J2 (J2 = J when
    omitted: identical antennas).  Shape (..., 4, 4)."""
    if J2 is None:
        J2 = J
    a = J[..., :, None, :, None]
    b = np.conj(J2)[..., None, :, None, :]
    M = a * b  # (..., 2, 2, 2, 2) indices (a, b, c, d)
    return M.reshape(J.shape[:-2] + (4, 4))


def mueller_stokes(M: np.ndarray) -> np.ndarray:
    """Eq. 5: M^S = T M T^-1 (Stokes-basis Mueller matrix)."""
    return T_CORR_TO_STOKES @ M @ T_STOKES_TO_CORR


def regularise_beam(B: np.ndarray, eps: float, Bmax: Optional[float] = None) -> np.ndarray:
    """Eq. 6: B' = B / |B| * (|B| + beta / |B|), beta = ((eps/2) * max|B|)^2.

    |B| below 1e-12 * max|B| is clamped to that value with phase 0 (reading
    for the null itself, where B / |B| is undefined)."""
    B = np.asarray(B)
    absB = np.abs(B)
    if Bmax is None:
        Bmax = float(absB.max())
    beta = ((eps / 2.0) * Bmax) ** 2
    floor = 1e-12 * Bmax
    small = absB < floor
    a = np.where(small, floor, absB)
    phase = np.where(small, 1.0 + 0j, B / np.where(small, 1.0, absB))
    return phase * (a + beta / a)


def invert4(A: np.ndarray) -> np.ndarray:
    """Per-pixel 4x4 complex inverse by Gauss-Jordan elimination with partial
    pivoting, written out (pinned against numpy.linalg.inv in the tests)."""
    A = np.array(A, dtype=np.complex128)
    shp = A.shape[:-2]
    A = A.reshape(-1, 4, 4)
    n = A.shape[0]
    aug = np.concatenate([A, np.broadcast_to(np.eye(4, dtype=np.complex128), (n, 4, 4))], axis=2).copy()
    idx = np.arange(n)
    for col in range(4):
        piv = col + np.argmax(np.abs(aug[:, col:, col]), axis=1)
        rows = aug[idx, piv].copy()
        aug[idx, piv] = aug[:, col]
        aug[:, col] = rows
        aug[:, col] = aug[:, col] / aug[:, col, col][:, None]
        for r in range(4):
            if r == col:
                continue
            f = aug[:, r, col][:, None]
            aug[:, r] = aug[:, r] - f * aug[:, col]
    return aug[:, :, 4:].reshape(shp + (4, 4))


# ----------------------------------------------------------------------------
# Kernel sets (Sec. 3.2: kernels are the FFT of the Mueller cells after the
# anti-aliasing function and the w term; Sec. 3.3 for the gridding copy)
# ----------------------------------------------------------------------------

ROLE_GRID, ROLE_DEGRID, ROLE_ADJOINT, ROLE_BEAM = 0, 1, 2, 3


@dataclasses.dataclass
class KernelSpec:
    N: int                      # grid side
    dl: float                   # image cell, radians
    OS: int                     # oversampling
    W: float = 7.0              # taper (PSWF) support in cells
    npol: int = 1               # 1: Stokes I, no A term; 4: full-pol AW
    nw: int = 1                 # number of w planes (1: w term off)
    w_max: float = 0.0          # |w| range covered by the planes, wavelengths
    supports: Sequence[int] = (7,)        # full kernel width per w plane
    pa: Sequence[float] = (0.0,)          # parallactic-angle bin centres, rad
    fbin_freqs: Sequence[float] = (1.4e9,)  # beam-frequency bin centres, Hz
    dish_d: float = 12.0
    d_xy: complex = 0.0
    d_yx: complex = 0.0
    eps: float = 0.2
    role: int = ROLE_GRID
    # pointing of the antennas relative to the image phase centre (direction
    # cosines): the beam is evaluated at (l - point_l, m - point_m)
    point_l: float = 0.0
    point_m: float = 0.0
    # per-baseline Mueller kernels: leakage (d_xy, d_yx) of each antenna type;
    # with two or more types every ordered type pair (ti, tj) is a baseline
    # class with its own kernels, M = J_ti kron conj(J_tj).  Empty: every
    # antenna has (d_xy, d_yx) and the kernels are baseline-averaged.
    type_leak: Sequence = ()

    @property
    def npa(self) -> int:
        return len(self.pa)

    @property
    def nfb(self) -> int:
        return len(self.fbin_freqs)

    @property
    def ntype(self) -> int:
        return len(self.type_leak)

    @property
    def nclass(self) -> int:
        return self.ntype * self.ntype if self.ntype >= 2 else 1

    @property
    def nbins(self) -> int:
        return self.nclass * self.nw * self.npa * self.nfb

    def decode_bin(self, b: int):
        """(class k, w plane p, PA bin a, frequency bin f) of bin
        b = ((k nw + p) npa + a) nfb + f."""
        f = b % self.nfb
        a = (b // self.nfb) % self.npa
        p = (b // (self.nfb * self.npa)) % self.nw
        k = b // (self.nfb * self.npa * self.nw)
        return k, p, a, f

    def plane_of(self, b):
        return (np.asarray(b) // (self.npa * self.nfb)) % self.nw

    def leakages(self, k: int):
        """((d_xy, d_yx) of the first antenna, (d_xy, d_yx) of the second) of
        baseline class k = ti * ntype + tj."""
        if self.nclass == 1:
            return (self.d_xy, self.d_yx), (self.d_xy, self.d_yx)
        ti, tj = divmod(k, self.ntype)
        return tuple(self.type_leak[ti]), tuple(self.type_leak[tj])

    def w_centre(self, p: int) -> float:
        if self.nw <= 1:
            return 0.0
        return (p + 0.5) * self.w_max / self.nw

    def image_size(self, p: int) -> int:
        """M for w plane p: the smallest power of two >= 2 S_p (and >= 16)."""
        S = int(self.supports[p])
        M = 16
        while M < 2 * S:
            M *= 2
        return M

    def bin_index(self, p: int, a: int, f: int) -> int:
        return (p * self.npa + a) * self.nfb + f


def image_coords(spec: KernelSpec, M: int):
    F = spec.N * spec.dl
    p = np.arange(M)
    l1 = (p - M // 2) * F / M
    return l1


def cell_functions(spec: KernelSpec, p: int, a: int, f: int, k: int = 0) -> np.ndarray:
    """Image-domain functions [P][M][M] whose uv transforms are the kernels.

    grid:    f_{s,c} = psi psi * exp(+2 pi i w (n-1)) * ((M^S)'^-1 T)_{s,c}
    degrid:  f_{c,s} = psi psi * exp(-2 pi i w (n-1)) * (M T^-1)_{c,s}
    adjoint: f_{c,s} = conj(grid f_{s,c})
    beam:    f_{s,c} = conj(degrid f_{c,s}): gridding weighted by the beam (the
             exact adjoint of degridding; UV-domain mosaics, Sec. 2.2)
    npol == 1 has no A term: the Mueller factor is 1.
    (M^S)' is M^S with its diagonal regularised by Eq. 6.  The beam is the
    Jones matrix at (l - point_l, m - point_m); M = J_i kron conj(J_j) with the
    two antennas' leakages of baseline class k.
    """
    M = spec.image_size(p)
    l1 = image_coords(spec, M)
    L = l1[None, :]
    Mm = l1[:, None]
    l = np.broadcast_to(L, (M, M))
    m = np.broadcast_to(Mm, (M, M))
    t = taper_samples(spec.W, M)
    psi2 = t[None, :] * t[:, None]
    n = np.sqrt(1.0 - l * l - m * m)
    w = spec.w_centre(p)
    wphase = np.exp(2j * math.pi * w * (n - 1.0))  # gridding sign
    role = spec.role
    if spec.npol == 1:
        if role in (ROLE_GRID, ROLE_BEAM):
            return (psi2 * wphase)[None]
        return np.conj(psi2 * wphase)[None]
    (dxy_i, dyx_i), (dxy_j, dyx_j) = spec.leakages(k)
    Ji = jones(l - spec.point_l, m - spec.point_m, spec.fbin_freqs[f], spec.pa[a], spec.dish_d, dxy_i, dyx_i)
    Jj = jones(l - spec.point_l, m - spec.point_m, spec.fbin_freqs[f], spec.pa[a], spec.dish_d, dxy_j, dyx_j)
    Mu = mueller_from_jones(Ji, Jj)
    if role in (ROLE_DEGRID, ROLE_BEAM):
        A = Mu @ T_STOKES_TO_CORR                           # [M][M][c][s]
        fn = (psi2 * np.conj(wphase))[..., None, None] * A
        if role == ROLE_BEAM:
            fn = np.conj(np.swapaxes(fn, -1, -2))           # [s][c] = conj(degrid[c][s])
        return np.moveaxis(fn.reshape(M, M, 16), -1, 0)
    MS = mueller_stokes(Mu)
    MSr = MS.copy()
    for q in range(4):
        MSr[..., q, q] = regularise_beam(MS[..., q, q], spec.eps)
    Ginv = invert4(MSr) @ T_CORR_TO_STOKES                  # [M][M][s][c]
    fn = (psi2 * wphase)[..., None, None] * Ginv
    if role == ROLE_GRID:
        return np.moveaxis(fn.reshape(M, M, 16), -1, 0)
    adj = np.conj(np.swapaxes(fn, -1, -2))                  # [c][s] = conj(grid[s][c])
    return np.moveaxis(adj.reshape(M, M, 16), -1, 0)


def _dft_rows(M: int, OS: int, S: int, sign: float, offsets: Sequence[int]) -> np.ndarray:
    """1-D DFT rows for uv samples k = j OS - rho - o (rho = (S - 2) OS / 2) of
    an image sampled on M points l_p = (p - M/2) F / M, zero-padded to M OS:
    E[(o, j), p] = exp(sign 2 pi i k (p - M/2) / (M OS))."""
    rho = (S - 2) * OS // 2
    p = np.arange(M) - M // 2
    rows = []
    for o in offsets:
        k = np.arange(S) * OS - rho - o
        rows.append(np.exp(sign * 2j * math.pi * np.outer(k, p) / (M * OS)))
    return np.concatenate(rows, axis=0)


def synth_bin(spec: KernelSpec, b: int, offsets_y: Optional[Sequence[int]] = None,
              offsets_x: Optional[Sequence[int]] = None) -> np.ndarray:
    """Kernel table of bin b: [len(oy)][len(ox)][S][S][P] complex128.

    K(ky, kx) = (1/M^2) sum_{q,p} f[q][p] exp(sign 2 pi i (ky (q-M/2) + kx (p-M/2)) / (M OS))
    with sign = -1 for the gridding and beam roles and +1 for degrid/adjoint: the DFT of
    the zero-padded image function evaluated at the uv samples the table needs.
    The 1/M^2 (with psi(0) = 1) makes the untruncated zero-offset taper kernel
    sum to one over integer cells (Poisson summation of the M-point DFT).
    """
    k, p, a, f = spec.decode_bin(b)
    S = int(spec.supports[p])
    M = spec.image_size(p)
    OS = spec.OS
    oy = list(range(OS)) if offsets_y is None else list(offsets_y)
    ox = list(range(OS)) if offsets_x is None else list(offsets_x)
    sign = -1.0 if spec.role in (ROLE_GRID, ROLE_BEAM) else 1.0
    fn = cell_functions(spec, p, a, f, k)              # [P][M][M] (q = y, p = x)
    Ey = _dft_rows(M, OS, S, sign, oy)                 # [(oy, jy)][q]
    Ex = _dft_rows(M, OS, S, sign, ox)                 # [(ox, jx)][p]
    P = fn.shape[0]
    out = np.empty((len(oy), len(ox), S, S, P), dtype=np.complex128)
    for mi in range(P):
        K = Ey @ fn[mi] @ Ex.T / (M * M)               # [(oy, jy)][(ox, jx)]
        K = K.reshape(len(oy), S, len(ox), S).transpose(0, 2, 1, 3)
        out[..., mi] = K
    return out


@dataclasses.dataclass
class KernelSet:
    spec: KernelSpec
    table: np.ndarray          # flat complex128
    offsets: np.ndarray        # int64[nbins], element offset of each bin
    bin_support: np.ndarray    # int32[nbins]


def make_kernels(spec: KernelSpec, bins: Optional[Sequence[int]] = None) -> KernelSet:
    """Synthesise the tables of all bins (or of `bins` only; the others are
    left empty with support kept, which is enough for visibilities that fall
    in the synthesised bins)."""
    nb = spec.nbins
    want = set(range(nb)) if bins is None else set(int(x) for x in bins)
    offs = np.zeros(nb, dtype=np.int64)
    sup = np.zeros(nb, dtype=np.int32)
    chunks = []
    pos = 0
    P = spec.npol * spec.npol
    for b in range(nb):
        S = int(spec.supports[spec.plane_of(b)])
        sup[b] = S
        offs[b] = pos
        if b in want:
            t = synth_bin(spec, b).reshape(-1)
            assert t.size == spec.OS * spec.OS * S * S * P
            chunks.append(t)
            pos += t.size
    table = np.concatenate(chunks) if chunks else np.zeros(0, np.complex128)
    return KernelSet(spec, table, offs, sup)


# ----------------------------------------------------------------------------
# uv grid -> image (Sec. 2.2: FFT; grid correction for the taper)
# ----------------------------------------------------------------------------


def fft_to_image(grid: np.ndarray, W: float, weight_sum: float) -> np.ndarray:
    """Dirty image planes from uv grid planes [npol][N][N].

    I(q) = sum_g G(g) exp(+2 pi i (g - N/2)(q - N/2) / N) (2-D), divided by the
    grid correction c(qx) c(qy) and by the weight sum; real part (Stokes planes
    are real).  Row or column q = 0 is written as 0."""
    grid = np.asarray(grid, dtype=np.complex128)
    npol, N, _ = grid.shape
    c = grid_correction_1d(W, N)
    corr = c[:, None] * c[None, :]
    out = np.zeros((npol, N, N), dtype=np.float64)
    safe = np.where(corr == 0.0, 1.0, corr)
    for s in range(npol):
        img = np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(grid[s]))) * (N * N)
        val = img.real / safe / weight_sum
        val[corr == 0.0] = 0.0
        out[s] = val
    return out


def image_to_grid(image: np.ndarray, W: float) -> np.ndarray:
    """Model image planes [npol][N][N] -> uv grid for degridding: divide by
    the grid correction, then G(g) = sum_q I(q) exp(-2 pi i (g-N/2)(q-N/2)/N)."""
    image = np.asarray(image, dtype=np.complex128)
    npol, N, _ = image.shape
    c = grid_correction_1d(W, N)
    corr = c[:, None] * c[None, :]
    safe = np.where(corr == 0.0, 1.0, corr)
    out = np.empty_like(image)
    for s in range(npol):
        x = np.where(corr == 0.0, 0.0, image[s] / safe)
        out[s] = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(x)))
    return out


# ----------------------------------------------------------------------------
# Mosaic weighting (Sec. 2.2, Eq. 1)
# ----------------------------------------------------------------------------


def mosaic_gamma(beams: np.ndarray, eps: float) -> np.ndarray:
    """gamma = [sqrt(sum B_i^2) / max sqrt(sum B_i^2)]_pbp * [1 / sum B_i^2]_wc,
    set to 0 where the normalised pattern (pbp) is below eps (the image mask)."""
    B = np.asarray(beams, dtype=np.float64)
    sumsq = np.sum(B * B, axis=0)
    root = np.sqrt(sumsq)
    pbp = root / np.max(root)
    with np.errstate(divide="ignore", invalid="ignore"):
        wc = 1.0 / sumsq
        gamma = pbp * wc
    gamma[pbp < eps] = 0.0
    return gamma


# ----------------------------------------------------------------------------
# C loops (coordinates, grid, degrid, direct DFT)
# ----------------------------------------------------------------------------

_lib = None


def _c():
    global _lib
    if _lib is None:
        import os
        _lib = ctypes.CDLL(_build.build(sanitize=os.environ.get("AW_ORACLE_SANITIZE") == "1"))
        P = ctypes.c_void_p
        i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        _lib.oracle_coords.argtypes = [i64, P, P, P, P, P, P, P, i32, dbl, i32, i32, dbl,
                                       i32, i32, P, P, P, P, P, P, P, P]
        _lib.oracle_coords.restype = None
        _lib.oracle_grid.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P, P, P, i32, i32, P, P]
        _lib.oracle_grid.restype = i64
        _lib.oracle_degrid.argtypes = [i64, i32, P, P, P, P, P, P, P, P, P, P, P, i32, i32, P]
        _lib.oracle_degrid.restype = None
        _lib.oracle_dft_predict.argtypes = [i64, P, i64, P, P, P]
        _lib.oracle_dft_predict.restype = None
        _lib.oracle_dft_adjoint.argtypes = [i64, P, P, i64, P, P]
        _lib.oracle_dft_adjoint.restype = None
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


@dataclasses.dataclass
class Coords:
    x0: np.ndarray      # first footprint cell along u
    y0: np.ndarray      # first footprint cell along v
    fx: np.ndarray      # fine (oversample) offset along u, [0, OS)
    fy: np.ndarray
    bin: np.ndarray
    flip: np.ndarray
    valid: np.ndarray


def coords(spec: KernelSpec, uvw: np.ndarray, row_of_vis: np.ndarray, chan_of_vis: np.ndarray,
           freq: np.ndarray, pa_bin: Optional[np.ndarray] = None,
           fbin: Optional[np.ndarray] = None, flags: Optional[np.ndarray] = None,
           row_types: Optional[np.ndarray] = None) -> Coords:
    """Per-visibility integer coordinates (see oracle_coords in aw_oracle.c).

    With per-baseline kernels (spec.ntype >= 2) row_types [nrow][2] gives the
    types of each row's two antennas (None: type 0 for both; types past the
    last count as the last).  A visibility flipped to w >= 0 is the reversed
    baseline, V_ji = P conj(V_ij) at -uvw, so its class takes the two types in
    swapped order."""
    nvis = int(row_of_vis.shape[0])
    uvw = np.ascontiguousarray(uvw, dtype=np.float64)
    row = np.ascontiguousarray(row_of_vis, dtype=np.uint32)
    chan = np.ascontiguousarray(chan_of_vis, dtype=np.uint16)
    freq = np.ascontiguousarray(freq, dtype=np.float64)
    pa_bin = None if pa_bin is None else np.ascontiguousarray(pa_bin, dtype=np.uint8)
    fbin = None if fbin is None else np.ascontiguousarray(fbin, dtype=np.uint8)
    flags = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    sup = np.ascontiguousarray(spec.supports, dtype=np.int32)
    out = [np.empty(nvis, np.int32) for _ in range(5)] + [np.empty(nvis, np.uint8) for _ in range(2)]
    _c().oracle_coords(nvis, _ptr(uvw), _ptr(row), _ptr(chan), _ptr(freq), _ptr(pa_bin),
                       _ptr(fbin), _ptr(flags), spec.N, spec.dl, spec.OS, spec.nw, spec.w_max,
                       spec.npa, spec.nfb, _ptr(sup), *[_ptr(a) for a in out])
    co = Coords(*out)
    if spec.nclass > 1 and row_types is not None:
        rt = np.minimum(np.asarray(row_types, np.int64).reshape(-1, 2), spec.ntype - 1)[row]
        ti = np.where(co.flip == 1, rt[:, 1], rt[:, 0])
        tj = np.where(co.flip == 1, rt[:, 0], rt[:, 1])
        co.bin = (co.bin + (ti * spec.ntype + tj) * (spec.nw * spec.npa * spec.nfb)).astype(np.int32)
    return co


def grid(ks: KernelSet, co: Coords, vis: np.ndarray, weight: Optional[np.ndarray] = None):
    """Gridding in FP64.  vis complex [nvis][npol] (or [nvis]); returns
    (grid complex128 [npol][N][N], weight_sum, n_nonfinite)."""
    spec = ks.spec
    npol = spec.npol
    v = np.ascontiguousarray(np.asarray(vis, dtype=np.complex128).reshape(-1, npol))
    w = None if weight is None else np.ascontiguousarray(np.asarray(weight, np.float64).reshape(-1, npol))
    G = np.zeros((npol, spec.N, spec.N), dtype=np.complex128)
    ws = ctypes.c_double(0.0)
    tab = np.ascontiguousarray(ks.table)
    nbad = _c().oracle_grid(v.shape[0], npol, _ptr(v), _ptr(w), _ptr(co.x0), _ptr(co.y0),
                            _ptr(co.fx), _ptr(co.fy), _ptr(co.bin), _ptr(co.flip), _ptr(co.valid),
                            _ptr(tab), _ptr(ks.offsets), _ptr(ks.bin_support), spec.OS, spec.N,
                            _ptr(G), ctypes.addressof(ws))
    return G, ws.value, int(nbad)


def degrid(ks: KernelSet, co: Coords, G: np.ndarray) -> np.ndarray:
    """Degridding in FP64: returns complex128 [nvis][npol]."""
    spec = ks.spec
    npol = spec.npol
    G = np.ascontiguousarray(np.asarray(G, dtype=np.complex128))
    nvis = co.x0.shape[0]
    out = np.empty((nvis, npol), dtype=np.complex128)
    tab = np.ascontiguousarray(ks.table)
    _c().oracle_degrid(nvis, npol, _ptr(G), _ptr(co.x0), _ptr(co.y0), _ptr(co.fx), _ptr(co.fy),
                       _ptr(co.bin), _ptr(co.flip), _ptr(co.valid), _ptr(tab), _ptr(ks.offsets),
                       _ptr(ks.bin_support), spec.OS, spec.N, _ptr(out))
    return out


def frame_axes(ra0: float, dec0: float) -> np.ndarray:
    """Rows: the unit vectors (east, north, towards the phase centre) of the
    frame about (ra0, dec0), in equatorial coordinates."""
    sa, ca, sd, cd = math.sin(ra0), math.cos(ra0), math.sin(dec0), math.cos(dec0)
    return np.array([[-sa, ca, 0.0], [-sd * ca, -sd * sa, cd], [cd * ca, cd * sa, sd]])


def phase_rotate(uvw: np.ndarray, row_of_vis: np.ndarray, chan_of_vis: np.ndarray, freq: np.ndarray,
                 vis: np.ndarray, src_centre, dst_centre):
    """Move visibilities from phase centre src_centre = (ra, dec) to dst_centre.

    The baseline b (metres) is unchanged; its components in the frame of the new
    centre are uvw' = B_dst B_src^T uvw.  With the degridding convention
    V = sum I exp(-2 pi i (u l + v m + w (n - 1))) = exp(2 pi i w) sum I exp(-2 pi i b.s / lambda),
    the visibility about the new centre is V' = V exp(2 pi i (w' - w) nu / c).
    Returns (uvw' [nrow][3], vis' [nvis][npol])."""
    R = frame_axes(*dst_centre) @ frame_axes(*src_centre).T
    uvw = np.asarray(uvw, np.float64)
    uvw2 = uvw @ R.T
    dw = (uvw2[:, 2] - uvw[:, 2])[np.asarray(row_of_vis, np.int64)]
    lam_inv = np.asarray(freq, np.float64)[np.asarray(chan_of_vis, np.int64)] / C_LIGHT
    ph = np.exp(2j * math.pi * dw * lam_inv)
    v = np.asarray(vis, np.complex128)
    return uvw2, v * (ph[:, None] if v.ndim == 2 else ph)


def uvw_lambda(uvw: np.ndarray, row_of_vis: np.ndarray, chan_of_vis: np.ndarray,
               freq: np.ndarray) -> np.ndarray:
    """Baselines in wavelengths per visibility (Eq. 2), no flip."""
    f = np.asarray(freq, np.float64)[chan_of_vis] / C_LIGHT
    return np.asarray(uvw, np.float64)[row_of_vis] * f[:, None]


def dft_predict(uvwl: np.ndarray, lm: np.ndarray, I: np.ndarray) -> np.ndarray:
    """Eq. 2 evaluated directly for pixels/sources at (l, m) with complex
    brightness I: V_k = sum_p I_p exp(-2 pi i (u l + v m + w (n - 1)))."""
    uvwl = np.ascontiguousarray(uvwl, np.float64)
    lm = np.ascontiguousarray(lm, np.float64)
    I = np.ascontiguousarray(np.asarray(I, np.complex128))
    out = np.empty(uvwl.shape[0], np.complex128)
    _c().oracle_dft_predict(uvwl.shape[0], _ptr(uvwl), lm.shape[0], _ptr(lm), _ptr(I), _ptr(out))
    return out


def dft_adjoint(uvwl: np.ndarray, vis: np.ndarray, lm: np.ndarray) -> np.ndarray:
    """Adjoint of dft_predict: D_p = sum_k V_k exp(+2 pi i (...))."""
    uvwl = np.ascontiguousarray(uvwl, np.float64)
    lm = np.ascontiguousarray(lm, np.float64)
    v = np.ascontiguousarray(np.asarray(vis, np.complex128))
    out = np.empty(lm.shape[0], np.complex128)
    _c().oracle_dft_adjoint(uvwl.shape[0], _ptr(uvwl), _ptr(v), lm.shape[0], _ptr(lm), _ptr(out))
    return out


def pixel_lm(N: int, dl: float, qx: np.ndarray, qy: np.ndarray) -> np.ndarray:
    """(l, m) of image pixels (qy, qx): l = (qx - N/2) dl, m = (qy - N/2) dl."""
    return np.stack([(np.asarray(qx) - N // 2) * dl, (np.asarray(qy) - N // 2) * dl], axis=-1).astype(np.float64)


def degrid_sampled(spec: KernelSpec, G: np.ndarray, co: Coords, idx) -> np.ndarray:
    """Degridding of selected visibilities only, one by one, each with just the
    kernel block of its own (bin, fine offset) synthesised (the same
    definition as `degrid`, for grids too large to tabulate every bin).
    Returns complex128 [len(idx)][npol]."""
    npol = spec.npol
    out = np.zeros((len(idx), npol), dtype=np.complex128)
    for n, k in enumerate(idx):
        if not co.valid[k]:
            continue
        b = int(co.bin[k])
        S = int(spec.supports[spec.plane_of(b)])
        K = synth_bin(spec, b, offsets_y=[int(co.fy[k])], offsets_x=[int(co.fx[k])])[0, 0]   # [S][S][P]
        x0, y0 = int(co.x0[k]), int(co.y0[k])
        win = np.asarray(G[:, y0:y0 + S, x0:x0 + S], dtype=np.complex128)                  # [s][S][S]
        Km = K.reshape(S, S, npol, npol)                                                      # [jy][jx][c][s]
        v = np.einsum("yxcs,syx->c", Km, win)
        if co.flip[k]:
            v = np.conj(v)
            if npol == 4:
                v = v[[0, 2, 1, 3]]
        out[n] = v
    return out
