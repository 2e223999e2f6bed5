"""Thin ctypes binding of libaw (include/aw.h) with the same function names.

Argument marshalling only: torch tensors are passed as device pointers, the
current torch CUDA stream as the cudaStream_t, and every step runs in the
library's CUDA kernels.  Loading fails loudly when libaw.so is missing or no
CUDA device is present; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
# AW_LIBAW selects another build of the library (the bounds-checked one in its test)
LIB_PATH = os.environ.get("AW_LIBAW") or os.path.join(HERE, "libaw.so")

AW_OK, AW_EINVAL, AW_ENOMEM, AW_ECUDA, AW_ETIMEOUT, AW_EUNSUPPORTED, AW_EREJECTED = range(7)
AW_ROLE_GRID, AW_ROLE_DEGRID, AW_ROLE_ADJOINT, AW_ROLE_BEAM = 0, 1, 2, 3
AW_STORAGE_FP32, AW_STORAGE_BF16, AW_STORAGE_FP16 = 0, 1, 2
AW_GRID_TILES, AW_GRID_OFFSETS, AW_GRID_HYBRID, AW_GRID_REGION = 0, 1, 2, 3
AW_INTERP_BILINEAR, AW_INTERP_CUBIC = 0, 1
AW_ENGINE_MMA_SYNC, AW_ENGINE_TCGEN05 = 0, 1
AW_TRAIN_FP32, AW_TRAIN_TCGEN05 = 0, 1
AW_FREQ_BIN, AW_FREQ_CHANNEL = 0, 1

c_i32, c_i64, c_dbl, c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class aw_kernel_spec(ctypes.Structure):
    _fields_ = [("N", c_i32), ("dl", c_dbl), ("OS", c_i32), ("W", c_dbl), ("npol", c_i32),
                ("nw", c_i32), ("w_max", c_dbl), ("supports", ctypes.POINTER(c_i32)),
                ("npa", c_i32), ("pa", ctypes.POINTER(c_dbl)), ("nfb", c_i32),
                ("fbin_freqs", ctypes.POINTER(c_dbl)), ("dish_d", c_dbl),
                ("d_xy", c_dbl * 2), ("d_yx", c_dbl * 2), ("eps", c_dbl), ("role", c_i32),
                ("storage", c_i32), ("point_l", c_dbl), ("point_m", c_dbl), ("ntype", c_i32),
                ("type_leak", ctypes.POINTER(c_dbl))]


class aw_kernel_info(ctypes.Structure):
    _fields_ = [("bytes", c_i64), ("nbins", c_i32), ("max_support", c_i32), ("npol", c_i32),
                ("role", c_i32), ("storage", c_i32), ("N", c_i32), ("OS", c_i32),
                ("n_rejected", c_i32)]


class aw_vis_desc(ctypes.Structure):
    _fields_ = [("nvis", c_i64), ("nrow", c_i64), ("nchan", c_i32), ("uvw", c_p),
                ("row_of_vis", c_p), ("chan_of_vis", c_p), ("freq", c_p), ("pa_bin", c_p),
                ("fbin", c_p), ("flags", c_p), ("row_types", c_p)]


class aw_tune(ctypes.Structure):
    _fields_ = [("tile", c_i32), ("chunk", c_i32), ("ctas_per_sm", c_i32), ("dg_tile", c_i32),
                ("grid_mode", c_i32), ("split_planes", c_i32)]


class aw_plan_info(ctypes.Structure):
    _fields_ = [("nvis", c_i64), ("nvalid", c_i64), ("n_outside", c_i64), ("n_flagged", c_i64),
                ("nitems", c_i64), ("tile", c_i32), ("chunk", c_i32), ("mean_taps", c_dbl),
                ("nitems_degrid", c_i64), ("grid_kernels", c_i32), ("region_lists", c_i32)]


class aw_sky_frame(ctypes.Structure):
    _fields_ = [("ra0", c_dbl), ("dec0", c_dbl), ("dl", c_dbl), ("cx", c_dbl), ("cy", c_dbl), ("N", c_i32),
                ("reserved", c_i32)]


def sky_frame(ra0: float, dec0: float, dl: float, N: int, cx: Optional[float] = None,
              cy: Optional[float] = None) -> aw_sky_frame:
    """SIN frame about (ra0, dec0); pixel (qx, qy) at l = (qx - cx) dl (cx, cy default N/2)."""
    return aw_sky_frame(float(ra0), float(dec0), float(dl), float(N // 2 if cx is None else cx),
                        float(N // 2 if cy is None else cy), int(N), 0)


class aw_clean_cfg(ctypes.Structure):
    _fields_ = [("n_major", c_i32), ("max_minor", c_i32), ("gain", ctypes.c_float), ("threshold", ctypes.c_float),
                ("cycle_factor", ctypes.c_float), ("patch_half", c_i32), ("window", c_i32 * 4)]


class aw_clean_report(ctypes.Structure):
    _fields_ = [("n_major", c_i32), ("n_minor", c_i32), ("peak_first", ctypes.c_float),
                ("peak_last", ctypes.c_float), ("sidelobe", ctypes.c_float), ("reserved", ctypes.c_float),
                ("weight_sum", c_dbl)]


class aw_stats(ctypes.Structure):
    _fields_ = [("n_gridded", c_i64), ("n_outside", c_i64), ("n_flagged", c_i64),
                ("n_nonfinite", c_i64), ("weight_sum", c_dbl)]


# name -> (restype, argtypes); the exported C ABI
SIGNATURES = {
    "aw_last_error": (ctypes.c_char_p, []),
    "aw_create": (ctypes.c_int, [ctypes.POINTER(c_p), ctypes.c_int]),
    "aw_destroy": (ctypes.c_int, [c_p]),
    "aw_make_kernels": (ctypes.c_int, [c_p, ctypes.POINTER(aw_kernel_spec), ctypes.POINTER(c_p), c_p]),
    "aw_kernel_set_import": (ctypes.c_int, [c_p, ctypes.POINTER(aw_kernel_spec), c_p, ctypes.POINTER(c_p), c_p]),
    "aw_kernel_set_export": (ctypes.c_int, [c_p, c_i32, c_p, c_p]),
    "aw_kernel_set_info": (ctypes.c_int, [c_p, ctypes.POINTER(aw_kernel_info)]),
    "aw_kernel_set_destroy": (ctypes.c_int, [c_p]),
    "aw_plan_create": (ctypes.c_int, [c_p, ctypes.POINTER(aw_vis_desc), c_p, ctypes.POINTER(aw_tune),
                                      ctypes.POINTER(c_p), c_p]),
    "aw_plan_query": (ctypes.c_int, [c_p, ctypes.POINTER(aw_plan_info)]),
    "aw_plan_destroy": (ctypes.c_int, [c_p]),
    "aw_plan_coords": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "aw_plan_order": (ctypes.c_int, [c_p, c_p, c_p]),
    "aw_grid": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, ctypes.POINTER(aw_stats), c_p]),
    "aw_degrid": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p]),
    "aw_grid_batched": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, ctypes.POINTER(aw_stats), c_p]),
    "aw_autotune": (ctypes.c_int, [c_p, ctypes.POINTER(aw_vis_desc), c_p, ctypes.POINTER(aw_tune), c_p]),
    "aw_fft_to_image": (ctypes.c_int, [c_p, c_p, c_p, c_dbl, c_p, c_p]),
    "mosaic_gamma": (ctypes.c_int, [c_p, c_p, c_i32, c_i32, ctypes.c_float, c_p, c_p]),
    "mosaic_gamma_noalloc": (ctypes.c_int, [c_p, c_i32, c_i32, ctypes.c_float, c_p, c_p]),
    "aw_image_to_grid": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p]),
    "aw_surrogate_set_engine": (ctypes.c_int, [c_p, c_i32]),
    "aw_surrogate_set_train_engine": (ctypes.c_int, [c_p, c_i32]),
    "aw_surrogate_set_freq_mode": (ctypes.c_int, [c_p, c_i32]),
    "aw_debug_fail_alloc": (ctypes.c_int, [c_i64]),
    "aw_debug_alloc_stats": (ctypes.c_int, [ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "aw_debug_wait_timeout": (ctypes.c_int, [c_p, c_i32, c_p]),
    "aw_debug_bounds_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint32), c_i32]),
    "aw_degrid_learned": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "aw_surrogate_save": (ctypes.c_int, [c_p, ctypes.c_char_p]),
    "aw_kernel_spec_hash": (ctypes.c_int, [ctypes.POINTER(aw_kernel_spec), ctypes.POINTER(ctypes.c_uint64)]),
    "aw_kernel_set_save": (ctypes.c_int, [c_p, ctypes.c_char_p]),
    "aw_kernel_set_load": (ctypes.c_int, [c_p, ctypes.c_char_p, ctypes.POINTER(c_p)]),
    "aw_surrogate_load": (ctypes.c_int, [c_p, ctypes.c_char_p, ctypes.POINTER(c_p)]),
    "aw_reproject": (ctypes.c_int, [c_p, c_p, ctypes.POINTER(aw_sky_frame), c_p, ctypes.POINTER(aw_sky_frame),
                                    c_i32, c_i32, ctypes.c_float, c_p]),
    "aw_mosaic_combine": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_i32, c_i32, c_i32, c_p, c_p]),
    "aw_phase_rotate": (ctypes.c_int, [c_p, ctypes.POINTER(aw_vis_desc), c_p, c_p, c_p, c_i32, c_dbl, c_dbl, c_dbl,
                                       c_dbl, c_p]),
    "aw_degrid_subtract": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "aw_psf_sidelobe": (ctypes.c_int, [c_p, c_p, c_i32, ctypes.POINTER(ctypes.c_float), c_p]),
    "aw_hogbom": (ctypes.c_int, [c_p, c_p, c_p, c_i32, c_i32, ctypes.c_float, ctypes.c_float, c_i32, c_i32,
                                 ctypes.POINTER(c_i32), c_p, ctypes.POINTER(c_i32), c_p]),
    "aw_clean": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, ctypes.POINTER(aw_clean_cfg), c_p, c_p, c_p,
                                ctypes.POINTER(aw_clean_report), c_p]),
    "aw_surrogate_create": (ctypes.c_int, [c_p, c_p, ctypes.POINTER(c_p)]),
    "aw_surrogate_destroy": (ctypes.c_int, [c_p]),
    "aw_surrogate_nparams": (ctypes.c_int, [c_p, ctypes.POINTER(c_i64)]),
    "aw_surrogate_set_params": (ctypes.c_int, [c_p, c_p]),
    "aw_surrogate_get_params": (ctypes.c_int, [c_p, c_p]),
    "aw_surrogate_forward": (ctypes.c_int, [c_p, c_p, c_p, c_i32, c_p, c_p]),
    "aw_surrogate_loss_grad": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_i32, ctypes.POINTER(c_dbl), c_p, c_p]),
    "aw_surrogate_train": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p]),
    "aw_surrogate_tables": (ctypes.c_int, [c_p, c_p, c_p, ctypes.c_float, c_i32, ctypes.POINTER(c_p), c_p, c_p]),
    "aw_grid_learned": (ctypes.c_int, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, ctypes.POINTER(aw_stats), c_p]),
}


class aw_surrogate_cfg(ctypes.Structure):
    _fields_ = [("npol", c_i32), ("width", c_i32), ("n_hidden", c_i32), ("omega0", ctypes.c_float),
                ("D", c_dbl), ("w_max", c_dbl), ("f_c", c_dbl), ("f_h", c_dbl), ("chi_c", c_dbl),
                ("chi_h", c_dbl), ("out_scale", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("norm_nw", c_i32), ("norm_supports", ctypes.POINTER(c_i32))]


class aw_train_cfg(ctypes.Structure):
    _fields_ = [("steps", c_i32), ("batch", c_i32), ("lr", ctypes.c_float), ("lr_final", ctypes.c_float),
                ("seed", ctypes.c_uint64)]


class aw_train_report(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float), ("steps", c_i32),
                ("seconds", c_dbl)]

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libaw.so and declare every exported function (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libaw.so is not built (%s): run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class AWError(RuntimeError):
    def __init__(self, code: int, fn: str, msg: str):
        super().__init__("%s failed with status %d: %s" % (fn, code, msg))
        self.code = code


def _check(rc: int, fn: str):
    if rc != AW_OK:
        raise AWError(rc, fn, (load().aw_last_error() or b"").decode())


def _stream(stream=None):
    import torch
    if stream is None:
        return c_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return c_p(stream)
    return c_p(stream.cuda_stream)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libaw needs a CUDA device; none is available")


# ---------------------------------------------------------------- context
class Handle:
    """Owns a library handle; keeps the tensors it refers to alive."""

    def __init__(self, ptr, destroy: str, keep=()):
        self.ptr = ptr
        self._destroy = destroy
        self._keep = list(keep)

    def close(self):
        if self.ptr:
            getattr(load(), self._destroy)(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def aw_create(device: int = 0) -> Handle:
    _require_cuda()
    out = c_p()
    _check(load().aw_create(ctypes.byref(out), device), "aw_create")
    return Handle(out, "aw_destroy")


def aw_destroy(ctx: Handle):
    ctx.close()


def make_spec(N: int, dl: float, OS: int, W: float = 7.0, npol: int = 1, nw: int = 1,
              w_max: float = 0.0, supports: Sequence[int] = (7,), pa: Sequence[float] = (0.0,),
              fbin_freqs: Sequence[float] = (1.4e9,), dish_d: float = 12.0, d_xy: complex = 0j,
              d_yx: complex = 0j, eps: float = 0.2, role: int = AW_ROLE_GRID,
              storage: int = AW_STORAGE_FP32, point_l: float = 0.0, point_m: float = 0.0,
              type_leak: Optional[Sequence] = None):
    """Build an aw_kernel_spec (returns (spec, keepalive)).  type_leak: per
    antenna type a (d_xy, d_yx) pair of complex leakages (per-baseline kernels)."""
    sup = (c_i32 * len(supports))(*[int(s) for s in supports])
    pa_arr = (c_dbl * len(pa))(*[float(x) for x in pa])
    fb_arr = (c_dbl * len(fbin_freqs))(*[float(x) for x in fbin_freqs])
    s = aw_kernel_spec()
    s.N, s.dl, s.OS, s.W, s.npol, s.nw, s.w_max = int(N), float(dl), int(OS), float(W), int(npol), int(nw), float(w_max)
    s.supports = ctypes.cast(sup, ctypes.POINTER(c_i32))
    s.npa = len(pa)
    s.pa = ctypes.cast(pa_arr, ctypes.POINTER(c_dbl))
    s.nfb = len(fbin_freqs)
    s.fbin_freqs = ctypes.cast(fb_arr, ctypes.POINTER(c_dbl))
    s.dish_d = float(dish_d)
    s.d_xy[0], s.d_xy[1] = complex(d_xy).real, complex(d_xy).imag
    s.d_yx[0], s.d_yx[1] = complex(d_yx).real, complex(d_yx).imag
    s.eps, s.role, s.storage = float(eps), int(role), int(storage)
    s.point_l, s.point_m = float(point_l), float(point_m)
    tl = None
    if type_leak:
        vals = []
        for dxy_t, dyx_t in type_leak:
            vals += [complex(dxy_t).real, complex(dxy_t).imag, complex(dyx_t).real, complex(dyx_t).imag]
        tl = (c_dbl * len(vals))(*vals)
        s.ntype = len(type_leak)
        s.type_leak = ctypes.cast(tl, ctypes.POINTER(c_dbl))
    return s, (sup, pa_arr, fb_arr, tl)


def aw_make_kernels(ctx: Handle, stream=None, **spec_kw) -> Handle:
    spec, keep = make_spec(**spec_kw)
    out = c_p()
    _check(load().aw_make_kernels(ctx.ptr, ctypes.byref(spec), ctypes.byref(out), _stream(stream)),
           "aw_make_kernels")
    return Handle(out, "aw_kernel_set_destroy")


def aw_kernel_set_import(ctx: Handle, tables, stream=None, **spec_kw) -> Handle:
    """tables: CUDA complex64 tensor holding all bins' blocks consecutively."""
    spec, keep = make_spec(**spec_kw)
    out = c_p()
    _check(load().aw_kernel_set_import(ctx.ptr, ctypes.byref(spec), _ptr(tables), ctypes.byref(out),
                                       _stream(stream)), "aw_kernel_set_import")
    return Handle(out, "aw_kernel_set_destroy")


def aw_kernel_set_info(kset: Handle) -> aw_kernel_info:
    info = aw_kernel_info()
    _check(load().aw_kernel_set_info(kset.ptr, ctypes.byref(info)), "aw_kernel_set_info")
    return info


def aw_kernel_set_export(kset: Handle, b: int, dst, stream=None):
    _check(load().aw_kernel_set_export(kset.ptr, int(b), _ptr(dst), _stream(stream)), "aw_kernel_set_export")


def aw_kernel_spec_hash(**spec_kw) -> int:
    spec, keep = make_spec(**spec_kw)
    h = ctypes.c_uint64()
    _check(load().aw_kernel_spec_hash(ctypes.byref(spec), ctypes.byref(h)), "aw_kernel_spec_hash")
    return h.value


def aw_kernel_set_save(kset: Handle, path: str):
    _check(load().aw_kernel_set_save(kset.ptr, os.fsencode(path)), "aw_kernel_set_save")


def aw_kernel_set_load(ctx: Handle, path: str) -> Handle:
    out = c_p()
    _check(load().aw_kernel_set_load(ctx.ptr, os.fsencode(path), ctypes.byref(out)), "aw_kernel_set_load")
    return Handle(out, "aw_kernel_set_destroy")


def cached_kernels(ctx: Handle, cache_dir: str, **spec_kw) -> Handle:
    """aw_make_kernels through an on-disk cache keyed by aw_kernel_spec_hash."""
    key = aw_kernel_spec_hash(**spec_kw)
    path = os.path.join(cache_dir, "awkset-%016x.bin" % key)
    if os.path.exists(path):
        return aw_kernel_set_load(ctx, path)
    ks = aw_make_kernels(ctx, **spec_kw)
    os.makedirs(cache_dir, exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    aw_kernel_set_save(ks, tmp)
    os.replace(tmp, path)
    return ks


def aw_kernel_set_destroy(kset: Handle):
    kset.close()


def vis_desc(uvw, row_of_vis, chan_of_vis, freq, pa_bin=None, fbin=None, flags=None,
             row_types=None) -> aw_vis_desc:
    d = aw_vis_desc()
    d.nvis = int(row_of_vis.numel())
    d.nrow = int(uvw.shape[0])
    d.nchan = int(freq.numel())
    d.uvw, d.row_of_vis, d.chan_of_vis, d.freq = _ptr(uvw), _ptr(row_of_vis), _ptr(chan_of_vis), _ptr(freq)
    d.pa_bin, d.fbin, d.flags = _ptr(pa_bin), _ptr(fbin), _ptr(flags)
    d.row_types = _ptr(row_types)
    d._keep = (uvw, row_of_vis, chan_of_vis, freq, pa_bin, fbin, flags, row_types)
    return d


def aw_plan_create(ctx: Handle, vis: aw_vis_desc, kset: Handle, tune: Optional[aw_tune] = None,
                   stream=None) -> Handle:
    out = c_p()
    _check(load().aw_plan_create(ctx.ptr, ctypes.byref(vis), kset.ptr,
                                 ctypes.byref(tune) if tune is not None else None, ctypes.byref(out),
                                 _stream(stream)), "aw_plan_create")
    return Handle(out, "aw_plan_destroy", keep=[vis, getattr(vis, "_keep", None)])


def aw_plan_query(plan: Handle) -> aw_plan_info:
    info = aw_plan_info()
    _check(load().aw_plan_query(plan.ptr, ctypes.byref(info)), "aw_plan_query")
    return info


def aw_plan_destroy(plan: Handle):
    plan.close()


def aw_plan_coords(plan: Handle, x0=None, y0=None, fx=None, fy=None, bin=None, flip=None, valid=None,
                   stream=None):
    _check(load().aw_plan_coords(plan.ptr, _ptr(x0), _ptr(y0), _ptr(fx), _ptr(fy), _ptr(bin), _ptr(flip),
                                 _ptr(valid), _stream(stream)), "aw_plan_coords")


def aw_plan_order(plan: Handle, perm, stream=None):
    _check(load().aw_plan_order(plan.ptr, _ptr(perm), _stream(stream)), "aw_plan_order")


def aw_grid(ctx: Handle, plan: Handle, kset: Handle, vis, weight, grid, want_stats: bool = False,
            stream=None) -> Optional[aw_stats]:
    st = aw_stats() if want_stats else None
    _check(load().aw_grid(ctx.ptr, plan.ptr, kset.ptr, _ptr(vis), _ptr(weight), _ptr(grid),
                          ctypes.byref(st) if st is not None else None, _stream(stream)), "aw_grid")
    return st


def aw_grid_batched(ctx: Handle, plan: Handle, kset: Handle, vis, weight, grid, want_stats: bool = False,
                    stream=None) -> Optional[aw_stats]:
    st = aw_stats() if want_stats else None
    _check(load().aw_grid_batched(ctx.ptr, plan.ptr, kset.ptr, _ptr(vis), _ptr(weight), _ptr(grid),
                                  ctypes.byref(st) if st is not None else None, _stream(stream)),
           "aw_grid_batched")
    return st


def aw_degrid(ctx: Handle, plan: Handle, kset: Handle, grid, vis_out, stream=None):
    _check(load().aw_degrid(ctx.ptr, plan.ptr, kset.ptr, _ptr(grid), _ptr(vis_out), _stream(stream)),
           "aw_degrid")


def aw_autotune(ctx: Handle, vis: aw_vis_desc, kset: Handle, stream=None) -> aw_tune:
    t = aw_tune()
    _check(load().aw_autotune(ctx.ptr, ctypes.byref(vis), kset.ptr, ctypes.byref(t), _stream(stream)),
           "aw_autotune")
    return t


def aw_fft_to_image(ctx: Handle, kset: Handle, grid, weight_sum: float, image, stream=None):
    _check(load().aw_fft_to_image(ctx.ptr, kset.ptr, _ptr(grid), float(weight_sum), _ptr(image),
                                  _stream(stream)), "aw_fft_to_image")


def mosaic_gamma(ctx: Handle, beams, eps: float, gamma, stream=None):
    nfield, N = int(beams.shape[0]), int(beams.shape[-1])
    _check(load().mosaic_gamma(ctx.ptr, _ptr(beams), nfield, N, ctypes.c_float(eps), _ptr(gamma),
                               _stream(stream)), "mosaic_gamma")


def mosaic_gamma_noalloc(beams, eps: float, gamma, stream=None):
    """mosaic_gamma without a context and without any device allocation (for
    callers that cannot allocate); see include/aw.h for the scratch rules."""
    nfield, N = int(beams.shape[0]), int(beams.shape[-1])
    _check(load().mosaic_gamma_noalloc(_ptr(beams), nfield, N, ctypes.c_float(eps), _ptr(gamma),
                                       _stream(stream)), "mosaic_gamma_noalloc")


def aw_image_to_grid(ctx: Handle, kset: Handle, image, grid, stream=None):
    _check(load().aw_image_to_grid(ctx.ptr, kset.ptr, _ptr(image), _ptr(grid), _stream(stream)), "aw_image_to_grid")


def aw_reproject(ctx: Handle, src, src_frame: aw_sky_frame, dst, dst_frame: aw_sky_frame,
                 interp: int = AW_INTERP_CUBIC, fill: float = 0.0, stream=None):
    """src: CUDA float [nplane][Ns][Ns] -> dst: CUDA float [nplane][Nd][Nd]."""
    nplane = int(src.shape[0])
    _check(load().aw_reproject(ctx.ptr, _ptr(src), ctypes.byref(src_frame), _ptr(dst), ctypes.byref(dst_frame),
                               nplane, int(interp), ctypes.c_float(fill), _stream(stream)), "aw_reproject")


def aw_phase_rotate(ctx: Handle, vd: aw_vis_desc, uvw_out, vis, vis_out, src_centre, dst_centre, stream=None):
    """uvw_out: CUDA float64 [nrow][3] or None; vis, vis_out: CUDA complex64 [nvis][npol]."""
    npol = int(vis.shape[1]) if vis is not None and vis.dim() == 2 else 1
    _check(load().aw_phase_rotate(ctx.ptr, ctypes.byref(vd), _ptr(uvw_out), _ptr(vis), _ptr(vis_out), npol,
                                  float(src_centre[0]), float(src_centre[1]), float(dst_centre[0]),
                                  float(dst_centre[1]), _stream(stream)), "aw_phase_rotate")


def aw_mosaic_combine(ctx: Handle, images, beams, gamma, out, stream=None):
    """images [nfield][nplane][N][N], beams [nfield][N][N], gamma [N][N] -> out [nplane][N][N]."""
    nfield, nplane, N = int(images.shape[0]), int(images.shape[1]), int(images.shape[-1])
    _check(load().aw_mosaic_combine(ctx.ptr, _ptr(images), _ptr(beams), _ptr(gamma), nfield, nplane, N, _ptr(out),
                                    _stream(stream)), "aw_mosaic_combine")


def aw_degrid_subtract(ctx: Handle, plan: Handle, kset: Handle, grid, vis, vis_out, stream=None):
    _check(load().aw_degrid_subtract(ctx.ptr, plan.ptr, kset.ptr, _ptr(grid), _ptr(vis), _ptr(vis_out),
                                     _stream(stream)), "aw_degrid_subtract")


def aw_psf_sidelobe(ctx: Handle, psf, stream=None) -> float:
    out = ctypes.c_float(0.0)
    _check(load().aw_psf_sidelobe(ctx.ptr, _ptr(psf), int(psf.shape[-1]), ctypes.byref(out), _stream(stream)),
           "aw_psf_sidelobe")
    return out.value


def aw_hogbom(ctx: Handle, residual, psf, gain: float, threshold: float, max_iter: int, patch_half: int,
              window, model, stream=None) -> int:
    """residual, model: CUDA float [npol][N][N] (updated); psf: CUDA float [N][N]."""
    npol, N = int(residual.shape[0]), int(residual.shape[-1])
    win = (c_i32 * 4)(*[int(x) for x in window])
    n = c_i32(0)
    _check(load().aw_hogbom(ctx.ptr, _ptr(residual), _ptr(psf), npol, N, ctypes.c_float(gain),
                            ctypes.c_float(threshold), int(max_iter), int(patch_half), win, _ptr(model),
                            ctypes.byref(n), _stream(stream)), "aw_hogbom")
    return n.value


def aw_clean(ctx: Handle, plan: Handle, kgrid: Handle, kdegrid: Handle, vis, weight, model, residual, psf,
             n_major: int, max_minor: int, gain: float, threshold: float, cycle_factor: float, patch_half: int,
             window=(0, 0, 0, 0), stream=None) -> aw_clean_report:
    cfg = aw_clean_cfg(n_major, max_minor, gain, threshold, cycle_factor, patch_half,
                       (c_i32 * 4)(*[int(x) for x in window]))
    rep = aw_clean_report()
    _check(load().aw_clean(ctx.ptr, plan.ptr, kgrid.ptr, kdegrid.ptr, _ptr(vis), _ptr(weight), ctypes.byref(cfg),
                           _ptr(model), _ptr(residual), _ptr(psf), ctypes.byref(rep), _stream(stream)), "aw_clean")
    return rep


def device_observation(ob, device="cuda:0", flags=None, row_types=None):
    """Copy a synthetic Observation's arrays to the device and describe them.

    Returns (aw_vis_desc, dict of tensors).  Row and channel indices are
    passed as int32 / int16 bit patterns of the uint32 / uint16 ABI types.
    row_types: optional host uint8 [nrow][2] antenna types of each row."""
    import numpy as np
    import torch

    def t(a, dt):
        return torch.as_tensor(np.ascontiguousarray(a), device=device).view(dt) if a is not None else None

    tens = {
        "uvw": torch.as_tensor(np.ascontiguousarray(ob.uvw, dtype=np.float64), device=device),
        "row": t(ob.row_of_vis.astype(np.uint32).view(np.int32), torch.int32),
        "chan": t(ob.chan_of_vis.astype(np.uint16).view(np.int16), torch.int16),
        "freq": torch.as_tensor(np.ascontiguousarray(ob.freq, dtype=np.float64), device=device),
        "pa_bin": t(ob.pa_bin.astype(np.uint8), torch.uint8),
        "fbin": t(ob.fbin.astype(np.uint8), torch.uint8),
        "flags": t(None if flags is None else flags.astype(np.uint8), torch.uint8),
        "row_types": t(None if row_types is None else np.asarray(row_types, np.uint8).reshape(-1, 2), torch.uint8),
    }
    d = vis_desc(tens["uvw"], tens["row"], tens["chan"], tens["freq"], tens["pa_bin"], tens["fbin"],
                 tens["flags"], tens["row_types"])
    return d, tens


# ---------------------------------------------------------------- learned surrogate
def aw_surrogate_create(ctx: Handle, npol: int = 4, width: int = 128, n_hidden: int = 4, omega0: float = 30.0,
                        D: float = 1.0, norm_supports=(8,), w_max: float = 1.0, f_c: float = 1.35e9,
                        f_h: float = 0.15e9, chi_c: float = 0.0, chi_h: float = 1.5, out_scale: float = 0.02,
                        seed: int = 1) -> Handle:
    ns = (c_i32 * len(norm_supports))(*[int(x) for x in norm_supports])
    c = aw_surrogate_cfg(int(npol), int(width), int(n_hidden), float(omega0), float(D), float(w_max),
                         float(f_c), float(f_h), float(chi_c), float(chi_h), float(out_scale), int(seed),
                         len(norm_supports), ctypes.cast(ns, ctypes.POINTER(c_i32)))
    out = c_p()
    _check(load().aw_surrogate_create(ctx.ptr, ctypes.byref(c), ctypes.byref(out)), "aw_surrogate_create")
    h = Handle(out, "aw_surrogate_destroy")
    h.cfg = c
    return h


def aw_surrogate_nparams(sur: Handle) -> int:
    n = c_i64()
    _check(load().aw_surrogate_nparams(sur.ptr, ctypes.byref(n)), "aw_surrogate_nparams")
    return int(n.value)


def aw_surrogate_set_params(sur: Handle, params):
    import numpy as np
    p = np.ascontiguousarray(params, dtype=np.float32)
    _check(load().aw_surrogate_set_params(sur.ptr, p.ctypes.data), "aw_surrogate_set_params")


def aw_surrogate_get_params(sur: Handle):
    import numpy as np
    p = np.empty(aw_surrogate_nparams(sur), dtype=np.float32)
    _check(load().aw_surrogate_get_params(sur.ptr, p.ctypes.data), "aw_surrogate_get_params")
    return p


def aw_surrogate_forward(ctx: Handle, sur: Handle, X, Y, stream=None):
    _check(load().aw_surrogate_forward(ctx.ptr, sur.ptr, _ptr(X), int(X.shape[0]), _ptr(Y), _stream(stream)),
           "aw_surrogate_forward")


def aw_surrogate_loss_grad(ctx: Handle, sur: Handle, X, T, grad, stream=None) -> float:
    loss = c_dbl()
    _check(load().aw_surrogate_loss_grad(ctx.ptr, sur.ptr, _ptr(X), _ptr(T), int(X.shape[0]), ctypes.byref(loss),
                                         _ptr(grad), _stream(stream)), "aw_surrogate_loss_grad")
    return float(loss.value)


def aw_surrogate_train(ctx: Handle, sur: Handle, exact: Handle, steps: int = 2000, batch: int = 65536,
                       lr: float = 1e-3, lr_final: float = 1e-5, seed: int = 7, stream=None) -> aw_train_report:
    c = aw_train_cfg(int(steps), int(batch), float(lr), float(lr_final), int(seed))
    rep = aw_train_report()
    _check(load().aw_surrogate_train(ctx.ptr, sur.ptr, exact.ptr, ctypes.byref(c), ctypes.byref(rep),
                                     _stream(stream)), "aw_surrogate_train")
    return rep


def aw_surrogate_tables(ctx: Handle, sur: Handle, exact: Handle, reject_rel: float, storage: int = AW_STORAGE_FP32,
                        stream=None):
    """Returns (kernel set handle, per-bin relative L2 errors, n_rejected bins)."""
    import numpy as np
    nb = aw_kernel_set_info(exact).nbins
    err = np.zeros(nb, dtype=np.float32)
    out = c_p()
    rc = load().aw_surrogate_tables(ctx.ptr, sur.ptr, exact.ptr, ctypes.c_float(reject_rel), int(storage),
                                    ctypes.byref(out), err.ctypes.data, _stream(stream))
    if rc not in (AW_OK, AW_EREJECTED):
        _check(rc, "aw_surrogate_tables")
    ks = Handle(out, "aw_kernel_set_destroy")
    return ks, err, aw_kernel_set_info(ks).n_rejected


def aw_surrogate_set_engine(sur: Handle, engine: int):
    _check(load().aw_surrogate_set_engine(sur.ptr, int(engine)), "aw_surrogate_set_engine")


def aw_surrogate_set_train_engine(sur: Handle, engine: int):
    _check(load().aw_surrogate_set_train_engine(sur.ptr, int(engine)), "aw_surrogate_set_train_engine")


def aw_degrid_learned(ctx: Handle, plan: Handle, sur: Handle, fallback: Handle, model, vis_out, stream=None):
    _check(load().aw_degrid_learned(ctx.ptr, plan.ptr, sur.ptr, fallback.ptr, _ptr(model), _ptr(vis_out),
                                    _stream(stream)), "aw_degrid_learned")


def aw_surrogate_set_freq_mode(sur: Handle, mode: int):
    _check(load().aw_surrogate_set_freq_mode(sur.ptr, int(mode)), "aw_surrogate_set_freq_mode")


def aw_surrogate_save(sur: Handle, path: str):
    _check(load().aw_surrogate_save(sur.ptr, os.fsencode(path)), "aw_surrogate_save")


def aw_surrogate_load(ctx: Handle, path: str) -> Handle:
    out = c_p()
    _check(load().aw_surrogate_load(ctx.ptr, os.fsencode(path), ctypes.byref(out)), "aw_surrogate_load")
    return Handle(out, "aw_surrogate_destroy")


def aw_grid_learned(ctx: Handle, plan: Handle, sur: Handle, fallback: Handle, vis, weight, grid,
                    want_stats: bool = False, stream=None) -> Optional[aw_stats]:
    st = aw_stats() if want_stats else None
    _check(load().aw_grid_learned(ctx.ptr, plan.ptr, sur.ptr, fallback.ptr, _ptr(vis), _ptr(weight), _ptr(grid),
                                  ctypes.byref(st) if st is not None else None, _stream(stream)), "aw_grid_learned")
    return st


def aw_debug_fail_alloc(n: int):
    _check(load().aw_debug_fail_alloc(int(n)), "aw_debug_fail_alloc")


def aw_debug_alloc_stats():
    """(live device buffers, device allocations attempted)"""
    live, calls = c_i64(), c_i64()
    _check(load().aw_debug_alloc_stats(ctypes.byref(live), ctypes.byref(calls)), "aw_debug_alloc_stats")
    return live.value, calls.value


def aw_debug_wait_timeout(ctx: Handle, which: int, stream=None) -> int:
    """Status code of the bounded-wait self-test (AW_ETIMEOUT is the expected outcome)."""
    return int(load().aw_debug_wait_timeout(ctx.ptr, int(which), _stream(stream)))


def aw_debug_bounds_status(reset: bool = False) -> int:
    """Code of the first failed bounds check (0: none); raises in a build without the checks."""
    st = ctypes.c_uint32()
    _check(load().aw_debug_bounds_status(ctypes.byref(st), int(bool(reset))), "aw_debug_bounds_status")
    return st.value
